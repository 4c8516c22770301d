"""Shared helpers of the test suite (no step of the method lives here)."""
import numpy as np

import oracle as O
from paper_1607_04069_gb300 import workloads as W


def gpu_discharge(cfg, **over):
    import paper_1607_04069_gb300 as P
    c = dict(cfg)
    c.update(over)
    return P.Discharge(P.params_from_workload(c))


def oracle_for(cfg, cap=None, **over):
    c = dict(cfg)
    c.update(over)
    ne, ni = c.get("n_e0", 0), c.get("n_i0", 0)
    cap = cap or (2 * max(ne, ni) + 4096)
    return O.Oracle(W.oracle_params(c), cap, cap, c.get("cap_tp", 0) or 4 * cap)


def by_id(sp):
    order = np.argsort(sp["id"], kind="stable")
    return {k: v[order] for k, v in sp.items()}


def match(g, o):
    """Align two particle dicts by id; returns (g, o) restricted to common ids
    and the ids present on one side only."""
    g, o = by_id(g), by_id(o)
    common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
    only_g = np.setdiff1d(g["id"], o["id"])
    only_o = np.setdiff1d(o["id"], g["id"])
    return ({k: v[gi] for k, v in g.items()}, {k: v[oi] for k, v in o.items()}, only_g, only_o)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


DIAG_KEYS = ("phi", "n_e", "n_i", "gamma_e", "gamma_i", "eedf", "iedf_l", "iedf_r", "ieadf_l", "ieadf_r",
             "sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r", "tp_dens")


def oracle_averages(args):
    """One oracle discharge from the initial loading: ``warm`` steps, then the
    time averages over ``avg`` steps.  ``args`` = (cfg, warm, avg); returns the
    diagnostics of DIAG_KEYS and the counters.  A module-level function so
    that a spawn process pool can run several seeds at once."""
    cfg, warm, avg = args
    ne, ni = cfg["n_e0"], cfg["n_i0"]
    orc = O.Oracle(W.oracle_params(cfg), 2 * ne + 4096, 2 * ni + 4096, cfg.get("cap_tp", 0) or 4 * (ne + ni))
    orc.init_species(0, ne, cfg["te0_ev"])
    orc.init_species(1, ni, cfg["ti0_ev"])
    orc.field()
    orc.step(warm)
    orc.reset_averages()
    orc.step(avg)
    out = {k: orc.diag(k) for k in DIAG_KEYS}
    out["counters"] = orc.counters()
    return out


def oracle_pool_run(cfgs, warm, avg):
    """oracle_averages of several configurations in parallel (spawn pool)."""
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(len(cfgs), os.cpu_count() or 1)) as pool:
        return pool.map(oracle_averages, [(c, warm, avg) for c in cfgs])


def ks_hist(x, y):
    """Two-sample Kolmogorov-Smirnov test of two histograms over the same
    bins: (p-value, D, n1, n2)."""
    import math
    from scipy.stats import kstwobign
    n1, n2 = float(x.sum()), float(y.sum())
    D = float(np.abs(np.cumsum(x) / n1 - np.cumsum(y) / n2).max())
    return float(kstwobign.sf(D * math.sqrt(n1 * n2 / (n1 + n2)))), D, int(n1), int(n2)
