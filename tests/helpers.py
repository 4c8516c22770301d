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
