"""Steady-state parity (Sec. "Kinetic Particle Simulation": averages after a
steady state; Sec. "Simulation Results", Figs. 5-9) of two discharges:

* the path the benchmark times, the 50 mm / 0.5 Pa / 300 V sputtering
  discharge reduced to 256 cells and 100k e- + 100k Ar+, 32-bit positions,
  sputtering on, TP steps of 40 PIC steps; the atoms in flight at the end
  continue to deposition;
* the 25 mm / 3 Pa / 100 V discharge, 128 cells, 20k e- + 20k Ar+, with
  64-bit and with 32-bit positions (the precision statement of the
  positions);
each 10 RF periods to settle, then 10 averaged.

The GPU runs 8 seeds (8001..8008) through the C ABI; the oracle's statistics
of 16 other seeds are stored in tests/golden/steady_state_*.json, written by
make_steady_state_ref.py from the oracle alone.  No seed is shared, so the
comparison is against the oracle's distribution, not a copy of one run:

* profiles -- the GPU mean against the oracle mean in relative L2.  For the
  potential, the densities and the ion flux the noise of that difference,
  sqrt(sigma_g^2 / 8 + sigma_o^2 / 16) summed over the nodes, is at most half
  the 3 % tolerance, and the test asserts that too; the electron flux, the
  test-particle density and moment, and the mean velocities (ratios of the
  averaged moments) have a seed-to-seed spread above that at this size, and
  are held to 3 times their noise (at least 3 %) instead;
* histograms -- two-sample KS between the pooled GPU and the pooled oracle
  histograms at a family-wise level of 1 % over the KS_TESTS comparisons of
  this module (each at p > 0.01 / KS_TESTS), with each run's sample size
  replaced by its
  effective number of independent samples, n_eff = 2 (0.8687 / D)^2 from the
  oracle's mean seed-to-seed KS distance D (0.8687 is the mean of the
  Kolmogorov distribution); for histograms of independent events n_eff is
  about the count, for the EEDF, whose samples repeat the same electrons
  every 10 steps, it is far smaller.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import kstwobign

from paper_1607_04069_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GPU_SEEDS = tuple(range(8001, 8009))
KS_MEAN = 0.8687                      # mean of the Kolmogorov distribution, sqrt(pi/2) ln 2
_RUNS = {}


def _ref(case):
    with open(os.path.join(HERE, "golden", f"steady_state_{case}.json")) as fh:
        return json.load(fh)


def _gpu_runs(case, prec):
    """8 GPU seeds of the case's discharge at the given position precision,
    run once per module and kept."""
    key = (case, prec)
    if key in _RUNS:
        return _RUNS[key]
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1607_04069_gb300 as P
    ref = _ref(case)
    runs = []
    for seed in GPU_SEEDS:
        if case == "ccp128":
            cfg = W.ccp_small(n_per_species=ref["n_per_species"], seed=seed)
        else:
            cfg = W.ccp_sputter(n_per_species=ref["n_per_species"], n_cells=ref["n_cells"], seed=seed)
            cfg.update(sort_every_e=400, sort_every_i=400, sort_every_tp=50)
        cfg["pos_precision"] = prec
        d = P.Discharge(P.params_from_workload(cfg))
        per = cfg["steps_per_period"]
        d.step(ref["warm_periods"] * per)
        d.sync()
        d.reset_averages()
        d.step(ref["avg_periods"] * per)
        d.sync()
        out = {k: d.diag(k) for k in ("phi", "n_e", "n_i", "gamma_e", "gamma_i", "tp_dens", "iedf_l", "iedf_r",
                                      "eedf", "ieadf_l", "ieadf_r")}
        # the TP v_x moment: tp_v is the mean velocity; the oracle stores the flux-like moment n <v_x>
        out["tp_vx"] = d.diag("tp_v") * out["tp_dens"]
        out["counters"] = d.counters()
        done, alive = 0, 1 if cfg["sputter_enable"] else 0
        while alive > 0 and done < ref["max_tp_steps"]:
            alive = d.tp_step(1000)
            done += 1000
        for k in ("sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r"):
            out[k] = d.diag(k)
        out["tp_left"] = alive
        d.close()
        runs.append(out)
    _RUNS[key] = runs
    return runs


CASES = [("sputter256", 32), ("ccp128", 64), ("ccp128", 32)]
IDS = ["sputter256_u32", "ccp128_f64", "ccp128_u32"]


def _marg(h, axis):
    return np.asarray(h).reshape(128, 90).sum(axis)


def _profile_check(ref, runs, k):
    g = np.array([r[k] for r in runs])
    gm, gs = g.mean(0), g.std(0, ddof=1)
    om, osd = np.array(ref["profiles"][k]["mean"]), np.array(ref["profiles"][k]["std"])
    ko = len(ref["seeds"])
    norm = np.linalg.norm(om)
    rel = float(np.linalg.norm(gm - om) / norm)
    noise = float(math.sqrt(np.sum(gs**2 / len(runs) + osd**2 / ko)) / norm)
    return rel, noise


@pytest.mark.parametrize("case,prec", CASES, ids=IDS)
@pytest.mark.parametrize("k", ["phi", "n_e", "n_i", "gamma_i"])
def test_profiles_within_3_percent(case, prec, k, record):
    ref, runs = _ref(case), _gpu_runs(case, prec)
    rel, noise = _profile_check(ref, runs, k)
    record(f"steady_state.{case}.u{prec}.{k}.rel_l2", rel)
    record(f"steady_state.{case}.u{prec}.{k}.noise", noise)
    assert noise <= 0.015, (k, noise)           # the run is sized so that 3 % is at least twice the noise
    assert rel < 0.03, (k, rel, noise)


@pytest.mark.parametrize("case,prec,k", [("sputter256", 32, "gamma_e"), ("sputter256", 32, "tp_dens"),
                                         ("sputter256", 32, "tp_vx"), ("ccp128", 64, "gamma_e"),
                                         ("ccp128", 32, "gamma_e")])
def test_noisy_profiles_within_their_noise(case, prec, k, record):
    ref, runs = _ref(case), _gpu_runs(case, prec)
    rel, noise = _profile_check(ref, runs, k)
    record(f"steady_state.{case}.u{prec}.{k}.rel_l2", rel)
    record(f"steady_state.{case}.u{prec}.{k}.noise", noise)
    assert rel < max(0.03, 3.0 * noise), (k, rel, noise)


@pytest.mark.parametrize("case,prec,flux,dens", [
    ("sputter256", 32, "gamma_e", "n_e"), ("sputter256", 32, "gamma_i", "n_i"),
    ("sputter256", 32, "tp_vx", "tp_dens"), ("ccp128", 64, "gamma_e", "n_e"), ("ccp128", 64, "gamma_i", "n_i")])
def test_mean_velocities(case, prec, flux, dens, record):
    """Mean velocity profiles (Fig. 8, Fig. 9): the averaged flux moment over
    the averaged density, on nodes where the density is above 5 % of its
    peak, against the oracle's within 3 times the combined noise of the two
    profiles (at least 3 %)."""
    ref, runs = _ref(case), _gpu_runs(case, prec)
    g = np.mean([r[flux] for r in runs], 0) / np.maximum(np.mean([r[dens] for r in runs], 0), 1e-300)
    om_f, om_n = np.array(ref["profiles"][flux]["mean"]), np.array(ref["profiles"][dens]["mean"])
    sel = om_n > 0.05 * om_n.max()
    o = om_f[sel] / om_n[sel]
    rel = float(np.linalg.norm(g[sel] - o) / np.linalg.norm(o))
    noise = math.hypot(_profile_check(ref, runs, flux)[1], _profile_check(ref, runs, dens)[1])
    record(f"steady_state.{case}.u{prec}.{flux}_over_{dens}.rel_l2", rel)
    assert rel < max(0.03, 3.0 * noise), (flux, rel, noise)


KS_SPUTTER = ["iedf_l", "iedf_r", "eedf", "ieadf_e_l", "ieadf_ang_l", "ieadf_e_r", "ieadf_ang_r", "sputter_e_l",
              "sputter_e_r", "sputter_ang_l", "sputter_ang_r"]
KS_CCP = ["iedf_l", "iedf_r", "eedf", "ieadf_e_l", "ieadf_ang_l", "ieadf_e_r", "ieadf_ang_r"]
KS_TESTS = len(KS_SPUTTER) + 2 * len(KS_CCP)
KS_ALPHA = 0.01 / KS_TESTS            # Bonferroni: 1 % family-wise over the module's KS comparisons


@pytest.mark.parametrize("case,prec,k", [("sputter256", 32, k) for k in KS_SPUTTER] +
                         [("ccp128", p, k) for p in (64, 32) for k in KS_CCP])
def test_distributions_ks(case, prec, k, record):
    ref, runs = _ref(case), _gpu_runs(case, prec)
    if k.startswith("ieadf_"):
        axis = 1 if "_e_" in k else 0
        g = sum(_marg(r["ieadf_" + k[-1]], axis) for r in runs)
    else:
        g = sum(r[k] for r in runs)
    h = ref["hists"][k]
    o = np.array(h["pooled"], dtype=float)
    D = float(np.abs(np.cumsum(g) / g.sum() - np.cumsum(o) / o.sum()).max())
    per_seed = h["per_seed_total_mean"]
    n_eff = min(per_seed, 2.0 * (KS_MEAN / h["pair_D_mean"]) ** 2)
    n1, n2 = n_eff * len(runs), n_eff * len(ref["seeds"])
    p = float(kstwobign.sf(D * math.sqrt(n1 * n2 / (n1 + n2))))
    record(f"steady_state.{case}.u{prec}.{k}.ks_p", p)
    assert g.sum() > 0.5 * len(runs) * per_seed and p > KS_ALPHA, (k, p, D, n_eff, g.sum())


def test_test_particles_deposited():
    """The continuation ran: at most as many atoms left in flight as the
    oracle's worst seed, plus a margin."""
    ref, runs = _ref("sputter256"), _gpu_runs("sputter256", 32)
    left = [r["tp_left"] for r in runs]
    assert min(left) >= 0 and max(left) <= ref["tp_left_max"] + 100, left
