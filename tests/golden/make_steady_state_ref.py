"""Writes the oracle's statistics of a discharge at periodic steady operation,
over many seeds, for the GPU steady-state parity tests:

* tests/golden/steady_state_sputter256.json (--case sputter256): the 50 mm /
  0.5 Pa / 300 V / 13.56 MHz sputtering case with 256 cells and 100k e- +
  100k Ar+ superparticles (sputtering on, TP steps of 40 PIC steps);
* tests/golden/steady_state_ccp128.json (--case ccp128): the 25 mm / 3 Pa /
  100 V case with 128 cells and 20k e- + 20k Ar+.

Only ``oracle/`` computes here.  From the uniform Maxwellian loading: 10 RF
periods to settle, then the time averages over 10 RF periods (Sec. "Kinetic
Particle Simulation": averaging after a steady state; Sec. "Simulation
Results", Figs. 5-9).  In the sputtering case the atoms still in flight at
the end then continue by TP steps until they deposit (at most MAX_TP_STEPS),
so that the deposited energy and angle distributions have thousands of
entries.

For every profile the file holds the mean over the seeds and the standard
deviation of one seed; for every histogram the pooled counts and the mean
two-sample KS distance between seeds (which gives the effective number of
independent samples of a correlated histogram).  The oracle source's hash is
recorded; a CPU test checks it against the current oracle.

Usage: python tests/golden/make_steady_state_ref.py [--case sputter256|ccp128]
[--seeds 16] [--workers N] (--quick writes a tiny run to --out, to try the
script).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = {"sputter256": dict(out="steady_state_sputter256.json", seed0=7001, n=100_000, cells=256, tp=True),
         "ccp128": dict(out="steady_state_ccp128.json", seed0=9001, n=20_000, cells=128, tp=False)}
WARM_PERIODS, AVG_PERIODS = 10, 10
MAX_TP_STEPS = 200_000
PROFILES = ("phi", "n_e", "n_i", "gamma_e", "gamma_i", "tp_dens", "tp_vx")
HISTS = ("iedf_l", "iedf_r", "eedf", "ieadf_l", "ieadf_r", "sputter_e_l", "sputter_e_r", "sputter_ang_l",
         "sputter_ang_r")


def workload(case: str, seed: int, n: int) -> dict:
    from paper_1607_04069_gb300 import workloads as W
    if case == "ccp128":
        return W.ccp_small(n_per_species=n, seed=seed)
    return W.ccp_sputter(n_per_species=n, n_cells=CASES[case]["cells"], seed=seed)


def oracle_hash() -> str:
    with open(os.path.join(ROOT, "oracle", "pic_oracle.c"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def run_seed(job) -> dict:
    """job = (case, seed, superparticles per species, steps of a settling and
    an averaging period block, settling periods, averaging periods, TP step
    cap)"""
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    case, seed, n_sp, P, warm, avg, max_tp = job
    cfg = workload(case, seed, n_sp)
    n = cfg["n_e0"]
    orc = O.Oracle(W.oracle_params(cfg), 2 * n, 2 * n, 400_000)
    orc.init_species(0, n, cfg["te0_ev"])
    orc.init_species(1, n, cfg["ti0_ev"])
    orc.field()
    t0 = time.time()
    orc.step(warm * P)
    orc.reset_averages()
    orc.step(avg * P)
    out = {k: orc.diag(k).tolist() for k in PROFILES + ("iedf_l", "iedf_r", "eedf", "ieadf_l", "ieadf_r")}
    c = orc.counters()
    out["counters"] = c
    # the atoms in flight continue by TP steps of the coupled length until they deposit
    tp_dt = cfg["tp_every"] * cfg["dt"]
    done = 0
    while cfg["sputter_enable"] and orc.counters()["n_tp"] > 0 and done < max_tp:
        orc.tp_step(1000, tp_dt)
        done += 1000
    for k in ("sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r"):
        out[k] = orc.diag(k).tolist()
    out["tp_steps_after"] = done
    out["tp_left"] = orc.counters()["n_tp"]
    out["seconds"] = time.time() - t0
    return out


def ks_D(x, y) -> float:
    x, y = np.asarray(x, float), np.asarray(y, float)
    if x.sum() == 0 or y.sum() == 0:
        return float("nan")
    return float(np.abs(np.cumsum(x) / x.sum() - np.cumsum(y) / y.sum()).max())


def marginals(h):
    a = np.asarray(h).reshape(128, 90)
    return a.sum(1), a.sum(0)


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="sputter256", choices=sorted(CASES))
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=None)
    ap.add_argument("--quick", action="store_true")
    opt = ap.parse_args()
    case = CASES[opt.case]
    out_path = opt.out or os.path.join(HERE, case["out"])
    seeds = [case["seed0"] + k for k in range(opt.seeds)]
    if opt.quick:
        jobs = [(opt.case, s, 2000, 30, 1, 1, 3000) for s in seeds]
    else:
        P = workload(opt.case, seeds[0], case["n"])["steps_per_period"]
        jobs = [(opt.case, s, case["n"], P, WARM_PERIODS, AVG_PERIODS, MAX_TP_STEPS) for s in seeds]
    with mp.get_context("spawn").Pool(min(opt.workers, len(jobs))) as pool:
        runs = pool.map(run_seed, jobs)
    n_seeds = len(seeds)
    ref = {"what": "oracle statistics of the reduced sputtering discharge, see make_steady_state_ref.py",
           "oracle_sha16": oracle_hash(), "case": opt.case, "seeds": seeds, "n_per_species": case["n"],
           "n_cells": case["cells"],
           "warm_periods": WARM_PERIODS, "avg_periods": AVG_PERIODS, "max_tp_steps": MAX_TP_STEPS,
           "profiles": {}, "hists": {}}
    for k in PROFILES:
        a = np.array([r[k] for r in runs])
        ref["profiles"][k] = {"mean": [float(f"{v:.9g}") for v in a.mean(0)],
                              "std": [float(f"{v:.6g}") for v in a.std(0, ddof=1)]}
    hists = {k: [np.asarray(r[k]) for r in runs] for k in HISTS}
    for el in "lr":
        m = [marginals(h) for h in hists["ieadf_" + el]]
        hists["ieadf_e_" + el] = [x[0] for x in m]
        hists["ieadf_ang_" + el] = [x[1] for x in m]
        del hists["ieadf_" + el]
    for k, hs in hists.items():
        D = [ks_D(a, b) for a, b in itertools.combinations(hs, 2)]
        ref["hists"][k] = {"pooled": [int(v) for v in np.sum(hs, axis=0)],
                           "per_seed_total_mean": float(np.mean([h.sum() for h in hs])),
                           "pair_D_mean": float(np.nanmean(D)) if np.isfinite(D).any() else None}
    ref["counters_mean"] = {k: float(np.mean([r["counters"][k] for r in runs])) for k in runs[0]["counters"]}
    ref["tp_left_max"] = int(max(r["tp_left"] for r in runs))
    ref["tp_steps_after_max"] = int(max(r["tp_steps_after"] for r in runs))
    ref["seconds_per_seed"] = float(np.mean([r["seconds"] for r in runs]))
    with open(out_path, "w") as fh:
        json.dump(ref, fh, separators=(",", ":"))
    print(f"wrote {out_path}: {n_seeds} seeds, {ref['seconds_per_seed']:.0f} s each, tp left {ref['tp_left_max']}")


if __name__ == "__main__":
    main()
