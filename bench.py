#!/usr/bin/env python
"""Benchmark of the PIC/MCC + test-particle hot path on GB300.

Workload (one GPU): the 50 mm / 1024-cell / 300 V / 0.5 Pa sputtering
discharge with 2M e- + 2M Ar+ superparticles (32-bit fixed-point positions,
FP32 velocities), sputtered Al atoms sub-cycled every 40 steps.  A step is
one PIC/MCC cycle of every particle (gather, push, wall + sputter launch,
null-collision MCC, int64 deposit, field solve), with the periodic
compaction and the coupled TP steps it schedules.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
same discharge instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Bytes the method moves per particle-step (read and write x, v_x, v_y, v_z; read the 8-byte id
# that keys the random stream): the roofline's algorithmic figure.
ALGO_BYTES = 40
# Bytes this design moves per particle-step: read x, v_x and the step of the next collision
# candidate, write x and v_x; v_y, v_z and the id are touched only by collisions and wall hits.
DESIGN_BYTES = 20
KERNEL_SOURCES = ["paper_1607_04069_gb300/csrc/pic_kernels.cu", "paper_1607_04069_gb300/csrc/common.cuh",
                  "paper_1607_04069_gb300/csrc/solve.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_copy_gbs", "hbm_GBps"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "fallback"


def traffic_per_launch():
    """dram bytes of one step-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "mover_traffic.json")) as fh:
            d = json.load(fh)
        if d.get("kernel_hash") == kernel_hash():
            return float(d["dram_bytes_per_launch_full_workload"])
    except (OSError, ValueError, KeyError):
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples: BENCH_CLOCKS_DIR if set, else the system's temporary directory
        out = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX)


def allreduce_sum(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.SUM)


def workload(n_per_species, seed):
    """The sputtering discharge.  With several ranks it is one discharge of
    ranks x n_per_species superparticles per species (the density kept by
    the weight), split over the ranks: each holds n_per_species of each."""
    from paper_1607_04069_gb300 import workloads as W
    cfg = W.ccp_sputter(n_per_species=n_per_species, seed=seed)
    # compaction every 400 steps: it restores the cell order the Ar+ deposit
    # profits from and removes the holes left by absorbed particles; electrons
    # lose their order within a few steps, so compacting them more often only
    # costs time
    cfg.update(sort_every_e=400, sort_every_i=400, sort_every_tp=50)
    return cfg


def host_cpu():
    """The host the CPU baseline ran on: logical CPUs and model name."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"host_cpus": os.cpu_count(), "cpu_model": model}


def extra_launches(cfg, h):
    """Kernels pic_step launches after the step kernel of host step h: a
    compaction (three kernels) of each species whose period ends there, and
    the coupled test-particle step (plus its own compaction) every tp_every
    steps."""
    n, h1 = 0, h + 1
    for every in (cfg.get("sort_every_e", 0), cfg.get("sort_every_i", 0)):
        if every > 0 and h1 % every == 0:
            n += 3
    te = cfg.get("tp_every", 0)
    if cfg.get("sputter_enable", 0) and te > 0 and h1 % te == 0:
        n += 1
        ste = cfg.get("sort_every_tp", 0)
        if ste > 0 and (h1 // te) % ste == 0:
            n += 3
    return n


def _oracle_all_cores_worker(cfg, n_sample, steps, barrier, out):
    """One process of oracle_rate_all_cores: build its sample, wait for the
    others, then time its steps on the wall clock."""
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    c = dict(cfg)
    c["weight"] = cfg["weight"] * cfg["n_e0"] / n_sample
    orc = O.Oracle(W.oracle_params(c), 2 * n_sample + 65536, 2 * n_sample + 65536, 65536)
    orc.init_species(0, n_sample, c["te0_ev"])
    orc.init_species(1, n_sample, c["ti0_ev"])
    orc.field()
    orc.step(1)
    barrier.wait(timeout=300)        # (a sibling that failed breaks it: this one ends too)
    t0 = time.time()
    orc.step(steps)
    t1 = time.time()
    cnt = orc.counters()
    out.put(((cnt["n_e"] + cnt["n_i"]) * steps, t0, t1))


def oracle_rate_all_cores(cfg, n_sample, steps, limit=180.0):
    """The oracle as it stands on every logical CPU of the host: one spawned
    process per CPU, each stepping its own sample of the same discharge, all
    started together; the rate is their particle-steps over the wall time
    from the first start to the last end.  None if a process failed or the
    run took longer than `limit` seconds."""
    import multiprocessing as mp
    import queue
    nproc = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(nproc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_all_cores_worker, args=(cfg, n_sample, steps, barrier, out))
             for _ in range(nproc)]
    for p in procs:
        p.start()
    res, deadline = [], time.time() + limit
    try:
        while len(res) < nproc and time.time() < deadline:
            try:
                res.append(out.get(timeout=1.0))
            except queue.Empty:
                if any(p.exitcode not in (None, 0) for p in procs):
                    break
    finally:
        for p in procs:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
                p.join()
    if len(res) < nproc:
        return None
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return sum(r[0] for r in res) / wall, nproc, wall


def oracle_rate(cfg, n_sample, steps, warmup=1):
    """FP64 oracle on a sample of the same discharge: n_sample superparticles
    per species with the weight scaled so the density is unchanged."""
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    c = dict(cfg)
    c["weight"] = cfg["weight"] * cfg["n_e0"] / n_sample
    orc = O.Oracle(W.oracle_params(c), 2 * n_sample + 65536, 2 * n_sample + 65536, 65536)
    orc.init_species(0, n_sample, c["te0_ev"])
    orc.init_species(1, n_sample, c["ti0_ev"])
    orc.field()
    orc.step(warmup)
    t0 = time.perf_counter()
    orc.step(steps)
    dt = time.perf_counter() - t0
    cnt = orc.counters()
    return (cnt["n_e"] + cnt["n_i"]) * steps / dt, dt


def tp_step_time(n_atoms, steps=20, warm=3):
    """Mean launch time (s) of the TP step on n_atoms atoms of the TP workload
    (thinned candidates), after warm steps, by the library's launch timers."""
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import workloads as W
    tc = W.tp_transport(n_atoms=n_atoms)
    tc.update(cap_tp=n_atoms + 1024, n_e0=0, n_i0=0, sort_every_tp=0)
    t = P.Discharge(P.params_from_workload(tc))
    t.tp_launch(n_atoms, 300.0)
    t.tp_step(warm, count_alive=False)
    t.sync()
    t.timing(True)
    t.tp_step(steps, count_alive=False)
    t.sync()
    ms, n = t.kernel_time("tp")
    t.close()
    return ms / n * 1e-3


def measure_rows(d, cfg, peak, cmp_ms, cmp_n, nsort_particles, n_atoms, want=None):
    """Per-row measurements besides the fused step kernel: test-particle flight
    (a separate run of n_atoms atoms, far larger than L2), compaction, and the
    FP64 field solve of the diagnostics.  want: the rows to measure (None: all)."""
    import torch
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import workloads as W
    rows = {}
    on = lambda name: want is None or name in want
    tc = W.tp_transport(n_atoms=n_atoms)
    tc.update(cap_tp=n_atoms + 1024, n_e0=0, n_i0=0, sort_every_tp=0)
    # a8: TP flight, one kernel per TP step
    per = tp_step_time(n_atoms) if on("a8_tp_step") else None
    # the method moves x, v_x, v_y, v_z (read and write) and reads the id per atom-step (40 B);
    # with thinned candidates this design reads x, v_x and the candidate step and writes x (16 B)
    ach = ALGO_BYTES * n_atoms / per / 1e9 if per else 0.0
    if per:
        rows["a8_tp_step"] = {"workload": "tp_transport: %d Al atoms, 0.5 Pa 300 K Ar, dt 1 ns, thinned "
                                          "collision candidates" % n_atoms,
                              "value": n_atoms / per, "unit": "atom-steps/s", "mean_launch_us": per * 1e6,
                              "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                           "frac": ach / peak, "algorithmic_bytes_per_atom_step": ALGO_BYTES,
                                           "design_bytes_per_atom_step": 16,
                                           "design_frac": 16 * n_atoms / per / 1e9 / peak}}
    # a8, event-driven form: the same source run to deposition, one launch per 32 events per atom
    if on("a8_tp_flight"):
        rows.update(measure_flights(tc, n_atoms))
    if on("n1_circuit_step"):
        rows["n1_circuit_step"] = measure_circuit(cfg)
    # a9: compaction (counting sort by cell of one species) in the timed run
    if cmp_n and on("a9_compaction"):
        per_sort = cmp_ms / cmp_n * 1e-3
        sb = 2 * 28 + 4       # read + write x, v_x, v_y, v_z, id, next-candidate step; one count pass
        ach = sb * nsort_particles / per_sort / 1e9
        rows["a9_compaction"] = {"value": nsort_particles / per_sort, "unit": "particles/s",
                                 "mean_sort_us": per_sort * 1e6,
                                 "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                              "frac": ach / peak, "algorithmic_bytes_per_particle": sb}}
    if on("cfg1_ccp_small"):
        rows["cfg1_ccp_small"] = measure_cfg1()
    if on("a7_poisson_fp64"):
        rows["a7_poisson_fp64"] = measure_poisson(d, cfg)
    return rows


def measure_flights(tc, n_atoms):
    """The TP source run to deposition by the event-driven flight, under hard
    spheres, VHS and M1."""
    import torch
    import paper_1607_04069_gb300 as P
    rows = {}
    t = P.Discharge(P.params_from_workload(tc))
    t.tp_launch(n_atoms, 300.0)
    t.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    left = t.tp_flight(10_000_000)
    wall_s = time.perf_counter() - t0
    cnt = t.counters()
    events = cnt["tp_coll"] + cnt["tp_dep_l"] + cnt["tp_dep_r"]
    rows["a8_tp_flight_to_deposition"] = {
        "workload": "tp_transport: %d Al atoms from 300 eV Ar+ impacts, 50 mm, 0.5 Pa 300 K Ar, event-driven "
                    "flight to deposition" % n_atoms,
        "value": events / wall_s, "unit": "atom-events/s", "seconds_to_deposition": wall_s,
        "events": int(events), "events_per_atom": events / n_atoms, "still_in_flight": int(left),
        "deposited_far": int(cnt["tp_dep_r"]), "deposited_source": int(cnt["tp_dep_l"])}
    t.close()
    # the same run under the VHS and M1 laws (argon's VHS data for the Al-Ar pair)
    for model, name in ((1, "vhs"), (2, "m1")):
        tv = dict(tc, tp_model=model, tp_dref=4.17e-10, tp_omega=0.81, tp_tref=273.0)
        t = P.Discharge(P.params_from_workload(tv))
        t.tp_launch(n_atoms, 300.0)
        t.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        left = t.tp_flight(10_000_000)
        wall_s = time.perf_counter() - t0
        cnt = t.counters()
        rows[f"a8_tp_flight_{name}_to_deposition"] = {
            "value": n_atoms / wall_s, "unit": "atoms deposited/s", "seconds_to_deposition": wall_s,
            "collisions_per_atom": cnt["tp_coll"] / n_atoms, "still_in_flight": int(left),
            "deposited_far": int(cnt["tp_dep_r"])}
        t.close()
    return rows


def measure_circuit(cfg):
    """NEXT-1: the step with the series capacitor against the ideal source."""
    import paper_1607_04069_gb300 as P
    per_launch = {}
    cb = 10.0 * 8.8541878128e-12 / cfg["gap_m"]
    for name, over in (("circuit", dict(circuit=1, c_block=cb)), ("ideal", {}),
                       ("two_harmonic_circuit", dict(waveform=1, rf_phase=0.0, circuit=1, c_block=cb))):
        dc = P.Discharge(P.params_from_workload(dict(cfg, **over)))
        dc.step(30)
        dc.sync()
        dc.timing(True)
        dc.step(300)
        dc.sync()
        ms, n = dc.kernel_time("step")
        c2 = dc.counters()
        dc.close()
        per_launch[name] = (ms / n * 1e-3, c2["n_e_slots"] + c2["n_i_slots"])
    per, slots = per_launch["circuit"]
    return {"workload": cfg["name"] + ", sine source through c = 10 eps0/L",
            "value": slots / per, "unit": "particle-steps/s", "mean_launch_us": per * 1e6,
            "ideal_source_mean_launch_us": per_launch["ideal"][0] * 1e6,
            "two_harmonic_circuit_mean_launch_us": per_launch["two_harmonic_circuit"][0] * 1e6,
            "note": "mean step launch by CUDA events, all without an L2 flush between steps; the "
                    "two-harmonic source peaks at 2 V0, so its electrons collide more often"}


def measure_cfg1():
    """The 25 mm / 128-cell discharge with 64-bit positions, 20 RF periods in
    full from the loading, and the oracle over the same 20 periods on one
    host core."""
    import torch
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import workloads as W
    sc = W.ccp_small()
    ds = P.Discharge(P.params_from_workload(sc))
    nsteps = sc["periods"] * sc["steps_per_period"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    ds.step(nsteps)
    e1.record()
    torch.cuda.synchronize()
    gpu_s = e0.elapsed_time(e1) * 1e-3
    cs = ds.counters()
    ds.close()
    n_avg = 0.5 * (sc["n_e0"] + sc["n_i0"] + cs["n_e_slots"] + cs["n_i_slots"])
    rate_o, sec_o = oracle_rate(dict(sc, weight=sc["weight"]), sc["n_e0"], nsteps, warmup=0)
    return {"workload": sc["name"] + ", 20 RF periods (8000 steps) from the loading",
            "value": n_avg * nsteps / gpu_s, "unit": "particle-steps/s", "gpu_s": gpu_s,
            "oracle_s": sec_o, "oracle_particle_steps_per_s": rate_o, "oracle_cores": 1,
            "note": "one launch per step, no L2 flush (the 40k-particle state is L2-resident); "
                    "slot counts include holes"}


def measure_poisson(d, cfg):
    """a7 (diagnostic form): the FP64 field solve of the current deposit, one CTA."""
    import torch
    import paper_1607_04069_gb300 as P
    f = d.get_field()
    qi = torch.tensor(f["q_i"], device="cuda")
    qe = torch.tensor(f["q_e"], device="cuda")
    dx = cfg["gap_m"] / cfg["n_cells"]
    for _ in range(3):
        P.op_poisson(qi, qe, cfg["n_cells"], dx, cfg["weight"], 0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        P.op_poisson(qi, qe, cfg["n_cells"], dx, cfg["weight"], 0.0)
    e1.record()
    torch.cuda.synchronize()
    return {"value": e0.elapsed_time(e1) / 20 * 1e3, "unit": "us per solve",
            "nodes": cfg["n_cells"] + 1, "bound": "latency (one CTA)"}


def measure_batched(n_discharges, steps, warmup, peak, run_periods=20):
    """The batched form: n_discharges independent discharges of uneven size
    (workloads.batched) stepped by one launch per step, against the plain
    loop that steps each of them alone.  Both are timed with CUDA events
    around every step of all members; the state (some 20 GB for 256
    members) is far larger than L2."""
    import torch
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import workloads as W
    cfgs = W.batched(n_discharges)
    n_part = sum(c["n_e0"] + c["n_i0"] for c in cfgs)
    stream = torch.cuda.current_stream()

    def timed(step_all):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, z in ev:
            a.record(stream)
            step_all()
            z.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(z) for a, z in ev) / steps

    plain = [P.Discharge(P.params_from_workload(c), stream=stream) for c in cfgs]

    def plain_step():
        for d in plain:
            d.step(1)

    for _ in range(warmup):
        plain_step()
    plain_ms = timed(plain_step)
    for d in plain:
        d.sync()
        d.close()
    del plain
    torch.cuda.synchronize()

    b = P.Batch(stream=stream)
    for c in cfgs:
        b.add(P.params_from_workload(c))
    best = b.autotune(steps_each=10)
    b.graphs(True)
    b.step(warmup + (-(warmup + 6 * 11)) % cfgs[0]["diag_every"])   # back onto the sampling grid
    batch_ms = timed(lambda: b.step(1))
    b.sync()
    # graph replay of whole sampling periods
    de = cfgs[0]["diag_every"]
    nblk = max(1, steps // de)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(nblk * de)
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / (nblk * de)
    b.sync()
    b.close()
    steps_per_run = run_periods * cfgs[0]["steps_per_period"]
    best_ms = min(batch_ms, graph_ms)
    ach = ALGO_BYTES * n_part / (best_ms * 1e-3) / 1e9
    return {"workload": f"{n_discharges} discharges, 256-2048 cells, 50k-2M per species (log-uniform), "
                        f"0.3-5 Pa, 50-500 V, dt = T_RF/{cfgs[0]['steps_per_period']}",
            "particles": n_part, "value": n_part / (best_ms * 1e-3), "unit": "particle-steps/s",
            "ms_per_step": best_ms, "ms_per_step_single_launch": batch_ms, "ms_per_step_graph": graph_ms,
            "plain_loop_ms_per_step": plain_ms, "plain_loop_particle_steps_per_s": n_part / (plain_ms * 1e-3),
            "speedup_vs_plain_loop": plain_ms / best_ms, "particles_per_cta": best,
            "discharges_per_hour_extrapolated": n_discharges * 3600.0 / (steps_per_run * best_ms * 1e-3),
            "plain_loop_discharges_per_hour_extrapolated": n_discharges * 3600.0 / (steps_per_run * plain_ms * 1e-3),
            "run_length": f"extrapolated: {run_periods} RF periods ({steps_per_run} steps) per discharge at the "
                          f"rate of {steps} timed steps",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "algorithmic_bytes_per_particle_step": ALGO_BYTES,
                         "design_frac": DESIGN_BYTES * n_part / (best_ms * 1e-3) / 1e9 / peak}}


def measure_served(n_requests, rate_hz, max_periods, tol=0.01, seed=1239, criterion="inventory", window=1):
    """The served form: a Poisson stream of discharge requests drawn from the
    batched workload's ranges, each run to periodic steady state (relative
    period-to-period change of the cycle-averaged n_e and n_i below tol, at
    most max_periods RF periods) by the library's request loop, once with
    the batched worker and once with the plain loop of pic_step calls.
    Latency is completion minus arrival on the server's clock."""
    import numpy as np
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import workloads as W
    cfgs = W.batched(n_requests, seed=seed)
    arrivals = W.poisson_arrivals(rate_hz, n_requests, seed)
    out = {}
    crit = {"inventory": 0, "profile": 1}[criterion]
    for mode, batched in (("batched", 1), ("plain_loop", 0)):
        srv = P.Server(batched=batched, max_periods=max_periods, tol=tol, criterion=crit, window_periods=window)
        t0 = srv.clock()
        ids = []
        for c, a in zip(cfgs, arrivals):
            while srv.clock() < t0 + a:
                time.sleep(min(0.005, max(0.0, t0 + a - srv.clock())))
            ids.append(srv.submit(P.params_from_workload(c), t0 + a))
        infos = [srv.wait(i) for i in ids]
        errors = sorted({srv.error(i) for i, info in zip(ids, infos) if info["state"] in ("failed", "rejected")})
        st = srv.stats()
        srv.close()
        lat = np.array([i["t_done"] - i["t_arrival"] for i in infos])
        ok = [i for i in infos if i["state"] in ("converged", "max_periods")]
        span = max(i["t_done"] for i in infos) - (t0 + arrivals[0])
        out[mode] = {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                     "discharges_per_hour": len(ok) * 3600.0 / span, "span_s": span,
                     "converged": sum(i["state"] == "converged" for i in infos),
                     "hit_max_periods": sum(i["state"] == "max_periods" for i in infos),
                     "failed": len(infos) - len(ok), "failure_reasons": errors,
                     "periods_mean": float(np.mean([i["periods"] for i in infos])),
                     "last_change_median": float(np.median([i["change"] for i in infos])),
                     "particle_steps_per_s_busy": st["particle_steps"] / max(st["busy_s"], 1e-9)}
    b, l = out["batched"], out["plain_loop"]
    measure = ("relative L2 change of the window-averaged n_e and n_i profiles" if criterion == "profile"
               else "relative change of the window-averaged e- and Ar+ inventories")
    return {"workload": f"{n_requests} requests, Poisson arrivals at {rate_hz:g}/s, sizes and conditions drawn "
                        f"as in the batched workload, each run to steady state ({measure} < {tol:g} between "
                        f"windows of {window} RF periods, at most {max_periods} periods)",
            "criterion": criterion, "window_periods": window, "max_periods": max_periods,
            "value": b["discharges_per_hour"], "unit": "discharges/hour",
            "p50_latency_s": b["p50_latency_s"], "p99_latency_s": b["p99_latency_s"],
            "speedup_vs_plain_loop": b["discharges_per_hour"] / l["discharges_per_hour"],
            "batched": b, "plain_loop": l}


def line_config(cfg, ws, n_per_species):
    """The workload's description, the same in both arms' lines."""
    return {"workload": cfg["name"], "particles_per_gpu": 2 * n_per_species, "n_cells": cfg["n_cells"],
            "sort_every": [cfg["sort_every_e"], cfg["sort_every_i"]], "tp_every": cfg["tp_every"],
            "parallelism": f"one discharge split over {ws} gpus (int64 deposit all-reduce per step)" if ws > 1
                           else "1 gpu",
            "l2": "flushed before every timed step (512 MiB write, then a 256 MiB read)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cfg = workload(args.n_per_species, 1236)
    # bounded sample: about 3e9 particle-steps in all (some 20 s on one core), so any
    # --steps ends within minutes
    n_sample = max(2000, min(args.ref_sample, int(1.5e9 / max(args.steps + args.warmup, 1))))
    rate, dt = oracle_rate(cfg, n_sample, args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": "particle-steps/s", "value": rate, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": line_config(cfg, args.gpus, args.n_per_species),
            "cpu_baseline": {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", **host_cpu(),
                             "sample": f"{n_sample}+{n_sample} superparticles of the same discharge "
                                       f"(weight x{cfg['n_e0'] / n_sample:g}), {args.steps} full steps"},
            "e2e": {"value": rate, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(d, stream, k_steps, flush, clean):
    """k_steps steps, each after an L2 flush and bracketed by CUDA events on
    the step's stream; returns the per-step times (ms)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
    torch.cuda.synchronize()
    for k in range(k_steps):
        flush.zero_()
        clean.max()
        starts[k].record(stream)
        d.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-per-species", type=int, default=2_000_000)
    ap.add_argument("--ref-sample", type=int, default=2_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--no-rows", action="store_true")
    ap.add_argument("--rows", default="all",
                    help="comma-separated rows to measure (a8_tp_step, a8_tp_flight, n1_circuit_step, "
                         "a9_compaction, cfg1_ccp_small, a7_poisson_fp64, b_batched, c_served) or all")
    ap.add_argument("--tp-step-only", type=int, default=0,
                    help="time only the TP step on this many atoms (profiling runs) and print it")
    ap.add_argument("--tp-atoms", type=int, default=100_000_000)
    ap.add_argument("--batch-discharges", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=4.0)
    ap.add_argument("--serve-max-periods", type=int, default=20)
    ap.add_argument("--serve-criterion", default="inventory", choices=["inventory", "profile"])
    ap.add_argument("--serve-window", type=int, default=1)
    ap.add_argument("--settle-periods", type=int, default=10,
                    help="after the other measurements, step the discharge to this many RF periods and time "
                         "600 more steps the same way (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch

    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import shard

    torch.cuda.set_device(local)
    if args.tp_step_only > 0:
        per = tp_step_time(args.tp_step_only)
        print(json.dumps({"tp_step_atoms": args.tp_step_only, "mean_launch_us": per * 1e6}), flush=True)
        return
    # one discharge; with several ranks its superparticles are split over them
    cfg_all = workload(args.n_per_species * ws, 1236)
    cfg = shard.shard_workload(cfg_all, rank, ws)
    stream = torch.cuda.current_stream()
    sd = shard.SplitDischarge(cfg_all, rank, ws, stream=stream)
    d = sd if ws > 1 else sd.d
    d.step(args.warmup)
    sd.sync()
    n_start = sd.alive() // ws
    # L2 flush between timed steps: write 512 MiB (> 129 MB L2), then read a
    # separate 256 MiB buffer so the flush's dirty lines are written back
    # before the step starts (the L2 then holds neither the state nor dirty data)
    flush = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")
    clean = torch.ones(64 * 2**20, dtype=torch.int32, device="cuda")
    # the library's per-launch timers stay off here: their event records would
    # add to every timed step; the step kernel's launch time is read from the
    # per-step events of the steps that launch nothing else
    with Clocks(local) as clk:
        barrier(ws)
        t0 = time.perf_counter()
        times = timed_steps(d, stream, args.steps, flush, clean)
        barrier(ws)
        wall = time.perf_counter() - t0
    sd.sync()
    n_end = sd.alive() // ws
    step_ms = sum(times)
    extra = [extra_launches(cfg, args.warmup + k) for k in range(args.steps)]
    alone = [t for t, x in zip(times, extra) if x == 0]
    mover_ms, mover_n = sum(alone), len(alone)
    launches = args.steps + sum(extra)
    t_max = allreduce_max(step_ms, ws)
    psteps = allreduce_sum(0.5 * (n_start + n_end) * args.steps, ws)
    value = psteps / (t_max * 1e-3)
    # one whole schedule of 400 steps (a compaction of each species, ten coupled
    # test-particle steps), timed the same way: the schedule-weighted step time
    h0 = args.warmup + args.steps
    sched = timed_steps(d, stream, 400, flush, clean)
    sd.sync()
    n_sched = sd.alive() // ws
    sched_ms = allreduce_max(sum(sched), ws)
    sched_value = allreduce_sum(0.5 * (n_end + n_sched) * 400, ws) / (sched_ms * 1e-3)
    # the library's timers on a further 400 steps: the compaction and TP launch
    # times, and a check of the launch schedule counted above
    sd.d.timing(True)
    d.step(400)
    sd.sync()
    _, chk_mover = sd.d.kernel_time("step")
    tp_ms, tp_n = sd.d.kernel_time("tp")
    cmp_ms, cmp_n = sd.d.kernel_time("compact")
    sd.d.timing(False)
    want = sum(extra_launches(cfg, h0 + 400 + k) for k in range(400))
    if chk_mover != 400 or tp_n + 3 * cmp_n != want:
        raise RuntimeError(f"launch schedule: {tp_n} TP and {cmp_n} compaction launches, {want} kernels expected")

    # roofline of the per-step kernel: algorithmic bytes / mean launch time
    peak, peak_kind = hbm_peak()
    per_launch_s = mover_ms / max(mover_n, 1) * 1e-3
    nmid = 0.5 * (n_start + n_end)
    achieved = ALGO_BYTES * nmid / per_launch_s / 1e9
    traffic = traffic_per_launch()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_mover (fused gather/push/wall/MCC/deposit, per-CTA field solve)",
                "algorithmic_bytes_per_particle_step": ALGO_BYTES, "peak_source": peak_kind,
                "design_bytes_per_particle_step": DESIGN_BYTES,
                "design_frac": DESIGN_BYTES * nmid / per_launch_s / 1e9 / peak,
                "dram_frac": (traffic / per_launch_s / 1e9 / peak) if traffic else None,
                "mean_launch_us": per_launch_s * 1e6}

    # end to end through the public API: pinned host state -> device, steps, diagnostics -> host
    e2e = None
    if args.e2e_steps > 0:
        sp = {s: sd.d.get_species(s) for s in (0, 1)}
        pinned = {}
        for s in (0, 1):
            n = len(sp[s]["id"])
            pos = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
            pos[:] = np.rint(sp[s]["xi"] * (2.0**32 / cfg["n_cells"])).astype(np.uint64).astype(np.uint32)
            arrs = []
            for k in ("vx", "vy", "vz"):
                a = torch.empty(n, dtype=torch.float32, pin_memory=True).numpy()
                a[:] = sp[s][k]
                arrs.append(a)
            ids = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
            ids[:] = sp[s]["id"]
            pinned[s] = (pos, *arrs, ids)
        h2d = sum(sum(a.nbytes for a in pinned[s]) for s in (0, 1))
        cap = max(len(pinned[s][0]) for s in (0, 1)) * 5 // 4 + 65536
        d2 = P.Discharge(P.params_from_workload(cfg, n_e0=0, n_i0=0, cap_e=cap, cap_i=cap), stream=stream)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in (0, 1):
            d2.set_species(s, *pinned[s])
        if ws > 1:
            shard.allreduce_(d2.exchange_slot())
        for _ in range(args.e2e_steps):
            d2.step(1)
            if ws > 1:
                shard.allreduce_(d2.exchange_slot())
        out = [d2.diag(k) for k in ("phi", "n_e", "n_i", "iedf_l")]
        cnt = d2.counters()
        torch.cuda.synchronize()
        e2e_wall = allreduce_max(time.perf_counter() - t0, ws)
        d2h = sum(a.nbytes for a in out) + 8 * len(cnt)
        n_e2e = allreduce_sum(sum(len(pinned[s][0]) for s in (0, 1)) * args.e2e_steps, ws)
        e2e = {"value": n_e2e / e2e_wall, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d / args.e2e_steps, "d2h_bytes_per_step": d2h / args.e2e_steps,
               "steps": args.e2e_steps, "note": "pinned host state uploaded, steps run, diagnostics read back"}
        d2.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n_sample, nst = cfg["n_e0"], 400            # the full discharge, 400 steps: some 10-20 s
        rate, dt = oracle_rate(cfg, n_sample, nst)
        cpu = {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", **host_cpu(),
               "sample": f"{n_sample}+{n_sample} superparticles of the same discharge, "
                         f"{nst} full PIC/MCC steps in {dt:.1f} s"}
        # the same oracle on every logical CPU (one process each), for context
        n_all, st_all = 1_000_000, 100           # samples far larger than a core's caches
        r = oracle_rate_all_cores(cfg, n_all, st_all)
        if r is not None:
            r_all, nproc, wall = r
            cpu["all_cores"] = {"value": r_all, "unit": "particle-steps/s", "processes": nproc,
                                "sample": f"{nproc} processes, each {n_all}+{n_all} superparticles of the same "
                                          f"discharge for {st_all} steps, {wall:.1f} s wall"}
    clocks = clk.summary()
    rows = None
    want = None if args.rows == "all" else set(args.rows.split(","))
    if rank == 0 and not args.no_rows:
        rows = measure_rows(sd.d, cfg, peak, cmp_ms, cmp_n, 0.25 * (n_start + n_end), args.tp_atoms, want)
        if args.batch_discharges > 0 and (want is None or "b_batched" in want):
            rows["b_batched"] = measure_batched(args.batch_discharges, 30, 10, peak)
        if args.serve_requests > 0 and (want is None or "c_served" in want):
            rows["c_served"] = measure_served(args.serve_requests, args.serve_rate, args.serve_max_periods,
                                              criterion=args.serve_criterion, window=args.serve_window)
    # the same discharge at steady operation: stepped on to settle_periods RF periods
    # from its loading, then 600 steps timed as above (its particle count has decayed
    # from the 2M + 2M of the loading)
    settled = None
    done = args.warmup + args.steps + 400 + 400
    target = args.settle_periods * cfg["steps_per_period"]
    if args.settle_periods > 0 and target > done:
        d.step(target - done)
        sd.sync()
        n_s0 = sd.alive() // ws
        st_ms = allreduce_max(sum(timed_steps(d, stream, 600, flush, clean)), ws)
        sd.sync()
        n_s1 = sd.alive() // ws
        settled = {"periods_before": args.settle_periods, "ms_per_step": st_ms / 600,
                   "value": allreduce_sum(0.5 * (n_s0 + n_s1) * 600, ws) / (st_ms * 1e-3),
                   "particles_per_gpu": int(0.5 * (n_s0 + n_s1)),
                   "note": "600 steps timed as the headline after the discharge ran this many RF periods "
                           "from its loading"}
    if rank == 0:
        line = {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": line_config(cfg_all, ws, args.n_per_species),
                "timing": "value from per-step CUDA events after an L2 flush each; the step kernel's "
                          "launch time from those of the steps that launch nothing else",
                "wall_s_incl_flush": wall, "particles_start_end_per_gpu": [int(n_start), int(n_end)],
                "schedule_400": {"ms_per_step": sched_ms / 400, "value": sched_value,
                                 "note": "400 further steps timed the same way: one compaction of each "
                                         "species and ten coupled test-particle steps fall inside"},
                "settled": settled,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches), "rows": rows,
                "kernel_us": {"step_alone_mean": mover_ms / max(mover_n, 1) * 1e3, "steps_alone": mover_n,
                              "tp_mean": tp_ms / max(tp_n, 1) * 1e3,
                              "compact_mean": cmp_ms / max(cmp_n, 1) * 1e3}}
        print(json.dumps(line), flush=True)
    sd.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
