"""The workload's shards split over ranks (paper_1607_04069_gb300.shard), on
CPU with two gloo ranks.  The oracle stands in for each rank's engine; the
split, the per-step exchange and the sums are the product's.

* A discharge whose superparticles are split over two ranks, with the int64
  deposits summed after every step (Sec. "Charge Assignment", "EM Field
  Solver"), equals the one-rank discharge: the time-averaged potential and
  densities bit for bit, the summed histograms and event counts bit for bit,
  the summed flux moments to rounding.
* A test-particle source split over two ranks (disjoint id ranges) deposits
  the same atoms as the whole source: histograms and counts bit for bit.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HIST = ("iedf_l", "iedf_r", "eedf", "ieadf_l", "ieadf_r", "sputter_e_l", "sputter_e_r", "sputter_ang_l",
        "sputter_ang_r")
COUNTS = ("imp_e_l", "imp_e_r", "imp_i_l", "imp_i_r", "ionizations", "sputtered_l", "sputtered_r", "tp_dep_l",
          "tp_dep_r", "elastic", "excitation", "cx", "iso", "tp_coll", "n_e", "n_i", "n_tp")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _discharge_cfg():
    sys.path.insert(0, ROOT)
    from paper_1607_04069_gb300 import workloads as W
    cfg = W.ccp_sputter(n_per_species=6000, n_cells=64, seed=91)
    cfg.update(rf_volt_v=1000.0, dt=W.T_RF / 400, tp_every=20)   # sputtering within a short run
    return cfg


def _run_discharge(cfg, first, count, exchange, steps):
    """The oracle on particles first .. first + count - 1 of cfg's loading;
    exchange(q) returns the deposit summed over the ranks."""
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    n = cfg["n_e0"]
    orc = O.Oracle(W.oracle_params(cfg), 2 * n, 2 * n, 8 * n)
    orc.init_species(0, count, cfg["te0_ev"], first=first)
    orc.init_species(1, count, cfg["ti0_ev"], first=first)

    def sync_deposit():
        f = orc.get_field()
        q = exchange(np.stack([f["q_e"], f["q_i"]]))
        orc.set_deposit(q[0], q[1])

    orc.field()
    sync_deposit()
    orc.solve()
    for _ in range(steps // 2):
        orc.step_particles()
        sync_deposit()
        orc.step_field()
    orc.reset_averages()
    for _ in range(steps - steps // 2):
        orc.step_particles()
        sync_deposit()
        orc.step_field()
    out = {k: orc.diag(k) for k in HIST + ("phi", "n_e", "n_i", "gamma_e", "gamma_i", "tp_dens")}
    c = orc.counters()
    out["counts"] = np.array([c[k] for k in COUNTS], dtype=np.int64)
    return out


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1607_04069_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _discharge_cfg()
    part = shard.shard_workload(cfg, rank, world)

    def exchange(qq):
        return shard.allreduce_(torch.from_numpy(qq.copy())).numpy()

    res = _run_discharge(cfg, part["id_offset"], part["n_e0"], exchange, 1600)
    summed = {k: shard.sum_host(res[k]) for k in HIST + ("gamma_e", "gamma_i", "tp_dens", "counts")}
    # a TP source split over the ranks: disjoint id ranges, histograms summed at the end
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    tc = W.tp_transport(n_atoms=6000)
    first, count = shard.part(6000, rank, world)
    orc = O.Oracle(W.oracle_params(tc), 1, 1, 6000)
    orc.tp_launch(count, 300.0, first_id=first)
    orc.tp_step(3000, 4e-9)
    c = orc.counters()
    tp = {k: shard.sum_host(orc.diag(k)) for k in ("sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r")}
    tp["counts"] = shard.sum_host(np.array([c["tp_dep_l"], c["tp_dep_r"], c["tp_coll"], c["n_tp"]], dtype=np.int64))
    dist.destroy_process_group()
    q.put((rank, {k: res[k] for k in ("phi", "n_e", "n_i")}, summed, tp))


def test_part_covers_every_index_once():
    sys.path.insert(0, ROOT)
    from paper_1607_04069_gb300 import shard
    for n in (0, 1, 7, 1000, 2_000_001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, c = shard.part(n, r, world)
                assert c >= 0
                seen.extend(range(a, a + c))
                assert list(shard.members(n, r, world)) == list(range(a, a + c))
            assert seen == list(range(n))


def test_split_runs_equal_the_one_rank_runs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in (0, 1)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, prof, summed, tp = q.get(timeout=600)
        got[r] = (prof, summed, tp)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = _discharge_cfg()
    whole = _run_discharge(cfg, 0, cfg["n_e0"], lambda qq: qq, 1600)
    for r in (0, 1):
        prof, summed, _ = got[r]
        for k in ("phi", "n_e", "n_i"):                      # global on every rank, bit for bit
            assert np.array_equal(prof[k], whole[k]), (r, k)
        for k in HIST:
            assert np.array_equal(summed[k], whole[k]), (r, k)
        assert np.array_equal(summed["counts"], whole["counts"]), (r, summed["counts"], whole["counts"])
        for k in ("gamma_e", "gamma_i", "tp_dens"):          # sums of per-rank moments: rounding only
            assert np.allclose(summed[k], whole[k], rtol=1e-12, atol=1e-12 * np.abs(whole[k]).max()), k
    c = dict(zip(COUNTS, whole["counts"].tolist()))
    assert c["sputtered_l"] + c["sputtered_r"] > 100 and c["ionizations"] > 100 and c["tp_coll"] > 0
    # the split TP source
    import oracle as O
    from paper_1607_04069_gb300 import workloads as W
    tc = W.tp_transport(n_atoms=6000)
    orc = O.Oracle(W.oracle_params(tc), 1, 1, 6000)
    orc.tp_launch(6000, 300.0)
    orc.tp_step(3000, 4e-9)
    oc = orc.counters()
    want = np.array([oc["tp_dep_l"], oc["tp_dep_r"], oc["tp_coll"], oc["n_tp"]])
    for r in (0, 1):
        tp = got[r][2]
        assert np.array_equal(tp["counts"], want)
        for k in ("sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r"):
            assert np.array_equal(tp[k], orc.diag(k)), k
    assert oc["tp_dep_r"] > 100 and oc["tp_coll"] > 100
