"""A discharge split over two shards on one GPU (paper_1607_04069_gb300.shard:
pic_params.id_offset, pic_exchange_slot) against the same discharge in one
context, through the C ABI.

The shards run one after the other, each its own step launch, and between
steps their exchange blocks are summed on the device and written back to
both -- the sum an int64 all-reduce over ranks gives; no kernel waits for
another.  Every step of the method is per particle except the field solve,
whose charge is that sum, and every random word is keyed by particle id and
step, so the split discharge must equal the whole one: time-averaged
potential, densities and fluxes bit for bit on each shard, histograms and
event counts summed over the shards bit for bit, and every particle with the
same state.  A split test-particle source (tp_source.first_id) likewise.
"""
import numpy as np
import pytest

from paper_1607_04069_gb300 import workloads as W

from helpers import match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


HIST = ("iedf_l", "iedf_r", "eedf", "ieadf_l", "sputter_e_l", "sputter_ang_r")
COUNTS = ("imp_e_l", "imp_e_r", "imp_i_l", "imp_i_r", "ionizations", "sputtered_l", "sputtered_r", "elastic",
          "excitation", "cx", "iso", "tp_coll", "tp_dep_l", "tp_dep_r")


@pytest.mark.parametrize("prec", [32, 64])
def test_split_discharge_equals_the_whole(torch, prec):
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import shard
    cfg = W.ccp_sputter(n_per_species=60_000, n_cells=256, seed=93)
    cfg.update(rf_volt_v=1000.0, dt=W.T_RF / 400, tp_every=20, pos_precision=prec, sort_every_e=7,
               sort_every_i=50, sort_every_tp=5)
    whole = P.Discharge(P.params_from_workload(cfg))
    parts = [P.Discharge(P.params_from_workload(shard.shard_workload(cfg, r, 2), sort_every_e=11 + r))
             for r in (0, 1)]
    def exchange():
        slots = [p.exchange_slot() for p in parts]           # the block of the current step
        s = slots[0] + slots[1]
        for t in slots:
            t.copy_(s)

    exchange()
    for k in range(800):
        if k == 400:
            for d in [whole] + parts:
                d.reset_averages()
        whole.step(1)
        for p in parts:
            p.step(1)
        exchange()
    for d in [whole] + parts:
        d.sync()
    for p in parts:
        for k in ("phi", "n_e", "n_i", "gamma_e", "gamma_i", "E"):
            assert np.array_equal(p.diag(k), whole.diag(k)), k
    for k in HIST:
        assert np.array_equal(parts[0].diag(k) + parts[1].diag(k), whole.diag(k)), k
    cw, c0, c1 = whole.counters(), parts[0].counters(), parts[1].counters()
    for k in COUNTS:
        assert c0[k] + c1[k] == cw[k], (k, c0[k], c1[k], cw[k])
    assert cw["sputtered_l"] + cw["sputtered_r"] > 100 and cw["ionizations"] > 100
    for s in (0, 1, 2):
        a = {k: np.concatenate([p.get_species(s)[k] for p in parts]) for k in ("xi", "vx", "vy", "vz", "id")}
        g, o, only_a, only_w = match(a, whole.get_species(s))
        assert len(only_a) == 0 and len(only_w) == 0, s
        for k in ("xi", "vx", "vy", "vz"):
            assert np.array_equal(g[k], o[k]), (s, k)
    for d in [whole] + parts:
        d.close()


def test_split_test_particle_source(torch):
    import paper_1607_04069_gb300 as P
    from paper_1607_04069_gb300 import shard
    n = 200_000
    tc = W.tp_transport(n_atoms=n)
    tc.update(cap_tp=n + 1024, n_e0=0, n_i0=0, sort_every_tp=7, tp_dt=4e-9)
    whole = P.Discharge(P.params_from_workload(tc))
    whole.tp_launch(n, 300.0)
    parts = []
    for r in (0, 1):
        first, count = shard.part(n, r, 2)
        p = P.Discharge(P.params_from_workload(tc, cap_tp=count + 1024))
        p.tp_launch(count, 300.0, first_id=first)
        parts.append(p)
    for d in [whole] + parts:
        d.tp_step(1500, count_alive=False)
    for k in ("sputter_e_l", "sputter_e_r", "sputter_ang_l", "sputter_ang_r"):
        assert np.array_equal(parts[0].diag(k) + parts[1].diag(k), whole.diag(k)), k
    cw, c0, c1 = whole.counters(), parts[0].counters(), parts[1].counters()
    for k in ("tp_dep_l", "tp_dep_r", "tp_coll"):
        assert c0[k] + c1[k] == cw[k], k
    assert cw["tp_dep_r"] > 1000
    for d in [whole] + parts:
        d.close()
