"""Batched discharges (pic_batch_*) against the same discharges stepped alone.

A member of a batch runs the step of pic_step on its own range of the
launch's CTAs; every quantity is either integer (charge, moments, counters,
histograms) or a function of the particle's id and step (the collision
draws), so a member's state after k steps must equal, bit for bit, that of
the same discharge stepped k times by itself -- on a different number of
CTAs, and whichever other members share the launch.  Particles are compared
per id: the order of slots depends on the scheduling of births.
"""
import numpy as np
import pytest

from paper_1607_04069_gb300 import workloads as W

from helpers import by_id, gpu_discharge

pytestmark = pytest.mark.gpu

DIAGS = ["phi", "n_e", "n_i", "gamma_e", "gamma_i", "v_e", "v_i", "eedf", "iedf_l", "iedf_r", "ieadf_l",
         "ieadf_r"]


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1607_04069_gb300 as P
    return P


def _cfg(n, seed, **over):
    c = W.ccp_small(n_per_species=n, seed=seed)
    c.update(pos_precision=32, sort_every_e=50, sort_every_i=70, cap_e=4 * n + 4096, cap_i=4 * n + 4096)
    c.update(over)
    return c


MEMBERS = [
    _cfg(20_000, 11),
    _cfg(6_000, 12, pressure_pa=5.0, rf_volt_v=150.0),
    _cfg(33_000, 13, rf_volt_v=80.0, sort_every_e=0),
    _cfg(9_000, 17, waveform=1, rf_phase=0.5, circuit=1, c_block=2.0 * 8.8541878128e-12 / 0.025),
]


def _state(d):
    s = {"counters": d.counters(), "field": d.get_field()}
    for k in DIAGS:
        s[k] = d.diag(k)
    for sp in ("e", "i"):
        s[sp] = by_id(d.get_species(sp))
    return s


def _alone(cfg, steps):
    d = gpu_discharge(cfg)
    d.step(steps)
    d.sync()
    s = _state(d)
    d.close()
    return s


def _same(a, b, what):
    assert a["counters"] == b["counters"], what
    for k in ("E", "phi", "q_e", "q_i"):
        assert np.array_equal(a["field"][k], b["field"][k]), (what, k)
    for k in DIAGS:
        assert np.array_equal(a[k], b[k]), (what, k)
    for sp in ("e", "i"):
        for k in ("id", "xi", "vx", "vy", "vz"):
            assert np.array_equal(a[sp][k], b[sp][k]), (what, sp, k)


@pytest.mark.parametrize("per_cta,chunk", [(16_384, 131_072), (2_048, 8_192), (16_384, 0)],
                         ids=["default", "chunks_of_4_slots", "one_cta_per_slot"])
def test_batch_equals_alone(P, per_cta, chunk):
    """Every member bit for bit equal to the discharge stepped alone, with the
    resident CTAs taking chunks of slots (the default launch: here the
    members' 2-5 slots are one-slot chunks; with 2048 particles per slot
    they form chunks of 4 slots whose later slots reuse the field of the
    first, and one-slot tail chunks) and with one CTA per slot."""
    steps = 120
    b = P.Batch(particles_per_cta=per_cta, particles_per_chunk=chunk)
    slots = [b.add(P.params_from_workload(c)) for c in MEMBERS]
    assert slots == [0, 1, 2, 3]
    b.step(steps // 2)
    b.step(steps - steps // 2)
    b.sync()
    got = [_state(b.member(k)) for k in slots]
    b.close()
    for k, c in enumerate(MEMBERS):
        _same(got[k], _alone(c, steps), f"member {k}")
        assert got[k]["counters"]["step"] == steps


def test_join_and_leave(P):
    """A member leaves after 60 steps and another joins in its slot; the
    others go on undisturbed and the newcomer matches 60 steps alone."""
    b = P.Batch(particles_per_cta=16_384)
    s0 = b.add(P.params_from_workload(MEMBERS[0]))
    s1 = b.add(P.params_from_workload(MEMBERS[1]))
    b.step(60)
    b.remove(s1)
    late = _cfg(9_000, 14, pressure_pa=2.0)
    assert b.add(P.params_from_workload(late)) == s1
    b.step(60)
    b.sync()
    got0, got1 = _state(b.member(s0)), _state(b.member(s1))
    b.close()
    _same(got0, _alone(MEMBERS[0], 120), "stayed")
    _same(got1, _alone(late, 60), "joined")


def test_admission_rules(P):
    b = P.Batch()
    b.add(P.params_from_workload(MEMBERS[0]))
    for bad in (dict(pos_precision=64), dict(dt=W.T_RF / 401), dict(diag_every=20),
                dict(sputter_enable=1, tp_every=40)):
        with pytest.raises(P.PicError):
            b.add(P.params_from_workload(_cfg(4_000, 15, **bad)))
    odd = P.Batch()                                # 400.5 steps per RF period
    with pytest.raises(P.PicError, match="RF period"):
        odd.add(P.params_from_workload(_cfg(4_000, 15, dt=W.T_RF / 400.5)))
    odd.close()
    b.step(5)                                      # off the sampling grid: no one may join now
    with pytest.raises(P.PicError):
        b.add(P.params_from_workload(_cfg(4_000, 16)))
    b.step(5)
    b.add(P.params_from_workload(_cfg(4_000, 16)))
    with pytest.raises(P.PicError):
        b.member(7)
    b.sync()
    b.close()
    empty = P.Batch()
    empty.step(3)                                  # nothing to do
    empty.close()


def test_graphs_timing_and_autotune_change_nothing(P):
    """Graph replay (with a member whose compaction period, 33, is no
    multiple of the sampling period, so some runs fall back to single
    launches), the launch timers and the autotuner's candidate divisions
    leave every member's state as it is when stepped alone."""
    members = [MEMBERS[0], _cfg(6_000, 12, pressure_pa=5.0, sort_every_i=33), MEMBERS[2]]
    b = P.Batch(particles_per_cta=16_384)
    b.graphs(True)
    slots = [b.add(P.params_from_workload(c)) for c in members]
    b.step(5)                                      # off the sampling grid: single launches first
    b.timing(True)
    b.step(40)
    ms, steps = b.timing(False)
    assert steps == 40 and ms > 0.0
    best = b.autotune([8192, 32768], steps_each=10)
    assert best in (8192, 32768)
    b.step(150 - 5 - 40 - 2 * 11)
    b.sync()
    got = [_state(b.member(k)) for k in slots]
    b.close()
    for k, c in enumerate(members):
        _same(got[k], _alone(c, 150), f"member {k}")
