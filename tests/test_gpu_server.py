"""The request loop (pic_server_*): admission by memory budget, period-by-
period steady-state test, and results.

A served discharge runs the same steps as one stepped alone, with the time
averages restarted at each RF period boundary, so its last period-averaged
n_e, n_i and phi must equal bit for bit those of the same discharge stepped
alone period by period -- whichever other requests share the worker, in the
batched and in the plain-loop mode.
"""
import numpy as np
import pytest

from paper_1607_04069_gb300 import workloads as W

from helpers import gpu_discharge

pytestmark = pytest.mark.gpu

PERIOD = 400                                   # steps per RF period at dt = T_RF / 400


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
    c.update(pos_precision=32, sort_every_e=200, sort_every_i=400)
    c.update(over)
    return c


def _alone(cfg, periods, window=1, period=PERIOD):
    d = gpu_discharge(cfg)
    out = None
    for p in range(periods):
        d.step(period)
        if (p + 1) % window == 0:
            out = {k: d.diag(k) for k in ("n_e", "n_i", "phi")}
            d.reset_averages()
    d.sync()
    d.close()
    return out


@pytest.mark.parametrize("batched", [1, 0], ids=["batched", "plain"])
def test_served_equals_alone(P, batched):
    cfgs = [_cfg(5_000, 21), _cfg(12_000, 22, pressure_pa=6.0), _cfg(3_000, 23, rf_volt_v=60.0)]
    s = P.Server(batched=batched, max_periods=3, tol=1e-12)
    ids = [s.submit(P.params_from_workload(c)) for c in cfgs]
    infos = [s.wait(i, timeout=120.0) for i in ids]
    got = [{k: s.result(i, k) for k in ("n_e", "n_i", "phi")} for i in ids]
    st = s.stats()
    s.close()
    assert st["done"] == 3 and st["running"] == 0 and st["queued"] == 0 and st["bytes_used"] == 0
    for c, info, g in zip(cfgs, infos, got):
        assert info["state"] == "max_periods" and info["periods"] == 3
        assert 0.0 <= info["t_arrival"] <= info["t_admit"] <= info["t_done"]
        assert info["change"] > 0.0
        want = _alone(c, 3)
        for k in ("n_e", "n_i", "phi"):
            assert np.array_equal(g[k], want[k]), k


def test_converged_budget_rejected_failed(P):
    c = _cfg(4_000, 31)
    nbytes = P.state_bytes(P.params_from_workload(c))
    assert nbytes > 4_000 * 2 * 28
    s = P.Server(hbm_budget_bytes=int(1.5 * nbytes), tol=1e6, criterion=1)   # room for one at a time
    a = s.submit(P.params_from_workload(c))
    b = s.submit(P.params_from_workload(_cfg(4_000, 32)))
    big = s.submit(P.params_from_workload(_cfg(400_000, 33)))
    bad = s.submit(P.params_from_workload(_cfg(4_000, 34, pos_precision=64)))
    ia, ib, ibig, ibad = (s.wait(r, timeout=120.0) for r in (a, b, big, bad))
    assert ia["state"] == "converged" and ia["periods"] == 2          # min_periods, any change < 1e6
    assert ib["state"] == "converged" and ib["t_admit"] >= ia["t_done"]
    assert ibig["state"] == "rejected" and "budget" in s.error(big)
    assert ibad["state"] == "failed" and "32-bit" in s.error(bad)
    assert s.result(a, "n_e").shape == (c["n_cells"] + 1,)
    s.forget(a)
    with pytest.raises(P.PicError):
        s.info(a)
    s.close()


def test_wait_times_out_and_close_abandons(P):
    s = P.Server(tol=1e-12)                                           # never converges
    r = s.submit(P.params_from_workload(_cfg(4_000, 41)))
    with pytest.raises(P.PicError) as e:
        s.wait(r, timeout=0.05)
    assert e.value.code == -9
    assert s.info(r)["state"] in ("queued", "running")
    s.close()


def test_averaging_windows_of_two_periods(P):
    c = _cfg(5_000, 51)
    s = P.Server(max_periods=4, window_periods=2, tol=1e-12, criterion=1)
    r = s.submit(P.params_from_workload(c))
    info = s.wait(r, timeout=120.0)
    got = {k: s.result(r, k) for k in ("n_e", "n_i", "phi")}
    s.close()
    assert info["state"] == "max_periods" and info["periods"] == 4 and info["change"] > 0.0
    want = _alone(c, 4, window=2)
    for k in ("n_e", "n_i", "phi"):
        assert np.array_equal(got[k], want[k]), k


def test_plain_loop_checks_each_request_at_its_own_period(P):
    """Without batching, discharges whose RF periods differ in steps share the
    worker (the chunk divides both); each is tested at its own period ends."""
    a = _cfg(4_000, 61)
    b = _cfg(4_000, 62, dt=W.T_RF / (2 * PERIOD))
    s = P.Server(batched=0, max_periods=2, tol=1e-12)
    ra, rb = s.submit(P.params_from_workload(a)), s.submit(P.params_from_workload(b))
    ia, ib = s.wait(ra, timeout=120.0), s.wait(rb, timeout=120.0)
    got = {k: s.result(rb, k) for k in ("n_e", "n_i", "phi")}
    s.close()
    assert ia["state"] == ib["state"] == "max_periods" and ia["periods"] == ib["periods"] == 2
    want = _alone(b, 2, period=2 * PERIOD)
    for k in ("n_e", "n_i", "phi"):
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("batched", [1, 0], ids=["batched", "plain"])
def test_request_of_another_period_waits_for_the_running_ones(P, batched):
    """A request whose RF period (420 steps) is no multiple of the running
    chunk (40 steps of a 400-step period) waits at the head of the queue,
    runs once the first request has finished -- with a chunk of its own --
    and gives the result of the discharge stepped alone."""
    a = _cfg(4_000, 71)
    b = _cfg(4_000, 72, dt=W.T_RF / 420)
    s = P.Server(batched=batched, max_periods=2, tol=1e-12)
    ra, rb = s.submit(P.params_from_workload(a)), s.submit(P.params_from_workload(b))
    ia, ib = s.wait(ra, timeout=120.0), s.wait(rb, timeout=120.0)
    got = {k: s.result(rb, k) for k in ("n_e", "n_i", "phi")}
    s.close()
    assert ia["state"] == ib["state"] == "max_periods" and ib["periods"] == 2
    assert ib["t_admit"] >= ia["t_done"]
    want = _alone(b, 2, period=420)
    for k in ("n_e", "n_i", "phi"):
        assert np.array_equal(got[k], want[k]), k
