"""Event-driven test-particle flight (tp_flight) through the C ABI against
the FP64 oracle's orc_tp_flight.

Both draw every random word from Philox keyed by (atom id, event index,
purpose), so an atom follows the same sequence of events on both sides; the
GPU computes in FP32, so its positions and velocities differ from the
oracle's by rounding (tolerances below), and a rounding can flip a decision
near a wall or an acceptance threshold for a handful of atoms, which the
counts allow for.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1607_04069_gb300 import workloads as W

from helpers import gpu_discharge, match, oracle_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield


def _cfg(n, **over):
    c = W.tp_transport(n_atoms=n)
    c.update(gap_m=0.02, n_cells=64, cap_tp=n + 1024, n_e0=0, n_i0=0, sort_every_tp=0)
    c.update(over)
    return c


def _pair(cfg, n):
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=1024, cap_tp=n + 1024)
    d.tp_launch(n, 300.0)
    orc.tp_launch(n, 300.0)
    return d, orc


def test_first_events_match_per_atom():
    """After 3 events every atom still in flight has the oracle's position
    (1e-4 of the gap plus rounding) and velocity (1e-4 of its speed), and the
    atoms deposited so far agree at each electrode to 0.1 %."""
    n = 50_000
    d, orc = _pair(_cfg(n), n)
    d.tp_flight(3)
    orc.tp_flight(3)
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) + len(only_o) <= n // 1000
    vm = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
    for k in ("vx", "vy", "vz"):
        assert (np.abs(g[k] - o[k]) <= 1e-4 * vm + 1e-3).mean() > 0.999, k
    assert (np.abs(g["xi"] - o["xi"]) <= 1e-4 * 64 + 1e-6).mean() > 0.999
    c, oc = d.counters(), orc.counters()
    for k in ("tp_dep_l", "tp_dep_r"):
        assert abs(c[k] - oc[k]) <= max(5, oc[k] // 1000), (k, c[k], oc[k])
    d.close()


def test_run_to_deposition_matches_oracle():
    """All atoms of a 300 eV-ion source through a 2 cm, 0.5 Pa gap to
    deposition: deposits per electrode and collisions within 0.5 %, energy
    and angle distributions at the far electrode by a KS test, and the
    time-weighted residence profile within 2 % relative L2."""
    n = 40_000
    d, orc = _pair(_cfg(n), n)
    assert d.tp_flight(1_000_000) == 0
    assert orc.tp_flight(1_000_000) == 0
    c, oc = d.counters(), orc.counters()
    assert c["tp_dep_l"] + c["tp_dep_r"] == n
    for k in ("tp_dep_l", "tp_dep_r", "tp_coll"):
        assert abs(c[k] - oc[k]) <= 0.005 * max(oc[k], 1000), (k, c[k], oc[k])
    for k in ("sputter_e_r", "sputter_ang_r"):
        x, y = d.diag(k), orc.diag(k)
        D = np.abs(np.cumsum(x) / x.sum() - np.cumsum(y) / y.sum()).max()
        p = stats.kstwobign.sf(D * math.sqrt(x.sum() * y.sum() / (x.sum() + y.sum())))
        assert p > 0.01, (k, p)
    t, to = d.diag("tpf_time"), orc.diag("tpf_time")
    assert np.linalg.norm(t - to) / np.linalg.norm(to) < 0.02
    assert t.sum() == pytest.approx(to.sum(), rel=0.005)
    d.close()


def test_without_gas_every_atom_flies_straight_to_its_electrode():
    """p = 0: each atom deposits at the electrode it heads for in one event
    with its launch energy; the residence time of the cells crossed whole is
    the oracle's to FP32 rounding."""
    n = 30_000
    d, orc = _pair(_cfg(n, pressure_pa=0.0), n)
    assert d.tp_flight(4) == 0 and orc.tp_flight(4) == 0
    c, oc = d.counters(), orc.counters()
    assert c["tp_dep_r"] == oc["tp_dep_r"] == n and c["tp_coll"] == 0
    h, ho = d.diag("sputter_e_r"), orc.diag("sputter_e_r")
    assert np.abs(h - ho).sum() <= 2e-3 * n
    t, to = d.diag("tpf_time"), orc.diag("tpf_time")
    assert np.allclose(t[1:], to[1:], rtol=1e-5)
    d.close()


VHS = dict(tp_dref=4.17e-10, tp_omega=0.81, tp_tref=273.0)


@pytest.mark.parametrize("model", [1, 2], ids=["vhs", "m1"])
def test_vhs_and_m1_flights_match_oracle(model):
    """The VHS and M1 laws (majorant rate, null events, gamma-distributed
    candidate speeds, M1 deflections): after 4 events the atoms in flight
    match the oracle's per atom, and run to deposition the deposits,
    collisions and far-electrode energies agree as in the hard-sphere case."""
    n = 30_000
    cfg = _cfg(n, tp_model=model, **VHS)
    d, orc = _pair(cfg, n)
    d.tp_flight(4)
    orc.tp_flight(4)
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) + len(only_o) <= n // 500
    vm = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
    for k in ("vx", "vy", "vz"):
        assert (np.abs(g[k] - o[k]) <= 1e-4 * vm + 1e-3).mean() > 0.998, k
    assert d.tp_flight(1_000_000) == 0 and orc.tp_flight(1_000_000) == 0
    c, oc = d.counters(), orc.counters()
    for k in ("tp_dep_l", "tp_dep_r", "tp_coll"):
        assert abs(c[k] - oc[k]) <= 0.01 * max(oc[k], 1000), (k, c[k], oc[k])
    x, y = d.diag("sputter_e_r"), orc.diag("sputter_e_r")
    D = np.abs(np.cumsum(x) / x.sum() - np.cumsum(y) / y.sum()).max()
    assert stats.kstwobign.sf(D * math.sqrt(x.sum() * y.sum() / (x.sum() + y.sum()))) > 0.01
    d.close()


@pytest.mark.parametrize("tp_mode", [0, 1], ids=["thinned", "literal"])
@pytest.mark.parametrize("model", [1, 2], ids=["vhs", "m1"])
def test_vhs_and_m1_per_step_transport_matches_oracle(model, tp_mode):
    """tp_step under the VHS and M1 laws (per-step probability 1 -
    exp(-n K g^alpha dt) with a sampled partner; thinned candidates or the
    test every step): 200 steps of 1 ns, every atom within FP32 rounding of
    the oracle's, the same atoms deposited.  With thinned candidates an atom
    whose candidate probability lies within FP32 rounding of a step of its
    8-bit grid may draw another gap on the two sides (about 3e-5 per draw),
    so up to 1 in 2000 atoms may follow another history."""
    cfg = W.tp_transport(n_atoms=50_000)
    cfg.update(cap_tp=60_000, n_e0=0, n_i0=0, sort_every_tp=0, tp_model=model, tp_mode=tp_mode, **VHS)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=10, cap_tp=60_000)
    d.tp_launch(50_000, 300.0)
    orc.tp_launch(50_000, 300.0)
    alive = d.tp_step(200)
    orc.tp_step(200, cfg["tp_dt"])
    c, oc = d.counters(), orc.counters()
    assert c["tp_dep_l"] + c["tp_dep_r"] + alive == 50_000
    slack = 6 if tp_mode == 1 else 25
    assert abs(c["tp_coll"] - oc["tp_coll"]) <= slack // 2
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) + len(only_o) <= slack
    vmag = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
    assert (np.abs(g["vx"] - o["vx"]) > 1e-3 * vmag + 1e-2).sum() <= slack
    assert c["numerics"] == oc["numerics"] == 0
    d.close()
