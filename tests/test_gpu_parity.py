"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written out per test):
* integer work -- charge deposits, ids, counters, histograms of integer
  keys -- is compared bit for bit;
* the FP32 push against the FP64 oracle: one-step velocity and displacement
  within 1e-5 relative (plus one 2^-32 L fixed-point unit for positions);
* the FP64 field solve within 1e-12 relative to max |phi|.
Random decisions (collision candidate, process, sputter trial) are taken
from identical Philox words on both sides, so they must agree exactly.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1607_04069_gb300 import workloads as W

from helpers import by_id, gpu_discharge, match, oracle_for

pytestmark = pytest.mark.gpu

QE, ME, AMU = 1.602176634e-19, 9.1093837015e-31, 1.66053906660e-27
MAR, MAL = 39.948 * AMU, 26.98 * AMU


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1607_04069_gb300 as P
    P.lib()
    yield


def _worst(err, ids, k=5):
    i = np.argsort(err)[::-1][:k]
    return [(int(ids[j]), float(err[j])) for j in i]


def _torch_pos(pos):
    import torch
    if pos.dtype == np.uint32:
        return torch.from_numpy(pos.view(np.int32).copy()).cuda()
    return torch.from_numpy(pos.copy()).cuda()


# ------------------------------------------------------------------ initial loading / Philox
@pytest.mark.parametrize("prec", [32, 64])
def test_initial_loading_bit_identical_positions(prec):
    """Philox stream on the GPU reproduces the oracle's: positions (raw Philox
    words) bit for bit, Box-Muller velocities within FP32 rounding."""
    n = 50_001
    cfg = W.ccp_small(n_per_species=n)
    cfg["pos_precision"] = prec
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg)
    orc.init_species(0, n, cfg["te0_ev"])
    orc.init_species(1, n, cfg["ti0_ev"])
    for s, T, m in ((0, cfg["te0_ev"], ME), (1, cfg["ti0_ev"], MAR)):
        g, o = by_id(d.get_species(s)), by_id(orc.get_species(s))   # the GPU keeps cell order
        assert np.array_equal(g["id"], o["id"])
        assert np.array_equal(g["xi"], o["xi"])
        vth = math.sqrt(T * QE / m)
        for c in ("vx", "vy", "vz"):
            assert np.abs(g[c] - o[c]).max() <= 2e-6 * vth * 8
    d.close()


# ------------------------------------------------------------------ deposit (bit-exact)
@pytest.mark.parametrize("ncell", [4, 128, 1024, 4096])
@pytest.mark.parametrize("layout", ["random", "sorted", "one_cell", "with_dead"])
def test_deposit_bit_exact(ncell, layout):
    """Linear weighting into int64: identical to the oracle bit for bit, for
    random and cell-sorted particles (the warp-aggregated path), all in one
    cell, and with removed slots; n spans several CTAs plus a ragged tail."""
    import paper_1607_04069_gb300 as P
    rng = np.random.default_rng(ncell + len(layout))
    n = 1_000_003
    pos = W.fixed_positions(rng, n)
    if layout == "sorted":
        pos = np.sort(pos)
    elif layout == "one_cell":
        cell = 2**32 // ncell
        base = min(5, ncell - 1) * cell + cell // 4
        pos = (pos.astype(np.uint64) % (cell // 2) + base).astype(np.uint32)
    elif layout == "with_dead":
        pos[rng.random(n) < 0.1] = 0
    xi = pos.astype(np.float64) * (ncell / 2.0**32)
    xi[pos == 0] = -1.0
    q = P.op_deposit(_torch_pos(pos), ncell).cpu().numpy()
    assert np.array_equal(q, O.deposit(xi, ncell))
    # 64-bit positions in cell units: same values, same deposit
    q64 = P.op_deposit(_torch_pos(xi), ncell).cpu().numpy()
    assert np.array_equal(q64, O.deposit(xi, ncell))


def test_deposit_edge_sizes():
    import paper_1607_04069_gb300 as P
    import torch
    for n in (0, 1, 31, 32, 33, 257):
        rng = np.random.default_rng(n)
        pos = W.fixed_positions(rng, max(n, 1))[:n]
        xi = pos.astype(np.float64) * (64 / 2.0**32)
        t = _torch_pos(pos) if n else torch.zeros(0, dtype=torch.int32, device="cuda")
        q = P.op_deposit(t, 64).cpu().numpy()
        assert np.array_equal(q, O.deposit(xi, 64))


# ------------------------------------------------------------------ field solve
@pytest.mark.parametrize("ncell", [4, 128, 1024, 2048, 4096])
def test_poisson_matches_oracle(ncell, record):
    """Exact double-prefix-sum solve on the GPU vs the oracle's Thomas sweep.
    Tolerance: the oracle's own forward error, which grows with the condition
    number of the 1D Laplacian (~ N^2): max(1e-12, N^2 eps / 100) of max
    |phi| (pinned against exact rationals in test_oracle_pins)."""
    tol = max(1e-12, ncell**2 * 2.2e-16 / 100)
    import paper_1607_04069_gb300 as P
    import torch
    rng = np.random.default_rng(ncell)
    L, w = 0.05, 1e11
    dx = L / ncell
    q_i = rng.integers(0, 2**46, size=ncell + 1, dtype=np.int64)
    q_e = q_i + rng.integers(-2**40, 2**40, size=ncell + 1, dtype=np.int64)
    for v_left in (0.0, 300.0, -123.4):
        phi, E = P.op_poisson(torch.from_numpy(q_i).cuda(), torch.from_numpy(q_e).cuda(), ncell,
                              dx, w, v_left)
        phi, E = phi.cpu().numpy(), E.cpu().numpy()
        phi_o, E_o = O.poisson(ncell, dx, w, q_i, q_e, v_left)
        record(f"poisson.N{ncell}.V{v_left:g}.phi_max_rel", float(np.abs(phi - phi_o).max() / np.abs(phi_o).max()))
        record(f"poisson.N{ncell}.V{v_left:g}.E_max_rel", float(np.abs(E - E_o).max() / np.abs(E_o).max()))
        assert np.abs(phi - phi_o).max() <= tol * np.abs(phi_o).max()
        assert np.abs(E - E_o).max() <= 100 * tol * np.abs(E_o).max()


# ------------------------------------------------------------------ one-step push
def _load_both(d, orc, sets, prec):
    for s, st in sets.items():
        d.set_species(s, st["pos"], st["vx"], st["vy"], st["vz"], st["id"])
        orc.set_species(s, st["xi"], st["vx"].astype(np.float64), st["vy"].astype(np.float64),
                        st["vz"].astype(np.float64), st["id"])


def _smooth_field(ncell, scale, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, ncell + 1)
    E = np.zeros(ncell + 1)
    for k in range(1, 6):
        E += rng.normal() * np.sin(k * np.pi * x + rng.uniform(0, np.pi))
    return scale * E


@pytest.mark.parametrize("prec", [32, 64])
def test_one_step_push_parity(prec, record):
    """Gather + leapfrog + wall, collisions off (p = 0): every particle's
    v_x^{l+1/2} and displacement within 1e-5 relative of the oracle, v_y, v_z
    untouched, the same particles absorbed, and Sum q = 2^32 x alive."""
    ncell = 1024
    cfg = W.ccp_sputter(n_per_species=1000, n_cells=ncell)
    cfg.update(pressure_pa=0.0, pos_precision=prec, sputter_enable=0, sort_every_e=0,
               sort_every_i=0, n_e0=0, n_i0=0, cap_e=300_000, cap_i=300_000)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=300_000)
    sets = {0: W.random_particles(200_001, ncell, 0, 2e6, 1, prec),
            1: W.random_particles(100_003, ncell, 1, 3e4, 2, prec)}
    _load_both(d, orc, sets, prec)
    E = _smooth_field(ncell, 2e4, 3)
    d.set_field(E)
    orc.set_field(E)
    d.step(1)
    d.sync()
    orc.step(1)
    unit = ncell / 2.0**32
    dt = cfg["dt"]
    for s in (0, 1):
        g, o, only_g, only_o = match(d.get_species(s), orc.get_species(s))
        x0 = dict(zip(sets[s]["id"].tolist(), sets[s]["xi"].tolist()))
        assert len(only_g) == 0 and len(only_o) == 0, (len(only_g), len(only_o))
        xi0 = np.array([x0[i] for i in o["id"].tolist()])
        v0 = dict(zip(sets[s]["id"].tolist(), sets[s]["vx"].tolist()))
        vx0 = np.array([v0[i] for i in o["id"].tolist()])
        # velocity error scale: |v_old| + |dv| (v^{l+1/2} may cancel to ~0)
        vscale = np.abs(vx0) + np.abs(o["vx"] - vx0)
        dvx = np.abs(g["vx"] - o["vx"])
        record(f"push.u{prec}.species{s}.dvx_max_rel", float((dvx / (vscale + 1e-30)).max()))
        assert (dvx <= 1e-5 * vscale + 1e-3).all(), _worst(dvx / (vscale + 1e-30), o["id"])
        # displacement error: 1e-5 of the same scale times dt/dx, plus the position resolution
        tol = 1e-5 * vscale * dt / (cfg["gap_m"] / ncell) + (2 * unit if prec == 32 else 1e-9)
        dxi = np.abs(g["xi"] - o["xi"])
        record(f"push.u{prec}.species{s}.dx_max_cells", float(dxi.max()))
        assert (dxi <= tol).all(), _worst(dxi / tol, o["id"])
        vy0 = dict(zip(sets[s]["id"].tolist(), sets[s]["vy"].tolist()))
        assert np.array_equal(g["vy"], np.array([vy0[i] for i in g["id"].tolist()], dtype=np.float32))
    f, fo = d.get_field(), orc.get_field()
    c = d.counters()
    alive = [len(d.get_species(s)["id"]) for s in (0, 1)]
    assert int(f["q_e"].sum()) == 2**32 * alive[0] and int(f["q_i"].sum()) == 2**32 * alive[1]
    assert np.abs(f["E"] - fo["E"]).max() <= 1e-5 * np.abs(fo["E"]).max()
    oc = orc.counters()
    assert c["imp_e_l"] + c["imp_e_r"] == oc["imp_e_l"] + oc["imp_e_r"]
    d.close()


@pytest.mark.parametrize("ne,ni", [(0, 0), (1, 0), (0, 1), (3, 2), (5, 9)])
def test_empty_and_tiny_species_steps(ne, ni, record):
    """Degenerate sizes of the stream: a species with no particle (every CTA of
    it empty), a single particle, a partial group of four, ionisation children
    appended after one particle.  Forty full steps (field, push, walls,
    collisions at 30 Pa: a few elastic events and ionisations) against the
    oracle: the same particles alive, the same collision and wall counts,
    Sum q = 2^32 x alive, velocities within 1e-3 and positions within 0.05
    cells.  (The FP32 field and push differ from the oracle's FP64 by about
    1e-5 over forty steps; an excitation or ionisation near its threshold
    amplifies that in the speed it leaves, by eps / (eps - threshold), and
    ionisation children start at their parent's position, so a slow ion
    carries its parent's drift.  The test is about the sizes: the counts are
    exact.)"""
    ncell = 128
    cfg = W.ccp_small(n_per_species=1000)
    cfg.update(n_cells=ncell, pressure_pa=30.0, rf_volt_v=100.0, pos_precision=32, sputter_enable=0,
               sort_every_e=0, sort_every_i=0, n_e0=0, n_i0=0, cap_e=1024, cap_i=1024,
               gap_m=0.02, dt=2e-11)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=1024)
    sets = {0: W.random_particles(ne, ncell, 0, math.sqrt(30 * QE / ME), 11, 32),
            1: W.random_particles(ni, ncell, 1, 3e3, 12, 32)}
    _load_both(d, orc, sets, 32)
    steps = 40
    d.step(steps)
    d.sync()
    orc.step(steps)
    c, oc = d.counters(), orc.counters()
    for k in ("elastic", "excitation", "ionizations", "cx", "iso", "imp_e_l", "imp_e_r", "imp_i_l", "imp_i_r"):
        assert c[k] == oc[k], (k, c[k], oc[k])
    for s in (0, 1):
        g, o, only_g, only_o = match(d.get_species(s), orc.get_species(s))
        assert len(only_g) == 0 and len(only_o) == 0, (s, len(only_g), len(only_o))
        if len(o["id"]) == 0:
            continue
        vo = np.stack([o["vx"], o["vy"], o["vz"]])
        vg = np.stack([g["vx"], g["vy"], g["vz"]]).astype(np.float64)
        scale = np.linalg.norm(vo, axis=0) + 1e4
        dv = np.linalg.norm(vg - vo, axis=0)
        record(f"tiny.{ne}_{ni}.species{s}.dv_max_rel", float((dv / scale).max()))
        assert (dv <= 1e-3 * scale).all(), _worst(dv / scale, o["id"])
        dxi = np.abs(g["xi"] - o["xi"])
        record(f"tiny.{ne}_{ni}.species{s}.dx_max_cells", float(dxi.max()))
        assert (dxi <= 0.05).all(), _worst(dxi, o["id"])
    # (the field follows the positions: a superparticle of this weight moved by
    # 0.02 cells shifts E by a few V/m, so only the charge is compared here)
    f = d.get_field()
    alive = [len(d.get_species(s)["id"]) for s in (0, 1)]
    assert int(f["q_e"].sum()) == 2**32 * alive[0] and int(f["q_i"].sum()) == 2**32 * alive[1]
    assert np.isfinite(f["E"]).all()
    d.close()


# ------------------------------------------------------------------ one-step MCC
@pytest.mark.parametrize("case", ["electrons", "ions"])
def test_one_step_collision_parity(case, record):
    """Null-collision MCC from identical Philox words: the same particles
    collide with the same process, post-collision velocities within FP32
    rounding, ionisation children with the same ids and states."""
    ncell = 256
    cfg = W.ccp_small(n_per_species=1000)
    cfg.update(n_cells=ncell, pressure_pa=3.0, rf_volt_v=100.0, pos_precision=32,
               sort_every_e=0, sort_every_i=0, n_e0=0, n_i0=0, cap_e=400_000, cap_i=400_000,
               gap_m=1.0, dt=1e-10 if case == "electrons" else 1e-8)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=400_000)
    sets = {0: W.random_particles(100_000, ncell, 0, math.sqrt(20 * QE / ME), 5, 32),
            1: W.random_particles(100_000, ncell, 1, 2e3, 6, 32)}
    if case == "electrons":
        sets[1] = W.random_particles(0, ncell, 1, 1.0, 7, 32)
    _load_both(d, orc, sets, 32)
    E = np.zeros(ncell + 1)
    d.set_field(E)
    orc.set_field(E)
    d.step(1)
    d.sync()
    orc.step(1)
    c, oc = d.counters(), orc.counters()
    keys = ["elastic", "excitation", "ionizations"] if case == "electrons" else ["cx", "iso"]
    for k in keys:
        assert c[k] == oc[k], (k, c[k], oc[k])
    assert sum(c[k] for k in keys) > 500
    for s, mass in ((0, ME), (1, MAR)):
        g, o, only_g, only_o = match(d.get_species(s), orc.get_species(s))
        assert len(only_g) == 0 and len(only_o) == 0
        # energies: FP32 rounding of the pre-collision energy (eps - threshold
        # cancels near a threshold, so compare energies, not speeds)
        e0 = {int(i): 0.5 * mass * (a * a + b * b + c * c) / QE for i, a, b, c in
              zip(sets[s]["id"], sets[s]["vx"].astype(np.float64), sets[s]["vy"].astype(np.float64),
                  sets[s]["vz"].astype(np.float64))}
        e_ref = max(e0.values()) if e0 else 1.0
        E0 = np.array([e0.get(int(i), e_ref) for i in o["id"]])
        Eg = 0.5 * mass * (g["vx"].astype(np.float64)**2 + g["vy"]**2.0 + g["vz"]**2.0) / QE
        Eo = 0.5 * mass * (o["vx"]**2 + o["vy"]**2 + o["vz"]**2) / QE
        dE = np.abs(Eg - Eo)
        record(f"collision.{case}.species{s}.dE_max_rel", float((dE / (E0 + Eo + 16.0)).max()))
        assert (dE <= 2e-6 * (E0 + Eo + 16.0)).all(), _worst(dE / (E0 + Eo + 16.0), o["id"])
        # directions
        vg = np.stack([g["vx"], g["vy"], g["vz"]]).astype(np.float64)
        vo = np.stack([o["vx"], o["vy"], o["vz"]])
        ng, no = np.linalg.norm(vg, axis=0), np.linalg.norm(vo, axis=0)
        ok = no > 0
        ddir = np.linalg.norm(vg[:, ok] / ng[ok] - vo[:, ok] / no[ok], axis=0)
        assert (ddir <= 1e-5).all(), _worst(ddir, o["id"][ok])
    d.close()


# ------------------------------------------------------------------ sputtering
@pytest.mark.parametrize("E_ion,V0", [(310.0, 300.0), (700.0, 300.0), (310.0, 0.0)])
def test_sputter_launch_parity(E_ion, V0):
    """Ar+ impacts at E_ion: the same trials succeed, the sputtered atoms
    carry the same ids, Thompson/cosine velocities within FP32 rounding, and
    the IEDF and IEADF counts agree bin for bin.  310 eV lies away from an
    IEDF bin edge of [0, 2 V0]; 700 eV lies beyond 2 V0 and V0 = 0 gives the
    [0, 1 eV] range, where every impact lands in the last bin."""
    ncell = 1024
    cfg = W.ccp_sputter(n_per_species=1000, n_cells=ncell)
    cfg.update(pressure_pa=0.0, n_e0=0, n_i0=0, cap_e=1000, cap_i=200_000, cap_tp=400_000,
               sort_every_e=0, sort_every_i=0, tp_every=0, dt=1e-10, rf_volt_v=V0)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=400_000)
    n = 100_000
    rng = np.random.default_rng(12)
    pos = rng.integers(1, 2000, size=n, dtype=np.uint64).astype(np.uint32)
    v = math.sqrt(2 * E_ion * QE / MAR)
    ids = np.arange(n, dtype=np.uint64) | np.uint64(1 << 62)
    vx = np.full(n, -v, dtype=np.float32)
    zero = np.zeros(n, dtype=np.float32)
    d.set_species(1, pos, vx, zero, zero, ids)
    orc.set_species(1, pos.astype(np.float64) * ncell / 2.0**32, vx.astype(np.float64), zero * 0.0,
                    zero * 0.0, ids)
    d.set_field(np.zeros(ncell + 1))
    orc.set_field(np.zeros(ncell + 1))
    d.step(1)
    d.sync()
    orc.step(1)
    c, oc = d.counters(), orc.counters()
    assert c["imp_i_l"] == oc["imp_i_l"] == n
    assert c["sputtered_l"] == oc["sputtered_l"] > 0
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) == 0 and len(only_o) == 0
    for comp in ("vx", "vy", "vz"):
        assert np.abs(g[comp] - o[comp]).max() <= 1e-4 * np.abs(o["vx"]).max()
    for k in ("iedf_l", "ieadf_l"):
        assert np.array_equal(d.diag(k), orc.diag(k)), k
    if E_ion > 2 * V0:
        assert d.diag("iedf_l")[-1] == n
    d.close()


# ------------------------------------------------------------------ test particles
@pytest.mark.parametrize("tp_mode", [0, 1], ids=["thinned", "literal"])
def test_tp_transport_parity(tp_mode):
    """Mono-energetic 300 eV source, 200 TP steps of 1 ns: every atom's state
    within FP32 rounding of the oracle's, the same atoms deposited, and the
    counts conserved (launched = deposited + in flight).  tp_mode 0: thinned
    candidates with geometric gaps; an atom whose candidate probability lies
    within FP32 rounding of a step of its 8-bit grid may draw another gap on
    the two sides (about 3e-5 per draw), so up to 1 in 2000 atoms may follow
    another history.  tp_mode 1: the literal test every step."""
    cfg = W.tp_transport(n_atoms=50_000)
    cfg.update(cap_tp=60_000, n_e0=0, n_i0=0, sort_every_tp=0, tp_mode=tp_mode)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=10, cap_tp=60_000)
    d.tp_launch(50_000, 300.0)
    orc.tp_launch(50_000, 300.0)
    alive = d.tp_step(200)
    orc.tp_step(200, cfg["tp_dt"])
    c, oc = d.counters(), orc.counters()
    slack = 4 if tp_mode == 1 else 25
    assert c["tp_dep_l"] + c["tp_dep_r"] + alive == 50_000
    assert abs(c["tp_coll"] - oc["tp_coll"]) <= slack // 2
    assert abs(c["tp_dep_r"] - oc["tp_dep_r"]) <= slack // 2 and abs(c["tp_dep_l"] - oc["tp_dep_l"]) <= slack // 2
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) + len(only_o) <= slack
    vmag = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
    bad = np.abs(g["vx"] - o["vx"]) > 1e-3 * vmag + 1e-2
    assert bad.sum() <= slack
    assert c["tp_coll"] > 1000 and c["numerics"] == oc["numerics"] == 0
    d.close()


@pytest.mark.parametrize("tp_mode", [0, 1], ids=["thinned", "literal"])
@pytest.mark.parametrize("n", [1, 3, 6])
def test_tp_tiny_sources(n, tp_mode):
    """A source of one to six atoms (one partial group of four, every other
    CTA of the TP step empty, sample steps among them): 400 TP steps of 20 ns
    against the oracle, the same atoms deposited at the same electrodes, the
    same collisions, and the atoms in flight within FP32 rounding."""
    cfg = W.tp_transport(n_atoms=n)
    cfg.update(cap_tp=64, n_e0=0, n_i0=0, sort_every_tp=0, tp_mode=tp_mode, tp_dt=2e-8)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=10, cap_tp=64)
    d.tp_launch(n, 300.0)
    orc.tp_launch(n, 300.0)
    alive = d.tp_step(400)
    orc.tp_step(400, cfg["tp_dt"])
    c, oc = d.counters(), orc.counters()
    for k in ("tp_dep_l", "tp_dep_r", "tp_coll"):
        assert c[k] == oc[k], (k, c[k], oc[k])
    assert c["tp_dep_l"] + c["tp_dep_r"] + alive == n
    g, o, only_g, only_o = match(d.get_species(2), orc.get_species(2))
    assert len(only_g) == 0 and len(only_o) == 0
    vmag = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
    assert (np.abs(g["vx"] - o["vx"]) <= 1e-3 * vmag + 1e-2).all()
    d.close()


# ------------------------------------------------------------------ determinism
def test_bitwise_independent_of_order_and_sort_period():
    """Randomness keyed by (id, step, purpose) and integer deposits make the
    run independent of particle order and of the compaction period: 60 steps
    from a shuffled input with compaction every step end bit-identical to 60
    steps from the ordered input without compaction."""
    cfg = W.ccp_small(n_per_species=20_000)
    cfg.update(pos_precision=32, sort_every_e=0, sort_every_i=0)
    a = gpu_discharge(cfg)
    sp = {s: a.get_species(s) for s in (0, 1)}
    b = gpu_discharge(cfg, sort_every_e=1, sort_every_i=3)
    rng = np.random.default_rng(0)
    for s in (0, 1):
        perm = rng.permutation(len(sp[s]["id"]))
        pos = np.rint(sp[s]["xi"][perm] * (2.0**32 / cfg["n_cells"])).astype(np.uint64).astype(np.uint32)
        b.set_species(s, pos, sp[s]["vx"][perm], sp[s]["vy"][perm], sp[s]["vz"][perm], sp[s]["id"][perm])
    a.step(60)
    b.step(60)
    a.sync()
    b.sync()
    for s in (0, 1):
        ga, gb, oa, ob = match(a.get_species(s), b.get_species(s))
        assert len(oa) == 0 and len(ob) == 0
        for k in ("xi", "vx", "vy", "vz"):
            assert np.array_equal(ga[k], gb[k]), k
    for k in ("phi", "n_e", "n_i", "gamma_e", "iedf_l", "eedf"):
        assert np.array_equal(a.diag(k), b.diag(k)), k
    a.close()
    b.close()


# ------------------------------------------------------------------ full size, bench launch shape
def test_full_size_step_matches_oracle(record):
    """The sputtering discharge at its full size (2M e- + 2M Ar+, 1024 cells)
    in the benchmark's launch configuration: after one step every particle
    matches the oracle's within the one-step tolerances, charge is conserved
    exactly, and the new field agrees to 1e-5 of max |E|."""
    cfg = W.ccp_sputter()
    cfg.update(sort_every_e=25, sort_every_i=200, sort_every_tp=50)
    n = cfg["n_e0"]
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=n + n // 4 + 65536)
    orc.init_species(0, n, cfg["te0_ev"])
    orc.init_species(1, n, cfg["ti0_ev"])
    orc.field()
    f0, fo0 = d.get_field(), orc.get_field()
    assert np.array_equal(f0["q_e"], fo0["q_e"]) and np.array_equal(f0["q_i"], fo0["q_i"])
    d.step(1)
    d.sync()
    orc.step(1)
    for s, mass in ((0, ME), (1, MAR)):
        g, o, only_g, only_o = match(d.get_species(s), orc.get_species(s))
        assert len(only_g) == 0 and len(only_o) == 0
        vmag = np.sqrt(o["vx"]**2 + o["vy"]**2 + o["vz"]**2)
        for comp in ("vx", "vy", "vz"):
            record(f"full_size_step.species{mass == MAR:d}.{comp}_max_rel",
                   float((np.abs(g[comp] - o[comp]) / (vmag + 1e-30)).max()))
            assert (np.abs(g[comp] - o[comp]) <= 2e-5 * vmag + 1e-2).all(), comp
        unit = cfg["n_cells"] / 2.0**32
        disp_tol = 2e-5 * vmag * cfg["dt"] / (cfg["gap_m"] / cfg["n_cells"]) + 2 * unit
        assert (np.abs(g["xi"] - o["xi"]) <= disp_tol).all()
    f, fo = d.get_field(), orc.get_field()
    alive = [len(d.get_species(s)["id"]) for s in (0, 1)]
    assert int(f["q_e"].sum()) == 2**32 * alive[0] and int(f["q_i"].sum()) == 2**32 * alive[1]
    record("full_size_step.E_max_rel", float(np.abs(f["E"] - fo["E"]).max() / np.abs(fo["E"]).max()))
    record("full_size_step.deposit_equal", bool(np.array_equal(f["q_e"], fo["q_e"]) and np.array_equal(f["q_i"], fo["q_i"])))
    assert np.abs(f["E"] - fo["E"]).max() <= 1e-5 * np.abs(fo["E"]).max()
    d.close()


# ------------------------------------------------------------------ statistics at steady operation
def _ks_hist(x, y):
    from scipy.stats import kstwobign
    n1, n2 = x.sum(), y.sum()
    D = np.abs(np.cumsum(x) / n1 - np.cumsum(y) / n2).max()
    return float(kstwobign.sf(D * math.sqrt(n1 * n2 / (n1 + n2)))), int(n1), int(n2)


def test_time_averaged_profiles_and_iedf_match_oracle():
    """The 25 mm / 128-cell / 100 V / 3 Pa discharge with 20k + 20k
    superparticles and 64-bit positions, 20 RF periods: potential and
    densities averaged over periods 10-20 within 3% relative L2 of the
    oracle's (same seed); ion energy distributions at both electrodes pass a
    two-sample KS test at p > 0.01."""
    cfg = W.ccp_small()
    n = cfg["n_e0"]
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=3 * n)
    orc.init_species(0, n, cfg["te0_ev"])
    orc.init_species(1, n, cfg["ti0_ev"])
    orc.field()
    half = 400 * 10
    d.step(half)
    orc.step(half)
    d.sync()
    d.reset_averages()
    orc.reset_averages()
    d.step(half)
    d.sync()
    orc.step(half)
    from helpers import rel_l2
    for k in ("phi", "n_e", "n_i"):
        assert rel_l2(d.diag(k), orc.diag(k)) < 0.03, k
    for k in ("iedf_l", "iedf_r"):
        p, n1, n2 = _ks_hist(d.diag(k), orc.diag(k))
        assert n1 > 300 and n2 > 300 and p > 0.01, (k, p, n1, n2)
    d.close()


def test_tp_far_electrode_energy_distribution():
    """Atoms from a 300 eV mono-energetic source crossing the 50 mm gap
    (4 ns steps, run to deposition within 3000 steps): the energy
    distribution of the atoms deposited on the far electrode passes a
    two-sample KS test against the oracle's at p > 0.01."""
    cfg = W.tp_transport(n_atoms=20_000)
    cfg.update(cap_tp=20_000, n_e0=0, n_i0=0, tp_dt=4e-9, sort_every_tp=100)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=10, cap_tp=20_000)
    d.tp_launch(20_000, 300.0)
    orc.tp_launch(20_000, 300.0)
    d.tp_step(3000, count_alive=False)
    orc.tp_step(3000, 4e-9)
    p, n1, n2 = _ks_hist(d.diag("sputter_e_r"), orc.diag("sputter_e_r"))
    assert n1 > 1000 and p > 0.01, (p, n1, n2)
    tpd, tpo = d.diag("tp_dens"), orc.diag("tp_dens")
    from helpers import rel_l2
    assert rel_l2(tpd, tpo) < 0.03
    d.close()


# ------------------------------------------------------------------ error paths
def test_capacity_overflow_is_reported_and_state_stays_consistent():
    """Ionisations beyond the slot capacity are dropped as pairs and reported
    by pic_sync as a capacity error; the charge bookkeeping stays exact."""
    import paper_1607_04069_gb300 as P
    ncell = 64
    cfg = W.ccp_small(n_per_species=1000)
    cfg.update(n_cells=ncell, pressure_pa=30.0, gap_m=1.0, dt=1e-8, n_e0=0, n_i0=0,
               cap_e=20_010, cap_i=20_010, sort_every_e=0, sort_every_i=0)
    d = gpu_discharge(cfg)
    st = W.random_particles(20_000, ncell, 0, math.sqrt(60 * QE / ME), 8, 64)
    d.set_species(0, st["pos"], st["vx"], st["vy"], st["vz"], st["id"])
    d.set_field(np.zeros(ncell + 1))
    d.step(1)
    with pytest.raises(P.PicError) as e:
        d.sync()
    assert e.value.code == -4
    f = d.get_field()
    ne, ni = len(d.get_species(0)["id"]), len(d.get_species(1)["id"])
    assert int(f["q_e"].sum()) == 2**32 * ne and int(f["q_i"].sum()) == 2**32 * ni
    assert ne - ni == 20_000 - d.counters()["imp_e_l"] - d.counters()["imp_e_r"] + d.counters()["imp_i_l"] + d.counters()["imp_i_r"]
    d.sync()                   # the error is reported once
    d.close()


def test_tp_step_bounded_wait_runs_out_and_is_reported():
    """The TP step's waits on its bulk copies are bounded.  One warp that
    issues no copies waits until its limit runs out: the launch completes,
    pic_sync reports PIC_ERR_TIMEOUT once, that warp's atoms stay where they
    were, and the next steps, on the same context, move them again."""
    import paper_1607_04069_gb300 as P
    n = 1_000_000
    tc = W.tp_transport(n_atoms=n)
    tc.update(cap_tp=n + 1024, n_e0=0, n_i0=0, sort_every_tp=0, tp_mode=0)
    d = P.Discharge(P.params_from_workload(tc))
    d.tp_launch(n, 300.0)
    d.tp_step(2, count_alive=False)
    d.sync()

    def positions():
        sp = d.get_species(2)
        order = np.argsort(sp["id"])
        return sp["id"][order], sp["xi"][order]

    id0, x0 = positions()
    d.test_wait_timeout(True)
    d.tp_step(1, count_alive=False)
    with pytest.raises(P.PicError) as e:
        d.sync()
    assert e.value.code == -9
    d.sync()                                   # reported once
    d.test_wait_timeout(False)
    id1, x1 = positions()
    _, a, b = np.intersect1d(id0, id1, assume_unique=True, return_indices=True)
    still = id1[b][x1[b] == x0[a]]
    assert 0 < len(still) < n // 1000          # one warp's run of groups did not move
    alive = d.tp_step(3)
    d.sync()
    id2, x2 = positions()
    _, a, b = np.intersect1d(id1, id2, assume_unique=True, return_indices=True)
    moved = x2[b] != x1[a]
    assert moved[np.isin(id1[a], still)].all()
    c = d.counters()
    assert c["tp_dep_l"] + c["tp_dep_r"] + alive == n
    d.close()


def test_atoms_in_flight_counts_coupled_births():
    """tp_step's count of atoms in flight includes the atoms that ion impacts
    sputtered inside the step launch (counted per CTA there): it equals the
    atoms actually held, and launched = deposited + in flight."""
    cfg = W.ccp_sputter(n_per_species=20_000, n_cells=64, seed=95)
    cfg.update(rf_volt_v=1000.0, dt=W.T_RF / 400, tp_every=20, sort_every_tp=0)
    d = gpu_discharge(cfg)
    d.step(1600)
    alive = d.tp_step(1)
    c = d.counters()
    held = len(d.get_species(2)["id"])
    assert c["sputtered_l"] + c["sputtered_r"] > 100
    assert alive == held == c["sputtered_l"] + c["sputtered_r"] - c["tp_dep_l"] - c["tp_dep_r"]
    d.close()
