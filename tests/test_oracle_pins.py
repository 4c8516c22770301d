"""Pins of the FP64 oracle against things other than itself: published
known-answer vectors, values printed in the paper, closed forms, exact
invariants and textbook kinetic theory.  CPU only.

Each test names the part of the paper (arXiv:1607.04069) the pinned oracle
function implements.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special, stats

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
QE, ME, AMU, KB, EPS0 = 1.602176634e-19, 9.1093837015e-31, 1.66053906660e-27, 1.380649e-23, 8.8541878128e-12
MAR, MAL = 39.948 * AMU, 26.98 * AMU


def prm(**kw):
    p = dict(L=0.05, p=0.0, Tg=300.0, f=13.56e6, V0=0.0, w=0.0, dt=1e-10, te0=2.0, ti0=0.026,
             tp_dt=1e-9, sigma_tp=3e-19, seed=7, ncell=1024, sputter=0, tp_every=0, diag_every=1)
    p.update(kw)
    return p


def load(orc, s, xi, v, ids=None):
    n = len(xi)
    if ids is None:
        ids = np.arange(n, dtype=np.uint64) | np.uint64([0, 1 << 62, 2 << 62][s])
    orc.set_species(s, xi, v[0], v[1], v[2], ids)


# ------------------------------------------------------------------ RNG
def test_philox_known_answers():
    """Philox4x32-10 (Salmon et al. SC'11) against its published KAT vectors."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gas_density_printed_in_paper():
    """n = p/(k_B T) reproduces the Ar density the paper prints (Sec. 'Simulation Scenario')."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_gas_density.txt"))
            if l.strip() and not l.startswith("#")]
    p, T, n_cm3, tol = map(float, rows[0])
    orc = O.Oracle(prm(p=p, Tg=T), 1, 1)
    n = orc.derived()["n_gas"] * 1e-6
    assert abs(n / n_cm3 - 1.0) < tol


# ------------------------------------------------------------------ charge assignment
def test_deposit_conserves_charge_and_dipole_exactly():
    """Linear weighting (Sec. 'Charge Assignment') conserves each particle's
    charge (2^32 per particle) and, for positions on the 2^-32 grid, the
    first moment exactly: sum_m m q_m = 2^32 sum_k xi_k."""
    rng = np.random.default_rng(3)
    N = 1024
    pos = rng.integers(1, 2**32, size=50_000, dtype=np.uint64)
    xi = pos.astype(np.float64) * (N / 2.0**32)
    q = O.deposit(xi, N)
    assert int(q.sum()) == 2**32 * len(xi)
    lhs = sum(int(m) * int(qm) for m, qm in enumerate(q))
    rhs = sum(int(p) for p in pos) * N          # 2^32 * sum(xi) with xi = pos N / 2^32
    assert lhs == rhs
    assert (q >= 0).all()


def test_deposit_special_positions():
    """A particle on a node deposits everything there; one at mid-cell splits evenly;
    a removed particle (xi < 0) deposits nothing."""
    q = O.deposit(np.array([5.0, 7.5, -1.0]), 16)
    assert q[5] == 2**32 and q[6] == 0
    assert q[7] == 2**31 and q[8] == 2**31
    assert q.sum() == 2 * 2**32


# ------------------------------------------------------------------ field solve
def test_poisson_constant_rho_matches_closed_form():
    """rho = const: phi = V_L (1 - x/L) + rho0 x (L - x)/(2 eps0), reproduced
    exactly by the discrete scheme (Sec. 'EM Field Solver'); E from the
    central difference and the half-cell Gauss rule is exact too."""
    N, L, w, VL = 256, 0.05, 1e11, 123.0
    dx = L / N
    Q = 3_000_000 * 2**32 // 1000
    q_i = np.full(N + 1, Q, dtype=np.int64)
    q_i[0] = q_i[N] = Q // 2                      # half-volume boundary nodes
    q_e = np.zeros(N + 1, dtype=np.int64)
    phi, E = O.poisson(N, dx, w, q_i, q_e, VL)
    rho0 = QE * w * Q / (2**32 * dx)
    x = np.arange(N + 1) * dx
    phi_ref = VL * (1 - x / L) + rho0 * x * (L - x) / (2 * EPS0)
    E_ref = VL / L - rho0 * (L - 2 * x) / (2 * EPS0)
    scale = np.abs(phi_ref).max()
    assert np.abs(phi - phi_ref).max() / scale < 1e-12
    assert np.abs(E - E_ref).max() / np.abs(E_ref).max() < 1e-10


def test_poisson_sine_matches_discrete_eigensolution():
    """rho_m = rho0 sin(pi x_m / L): phi_m = rho0 dx^2 sin(pi x_m/L) /
    (2 eps0 (1 - cos(pi dx / L))) solves the discrete equation exactly."""
    N, L, w = 512, 0.05, 1e11
    dx = L / N
    x = np.arange(N + 1) * dx
    amp = 1e15
    q_i = np.rint(amp * np.sin(np.pi * x / L)).astype(np.int64)
    q_i[0] = q_i[N] = 0
    rho = QE * w * q_i / (2**32 * dx)
    phi, _ = O.poisson(N, dx, w, q_i, np.zeros(N + 1, dtype=np.int64), 0.0)
    rho0 = QE * w * amp / (2**32 * dx)
    phi_ref = rho0 * dx**2 * np.sin(np.pi * x / L) / (2 * EPS0 * (1 - np.cos(np.pi * dx / L)))
    assert np.abs(phi - phi_ref).max() / np.abs(phi_ref).max() < 1e-9   # rint of q_i: 1e-15 rel


@pytest.mark.parametrize("N", [128, 1024, 4096])
def test_poisson_double_sum_identity_random_charge(N):
    """Thomas result against the independent double prefix sum
    phi_m = phi_0 + m D0 - (dx^2/eps0) sum_{k<m} S_k, evaluated exactly in
    rationals.  The FP64 Thomas error grows with the Laplacian's condition
    number (~N^2): bound max(1e-12, N^2 eps / 100)."""
    rng = np.random.default_rng(11)
    L, w, VL = 0.025, 1.25e12, -87.5
    dx = L / N
    q_i = rng.integers(0, 2**44, size=N + 1, dtype=np.int64)
    q_e = rng.integers(0, 2**44, size=N + 1, dtype=np.int64)
    phi, E = O.poisson(N, dx, w, q_i, q_e, VL)
    A = Fraction(dx) * Fraction(QE) * Fraction(w) / (2**32 * Fraction(EPS0))  # dx^2 rho / eps0 per unit q
    qn = [int(a) - int(b) for a, b in zip(q_i, q_e)]
    S = [0] * (N + 1)
    for m in range(1, N + 1):
        S[m] = S[m - 1] + qn[m]
    T = [0] * (N + 1)
    for m in range(1, N + 1):
        T[m] = T[m - 1] + S[m - 1]
    D0 = (Fraction(0) - Fraction(VL) + A * T[N]) / N
    ref = [float(Fraction(VL) + m * D0 - A * T[m]) for m in range(N + 1)]
    ref = np.array(ref)
    assert np.abs(phi - ref).max() / np.abs(ref).max() < max(1e-12, N * N * 2.2e-16 / 100)
    Eref = np.array([float(-(2 * D0 - A * (S[m] + S[m - 1])) / (2 * Fraction(dx))) for m in range(1, N)])
    assert np.abs(E[1:N] - Eref).max() / np.abs(Eref).max() < max(1e-10, N * N * 2.2e-16)


# ------------------------------------------------------------------ push / interpolation
def test_leapfrog_uniform_field_closed_form():
    """Eqs. pushinr/pushinv in a uniform field with v^{-1/2} = v0 - a dt/2:
    x_n = x0 + v0 n dt + a (n dt)^2 / 2 exactly (FP64 round-off only)."""
    N, L, dt = 1024, 1.0, 1e-10
    orc = O.Oracle(prm(L=L, ncell=N, dt=dt), 4, 4)
    dx = L / N
    E0 = 35.0
    x0 = np.array([0.3, 0.5, 0.61, 0.42])
    v0 = np.array([1e5, -2e5, 0.0, 3e5])
    a = -QE / ME * E0
    load(orc, 0, x0 / dx, [v0 - a * dt / 2, v0 * 0, v0 * 0])
    for n in range(1, 201):
        orc.set_field(np.full(N + 1, E0))
        orc.step(1)
        sp = orc.get_species(0)
        ref = x0 + v0 * n * dt + a * (n * dt) ** 2 / 2
        assert np.allclose(sp["xi"] * dx, ref, rtol=1e-11, atol=1e-13)


def test_leapfrog_linear_field_discrete_oscillator():
    """Field interpolation (Sec. 'Field Interpolation') is exact for a field
    linear in x; leapfrog then gives the discrete oscillator
    x_n - xc = X cos(n theta), cos(theta) = 1 - (w dt)^2 / 2."""
    N, L, dt = 256, 0.01, 2e-11
    dx = L / N
    orc = O.Oracle(prm(L=L, ncell=N, dt=dt), 3, 3)
    xc, kappa = 0.005, 2e6               # E = kappa (x - xc): restoring for electrons
    om2 = QE / ME * kappa
    th = math.acos(1 - om2 * dt * dt / 2)
    X = np.array([1e-3, -2e-3, 0.5e-3])
    a0 = -om2 * X
    vm = X * (math.cos(th) - 1) / dt - a0 * dt
    load(orc, 0, (xc + X) / dx, [vm, 0 * X, 0 * X])
    Enode = kappa * (np.arange(N + 1) * dx - xc)
    for n in range(1, 301):
        orc.set_field(Enode)
        orc.step(1)
        x = orc.get_species(0)["xi"] * dx
        assert np.allclose(x - xc, X * np.cos(n * th), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ initial loading
def test_initial_loading_is_uniform_and_maxwellian():
    """Uniform positions and Box-Muller Maxwellian velocities
    (Sec. 'Kinetic Particle Simulation'): KS of x against U(0,L), of each
    velocity component against N(0, kT/m), and <E> = 3/2 T."""
    N = 64
    orc = O.Oracle(prm(ncell=N, seed=8), 100_000, 1)
    orc.init_species(0, 100_000, 2.0)
    sp = orc.get_species(0)
    assert stats.kstest(sp["xi"] / N, "uniform").pvalue > 1e-3
    vth = math.sqrt(2.0 * QE / ME)
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(sp[c] / vth, "norm").pvalue > 1e-3
    E = 0.5 * ME * (sp["vx"]**2 + sp["vy"]**2 + sp["vz"]**2) / QE
    assert abs(E.mean() / 3.0 - 1) < 4 * math.sqrt(2 / 3 / len(E))
    assert len(np.unique(sp["id"])) == len(E)


# ------------------------------------------------------------------ null-collision MCC
def test_cross_section_shapes():
    """Lotz-form ionisation peaks at eps = e*I with a q/(e I^2); thresholds hold."""
    s = O.sigma_e(11.5)
    assert s[1] == 0 and s[2] == 0 and s[0] == 1e-19
    assert O.sigma_e(15.8)[2] == 0
    eps = np.linspace(16, 200, 20001)
    si = np.array([O.sigma_e(e)[2] for e in eps])
    assert abs(eps[si.argmax()] / (math.e * 15.8) - 1) < 1e-3
    assert abs(si.max() / (4.5e-18 * 6 / (math.e * 15.8**2)) - 1) < 1e-6
    assert abs(O.sigma_e(1e9)[1] / 1e-20 - 1) < 1e-7
    assert abs(O.sigma_i(1.0) - 5e-19) < 1e-30 and abs(O.sigma_i(4.0) - 2.5e-19) < 1e-30


def _mono(n, speed, rng):
    d = rng.standard_normal((3, n))
    d /= np.linalg.norm(d, axis=0)
    return d * speed


def test_candidate_gap_is_geometric_with_the_per_step_probability():
    """The steps between null-collision candidates: every step is a candidate
    with probability P = 1 - exp(-nu_max dt) independently of the others
    (Sec. "Particle Collisions"), so gap n has probability (1-P)^(n-1) P.
    Checked by a chi-square test over gaps 1..40 plus the tail, the mean
    1/P, and the exact special cases P(gap=1) boundary and lam = 0."""
    lam = 0.05
    P = 1 - math.exp(-lam)
    words = [int(O.philox([k, 7, 3, 7], [11, 13])[0]) for k in range(60_000)]
    g = np.array([O.gap(lam, w) for w in words])
    assert g.min() >= 1
    nmax = 40
    obs = np.bincount(np.minimum(g, nmax + 1), minlength=nmax + 2)[1:]
    pn = [(1 - P) ** (n - 1) * P for n in range(1, nmax + 1)]
    exp_ = np.array(pn + [(1 - P) ** nmax]) * len(g)
    chi2 = ((obs - exp_) ** 2 / exp_).sum()
    assert stats.chi2.sf(chi2, len(exp_) - 1) > 1e-3
    assert abs(g.mean() - 1 / P) < 5 * math.sqrt((1 - P) / P**2 / len(g))
    # u = (w >> 9 + 1/2) 2^-23 close to 1 gives gap 1; a word with u <= exp(-lam) gives gap >= 2
    assert O.gap(lam, 0xFFFFFFFF) == 1
    w_edge = int((math.exp(-lam) / 2**-23 - 0.5)) << 9
    assert O.gap(lam, w_edge) == 2
    assert O.gap(0.0, 12345) == 2**31 - 1


@pytest.mark.parametrize("mode", [0, 1])
def test_electron_null_collision_rate_constant_sigma(mode):
    """Below every threshold only elastic scattering (constant sigma) is real:
    the real-collision fraction per step is P_max nu_el(v) / nu_max (binomial),
    with candidates by geometric gaps (mode 0) and by the paper's per-step
    test R <= P_c,tot (mode 1)."""
    rng = np.random.default_rng(5)
    n, p, T, dt = 200_000, 3.0, 300.0, 1e-9
    orc = O.Oracle(prm(L=1.0, ncell=1024, p=p, Tg=T, dt=dt, coll_mode=mode), n, 1)
    eps = 5.0
    v = math.sqrt(2 * eps * QE / ME)
    load(orc, 0, np.full(n, 512.3), _mono(n, v, rng))
    orc.step(1)
    c = orc.counters()
    ngas = p / (KB * T)
    sig_max = 1e-19 + 1e-20 + 4.5e-18 * 6 / (math.e * 15.8**2)
    nu_max = ngas * sig_max * math.sqrt(2 * 100.0 * QE / ME)           # eps_max = 2 V0 + 100 eV
    pexp = (1 - math.exp(-nu_max * dt)) * ngas * 1e-19 * v / nu_max
    assert c["excitation"] == 0 and c["ionizations"] == 0
    assert abs(c["elastic"] - n * pexp) < 4.5 * math.sqrt(n * pexp * (1 - pexp))


@pytest.mark.parametrize("mode", [0, 1])
def test_ion_candidate_rate_is_velocity_independent(mode):
    """Ar+: sigma(eps) g is constant, so the collision rate does not depend on
    the velocity and CX and isotropic scattering each take half (candidates by
    geometric gaps, mode 0, or by the per-step test, mode 1)."""
    n, p, T, dt = 200_000, 3.0, 300.0, 1e-7
    ngas = p / (KB * T)
    nu = 2 * ngas * 5e-19 * math.sqrt(2 * QE / (MAR / 2))
    pexp = 1 - math.exp(-nu * dt)
    for speed in (100.0, 3000.0):
        rng = np.random.default_rng(int(speed))
        orc = O.Oracle(prm(L=10.0, ncell=1024, p=p, Tg=T, dt=dt, seed=int(speed), coll_mode=mode), 1, n)
        load(orc, 1, np.full(n, 400.0), _mono(n, speed, rng))
        orc.step(1)
        c = orc.counters()
        tot = c["cx"] + c["iso"]
        assert abs(tot - n * pexp) < 4.5 * math.sqrt(n * pexp * (1 - pexp))
        assert abs(c["cx"] - tot / 2) < 4.5 * math.sqrt(tot / 4)


def test_candidates_per_step_are_binomial_in_both_modes():
    """Sec. "Particle Collisions": every step each particle is a null-collision
    candidate with probability P_c,tot = 1 - exp(-nu_max dt), independently of
    the other steps and particles, so the candidates of one step are
    Binomial(N, P).  Ar+ candidates are all real collisions (sigma g is
    constant), so the per-step CX + isotropic counts show them.  Both the
    paper's per-step test (mode 1) and the geometric gaps (mode 0) must give
    the binomial mean and variance step by step, and the same total."""
    n, p, T, steps = 50_000, 3.0, 300.0, 60
    ngas = p / (KB * T)
    nu = 2 * ngas * 5e-19 * math.sqrt(2 * QE / (MAR / 2))
    dt = 0.02 / nu
    P = 1 - math.exp(-nu * dt)
    totals = []
    for mode in (0, 1):
        rng = np.random.default_rng(71)
        orc = O.Oracle(prm(L=10.0, ncell=1024, p=p, Tg=T, dt=dt, seed=71, coll_mode=mode), 1, n)
        load(orc, 1, np.full(n, 400.0) + rng.uniform(-1, 1, n), _mono(n, 500.0, rng))
        per, last = [], 0
        for _ in range(steps):
            orc.step(1)
            c = orc.counters()
            per.append(c["cx"] + c["iso"] - last)
            last = c["cx"] + c["iso"]
        per = np.array(per, dtype=float)
        mean, var = n * P, n * P * (1 - P)
        assert abs(per.mean() - mean) < 4.5 * math.sqrt(var / steps), (mode, per.mean(), mean)
        chi2 = ((per - mean) ** 2 / var).sum()                 # dispersion: chi^2 with `steps` dof
        assert 1e-3 < stats.chi2.cdf(chi2, steps) < 1 - 1e-3, (mode, chi2)
        totals.append(per.sum())
    assert abs(totals[0] - totals[1]) < 4.5 * math.sqrt(2 * steps * n * P * (1 - P))


def test_literal_and_geometric_modes_agree_over_the_discharge():
    """The 25 mm / 128-cell / 100 V / 3 Pa discharge, 20k + 20k, 20 RF periods,
    with the paper's per-step candidate test (mode 1) and with geometric gaps
    (mode 0), three seeds each: the time-averaged potential and densities of
    the two modes differ by no more than the seed-to-seed spread allows (the
    difference of two three-seed means has the spread of one pair over sqrt(3);
    2.5 times that), and the pooled ion energy distributions at both
    electrodes pass a two-sample KS test at p > 0.01."""
    from helpers import ks_hist, oracle_pool_run
    from paper_1607_04069_gb300 import workloads as W
    seeds = (1235, 3001, 3002)
    cfgs = [dict(W.ccp_small(seed=s), coll_mode=m) for m in (0, 1) for s in seeds]
    res = oracle_pool_run(cfgs, 4000, 4000)
    geo, lit = res[:3], res[3:]
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for k in ("phi", "n_e", "n_i"):
        pairs = [rel(a[k], b[k]) for grp in (geo, lit) for a, b in ((grp[0], grp[1]), (grp[0], grp[2]),
                                                                   (grp[1], grp[2]))]
        spread = float(np.mean(pairs))
        m0 = np.mean([r[k] for r in geo], axis=0)
        m1 = np.mean([r[k] for r in lit], axis=0)
        assert rel(m1, m0) < 2.5 * spread / math.sqrt(3), (k, rel(m1, m0), spread)
        assert rel(m1, m0) < 0.03, k
    for k in ("iedf_l", "iedf_r"):
        pv, D, n1, n2 = ks_hist(sum(r[k] for r in geo), sum(r[k] for r in lit))
        assert n1 > 3000 and n2 > 3000 and pv > 0.01, (k, pv, n1, n2)


def test_ion_thermal_relaxation():
    """Field off, ions at E0 >> kT: <E>_n = E_g + (E0 - E_g)(1 - 3/4 P_max)^n,
    E_g = 3/2 kT; after many steps the energy follows the chi^2_3 law."""
    n, p, T, dt = 60_000, 3.0, 300.0, 1e-7
    rng = np.random.default_rng(9)
    orc = O.Oracle(prm(L=100.0, ncell=1024, p=p, Tg=T, dt=dt), 1, n)
    E0 = 1.0
    load(orc, 1, np.full(n, 512.0) + rng.uniform(-1, 1, n), _mono(n, math.sqrt(2 * E0 * QE / MAR), rng))
    ngas = p / (KB * T)
    P = 1 - math.exp(-2 * ngas * 5e-19 * math.sqrt(2 * QE / (MAR / 2)) * dt)
    Eg = 1.5 * KB * T / QE
    for steps in (5, 10):
        orc.step(5)
        sp = orc.get_species(1)
        E = 0.5 * MAR * (sp["vx"]**2 + sp["vy"]**2 + sp["vz"]**2) / QE
        ref = Eg + (E0 - Eg) * (1 - 0.75 * P) ** steps
        assert abs(E.mean() / ref - 1) < 0.01
    orc.step(90)
    sp = orc.get_species(1)
    E = 0.5 * MAR * (sp["vx"]**2 + sp["vy"]**2 + sp["vz"]**2) / QE
    kT = KB * T / QE
    assert stats.kstest(E / kT, stats.gamma(1.5).cdf).pvalue > 1e-3


def test_electron_elastic_energy_loss():
    """Mean fractional energy loss per elastic collision = 2 m_e / M (<1 - cos chi> = 1)."""
    rng = np.random.default_rng(21)
    n, dt = 200_000, 1e-9
    orc = O.Oracle(prm(L=1.0, ncell=1024, p=3.0, dt=dt), n, 1)
    v = math.sqrt(2 * 5.0 * QE / ME)
    v0 = _mono(n, v, rng)
    load(orc, 0, np.full(n, 512.7), v0)
    orc.step(1)
    sp = orc.get_species(0)
    v1 = np.stack([sp["vx"], sp["vy"], sp["vz"]])
    hit = np.any(v1 != v0, axis=0)
    loss = 1 - (v1[:, hit]**2).sum(0) / v**2
    ref = 2 * ME / MAR
    se = ref * math.sqrt(1 / 3) / math.sqrt(hit.sum())
    assert hit.sum() == orc.counters()["elastic"]
    assert abs(loss.mean() - ref) < 5 * se


@pytest.mark.parametrize("mode", [0, 1])
def test_inelastic_bookkeeping_at_50eV(mode):
    """At 50 eV: process fractions follow sigma_el : sigma_exc : sigma_ion,
    excitation removes exactly 11.5 eV, ionisation removes 15.8 eV and
    creates one e-/Ar+ pair at the parent's position (both candidate modes)."""
    rng = np.random.default_rng(33)
    n, dt = 200_000, 2e-10
    orc = O.Oracle(prm(L=1.0, ncell=1024, p=3.0, dt=dt, coll_mode=mode), 2 * n, n)
    eps = 50.0
    v = math.sqrt(2 * eps * QE / ME)
    v0 = _mono(n, v, rng)
    load(orc, 0, np.full(n, 512.25), v0)
    orc.step(1)
    c = orc.counters()
    s_el, s_exc, s_ion = 1e-19, 1e-20 * (1 - 11.5 / eps), 4.5e-18 * 6 * math.log(eps / 15.8) / (eps * 15.8)
    tot = c["elastic"] + c["excitation"] + c["ionizations"]
    for k, s in (("elastic", s_el), ("excitation", s_exc), ("ionizations", s_ion)):
        pk = s / (s_el + s_exc + s_ion)
        assert abs(c[k] - tot * pk) < 4.5 * math.sqrt(tot * pk * (1 - pk))
    e = orc.get_species(0)
    i = orc.get_species(1)
    assert len(e["xi"]) == n + c["ionizations"] and len(i["xi"]) == c["ionizations"]
    Ee = 0.5 * ME * (e["vx"]**2 + e["vy"]**2 + e["vz"]**2) / QE
    exc = np.abs(Ee[:n] - (eps - 11.5)) < 1e-9
    assert exc.sum() == c["excitation"]
    # energy balance over all electrons: -11.5 per excitation, -15.8 per ionisation,
    # elastic losses of mean 2 m/M eps each
    dE = Ee.sum() - n * eps
    exp_dE = -11.5 * c["excitation"] - 15.8 * c["ionizations"] - 2 * ME / MAR * eps * c["elastic"]
    assert abs(dE - exp_dE) < 6 * 2 * ME / MAR * eps * math.sqrt(c["elastic"] / 3) + 1e-6 * n
    # the pair is born at the parent's position x^{l+1}, electron and ion together
    assert np.array_equal(e["xi"][n:], i["xi"])
    assert np.isin(i["xi"], e["xi"][:n]).all()


def test_ionisation_products():
    """Ionisation (Sec. 'Particle Collisions'): the energy left after the
    15.8 eV threshold is shared by the scattered and the ejected electron,
    the ejected one's share uniform on [0, eps - 15.8]; the new ion is drawn
    from the gas Maxwellian (each velocity component normal with variance
    k_B T_g / M_Ar) at the parent's position."""
    rng = np.random.default_rng(35)
    n, dt, eps, Tg = 200_000, 2e-10, 50.0, 300.0
    orc = O.Oracle(prm(L=1.0, ncell=1024, p=3.0, Tg=Tg, dt=dt), 2 * n, n)
    load(orc, 0, np.full(n, 512.25), _mono(n, math.sqrt(2 * eps * QE / ME), rng))
    orc.step(1)
    e, i = orc.get_species(0), orc.get_species(1)
    k = orc.counters()["ionizations"]
    assert k > 2000 and len(i["xi"]) == k
    Ee = 0.5 * ME * (e["vx"]**2 + e["vy"]**2 + e["vz"]**2) / QE
    ej = Ee[n:]                                               # the ejected electrons, in birth order
    assert stats.kstest(ej / (eps - 15.8), "uniform").pvalue > 1e-3
    # each parent sits at its child's position and carries the rest of the energy
    par = {x: Ee[j] for j, x in enumerate(e["xi"][:n])}
    pairs = np.array([par[x] + ej[m] for m, x in enumerate(e["xi"][n:])])
    assert np.allclose(pairs, eps - 15.8, rtol=1e-5)
    sig = math.sqrt(KB * Tg / MAR)
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(i[c] / sig, "norm").pvalue > 1e-3
    assert abs(np.mean(i["vx"]**2 + i["vy"]**2 + i["vz"]**2) / (3 * sig**2) - 1) < 5 * math.sqrt(2 / (3 * k))


# ------------------------------------------------------------------ walls and sputtering
def test_sputter_yield_values():
    assert O.sputter_yield(30.0) == 0.0 and O.sputter_yield(10.0) == 0.0
    assert abs(O.sputter_yield(300.0) - 0.3) < 1e-15
    assert abs(O.sputter_yield(120.0) - 0.1 * math.sqrt(3)) < 1e-15


@pytest.mark.parametrize("E_ion,Y", [(300.0, 0.3), (12030.0, 2.0)])
def test_sputter_births_per_impact(E_ion, Y):
    """Ions reaching the target with energy E: mean number of sputtered atoms
    per impact = Y(E) (binomial); an integer yield gives exactly Y each."""
    n = 100_000
    rng = np.random.default_rng(int(E_ion))
    orc = O.Oracle(prm(sputter=1, V0=0.0, dt=1e-10), 1, n, 3 * n)
    v = math.sqrt(2 * E_ion * QE / MAR)
    load(orc, 1, rng.uniform(1e-3, 2e-3, n), [np.full(n, -v), np.zeros(n), np.zeros(n)])
    orc.step(1)
    c = orc.counters()
    assert c["imp_i_l"] == n
    if Y == int(Y):
        assert c["sputtered_l"] == int(Y) * n
    else:
        assert abs(c["sputtered_l"] - n * Y) < 4.5 * math.sqrt(n * Y * (1 - Y))
    tp = orc.get_species(2)
    Lam = 4 * MAR * MAL / (MAR + MAL) ** 2
    Es = 0.5 * MAL * (tp["vx"]**2 + tp["vy"]**2 + tp["vz"]**2) / QE
    assert (tp["vx"] > 0).all() and (Es <= Lam * E_ion * (1 + 1e-12)).all()


def test_impact_and_energy_histograms_place_known_particles():
    """Ion impacts (Sec. 'Wall Interactions': energy 1/2 M |v|^2 and angle to
    the electrode normal, at the electrode reached; IEDF on [0, 2 V0] in 512
    bins, IEADF 128 x 90 one-degree bins) and the EEDF (electrons in the
    central 10 % of the gap, 0.25 eV bins) put particles of chosen energy and
    angle in the bins those values name.  At step 0 the source voltage is 0
    and zero weight leaves no space charge, so nothing accelerates them."""
    N, L, V0 = 128, 0.025, 100.0
    dt = 1.0 / 13.56e6 / 400
    orc = O.Oracle(prm(L=L, ncell=N, dt=dt, V0=V0), 8, 8)
    Ei = np.array([10.3, 55.6, 149.2, 199.7])             # eV
    th = np.array([0.4, 30.5, 60.2, 88.7])                # degrees from the normal
    sp = np.sqrt(2 * Ei * QE / MAR)
    out = np.array([-1.0, -1.0, 1.0, 1.0])                # toward x = 0, x = 0, x = L, x = L
    xi = np.where(out < 0, 1e-4, N - 1e-4)                # within one step of the electrode
    load(orc, 1, xi, [out * sp * np.cos(np.radians(th)), sp * np.sin(np.radians(th)), 0 * sp])
    Ee = np.array([0.6, 7.3, 33.1, 63.9, 12.0])           # the last one outside the window
    ve = np.sqrt(2 * Ee * QE / ME)
    load(orc, 0, np.array([64.0, 60.0, 66.5, 69.9, 0.3 * N]), [0 * ve, 0.6 * ve, 0.8 * ve])
    orc.step(1)
    c = orc.counters()
    assert c["imp_i_l"] == 2 and c["imp_i_r"] == 2 and c["imp_e_l"] == c["imp_e_r"] == 0
    want_iedf = {"l": [26, 142], "r": [381, 511]}          # floor(E / 200 eV * 512)
    want_ieadf = {"l": [(6, 0), (35, 30)], "r": [(95, 60), (127, 88)]}   # floor(E / 200 * 128), floor(theta)
    for side in "lr":
        h = orc.diag("iedf_" + side)
        assert h.shape == (512,) and h.sum() == 2
        assert sorted(np.nonzero(h)[0].tolist()) == want_iedf[side]
        h2 = orc.diag("ieadf_" + side).reshape(128, 90)
        assert h2.sum() == 2
        assert sorted(zip(*[a.tolist() for a in np.nonzero(h2)])) == want_ieadf[side]
    e = orc.diag("eedf")
    assert e.shape == (256,) and e.sum() == 4
    assert np.nonzero(e)[0].tolist() == [2, 29, 132, 255]  # floor(E / 0.25 eV)


def test_thompson_cosine_distributions():
    """Sputtered-atom launch: energy follows the truncated Thompson CDF
    (E/(E+Ub))^2 / (Emax/(Emax+Ub))^2; cos(theta) law gives <cos theta> = 2/3
    and P(theta < t) = sin^2 t."""
    n = 200_000
    orc = O.Oracle(prm(), 1, 1, n)
    orc.tp_launch(n, 300.0)
    tp = orc.get_species(2)
    v2 = tp["vx"]**2 + tp["vy"]**2 + tp["vz"]**2
    E = 0.5 * MAL * v2 / QE
    Ub = 3.4
    Emax = 4 * MAR * MAL / (MAR + MAL) ** 2 * 300.0
    cdf = lambda e: (np.clip(e, 0, Emax) / (np.clip(e, 0, Emax) + Ub))**2 / (Emax / (Emax + Ub))**2
    assert stats.kstest(E, cdf).pvalue > 1e-3
    ct = tp["vx"] / np.sqrt(v2)
    assert (ct > 0).all()
    assert abs(ct.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / n)
    th = np.arccos(np.clip(ct, -1, 1))
    assert stats.kstest(th, lambda t: np.sin(np.clip(t, 0, np.pi / 2))**2).pvalue > 1e-3
    ph = np.arctan2(tp["vz"], tp["vy"])
    assert stats.kstest((ph + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


# ------------------------------------------------------------------ test particles
def test_tp_ballistic_flight_without_collisions():
    """sigma = 0: every atom reaches the far wall at the step it must,
    with its energy and angle recorded, and counts are conserved."""
    N, L, dt, K = 1024, 0.05, 1e-9, 37
    n = 1000
    orc = O.Oracle(prm(L=L, ncell=N, sigma_tp=0.0, p=0.5), 1, 1, n)
    vx = L / (K * dt) * (1 + 1e-9)
    load(orc, 2, np.full(n, N * 2.0**-32), [np.full(n, vx), np.zeros(n), np.zeros(n)])
    orc.tp_step(K - 1, dt)
    assert orc.counters()["n_tp"] == n
    orc.tp_step(1, dt)
    c = orc.counters()
    assert c["tp_dep_r"] == n and c["n_tp"] == 0 and c["tp_coll"] == 0
    ang = orc.diag("sputter_ang_r")
    assert ang[0] == n
    e = orc.diag("sputter_e_r")
    E = 0.5 * MAL * vx**2 / QE
    assert e[min(int(E / 300 * 600), 599)] == n


@pytest.mark.parametrize("tp_mode", [0, 1])
def test_tp_collision_rate_in_maxwellian_gas(tp_mode):
    """TP collision probability per step for speed v in a Maxwellian gas:
    n sigma <g> dt - (n sigma dt)^2 <g^2>/2 + O(3), with the textbook mean
    relative speed <g> = c[(s + 1/(2s)) erf(s) + exp(-s^2)/sqrt(pi)],
    s = v/c, c = sqrt(2kT/M) and <g^2> = v^2 + 3kT/M."""
    n, p, T, dt, sig = 400_000, 0.5, 300.0, 2e-8, 3e-19
    for v in (300.0, 2000.0):
        rng = np.random.default_rng(int(v))
        orc = O.Oracle(prm(L=100.0, ncell=1024, p=p, Tg=T, sigma_tp=sig, tp_mode=tp_mode), 1, 1, n)
        load(orc, 2, np.full(n, 512.0), _mono(n, v, rng))
        orc.tp_step(1, dt)
        ngas = p / (KB * T)
        c = math.sqrt(2 * KB * T / MAR)
        s = v / c
        g = c * ((s + 1 / (2 * s)) * special.erf(s) + math.exp(-s * s) / math.sqrt(math.pi))
        g2 = v * v + 3 * KB * T / MAR
        x = ngas * sig * dt
        pexp = x * g - x * x * g2 / 2
        got = orc.counters()["tp_coll"]
        assert abs(got - n * pexp) < 4.5 * math.sqrt(n * pexp)


def _rel_speed_density(g, v, c):
    """Density of g = |v - w| for a fixed velocity of magnitude v and w from
    the Maxwellian of most probable speed c (kinetic theory)."""
    return g / (v * c * math.sqrt(math.pi)) * (np.exp(-(g - v) ** 2 / c**2) - np.exp(-(g + v) ** 2 / c**2))


@pytest.mark.parametrize("model", [0, 1, 2])
def test_tp_candidate_thinning_gives_the_exact_per_step_law(model):
    """The thinned candidates of the TP step (tp_mode 0) reproduce the per-step
    law of Eq. collisionprobability1 with a sampled partner exactly, not only
    to first order: at P^ ~ 0.6 the collision probability of one step equals
    E_w[1 - exp(-n K dt g^alpha)], by quadrature over the density of the
    relative speed, within the binomial error, in both modes; and the
    post-collision speeds of the two modes have one distribution (KS).  Hard
    spheres, VHS and M1 (omega = 0.81)."""
    n, p, T, v = 200_000, 0.5, 300.0, 2000.0
    ngas = p / (KB * T)
    c = math.sqrt(2 * KB * T / MAR)
    kw = dict(L=100.0, ncell=1024, p=p, Tg=T, sigma_tp=3e-19, tp_model=model, dref=4.17e-10, omega=0.81,
              tref=273.0, seed=31 + model)
    probe = O.Oracle(prm(**kw), 1, 1, 1)
    alpha = 1.0 if model == 0 else 2.0 - 2.0 * 0.81
    K = probe.tp_sigma(1.0) if model else 3e-19
    ma = c**alpha * special.gamma(0.5 * (3 + alpha)) / special.gamma(1.5)
    dt = 0.6 / (ngas * K * (v**alpha + ma))                       # P^ = 0.6
    b = ngas * K * dt
    g = np.linspace(0.0, v + 12 * c, 400_001)
    fg = _rel_speed_density(g, v, c)
    assert abs(np.trapezoid(fg, g) - 1) < 1e-9
    P = float(np.trapezoid(fg * -np.expm1(-b * g**alpha), g))
    speeds = []
    for mode in (0, 1):
        rng = np.random.default_rng(77)
        orc = O.Oracle(prm(tp_mode=mode, **kw), 1, 1, n)
        load(orc, 2, np.full(n, 512.0), _mono(n, v, rng))
        orc.tp_step(1, dt)
        got = orc.counters()["tp_coll"]
        assert abs(got - n * P) < 4.5 * math.sqrt(n * P * (1 - P)), (mode, got, n * P)
        assert orc.counters()["numerics"] == 0
        sp = orc.get_species(2)
        vm = np.sqrt(sp["vx"]**2 + sp["vy"]**2 + sp["vz"]**2)
        speeds.append(vm[np.abs(vm - v) > 1e-6 * v])
    assert stats.ks_2samp(speeds[0], speeds[1]).pvalue > 1e-3


def test_tp_candidate_gap_is_geometric():
    """TP steps between candidates at the per-step probability P^: gap n has
    probability (1 - P^)^(n-1) P^ (chi-square over 1..40 and the tail, and the
    mean 1/P^); P^ >= 1 makes every step a candidate, P^ = 0 none."""
    Ph = 0.07
    words = [int(O.philox([k, 9, 4, 290], [5, 6])[0]) for k in range(60_000)]
    g = np.array([O.tp_gap(Ph, w) for w in words])
    assert g.min() >= 1
    nmax = 40
    obs = np.bincount(np.minimum(g, nmax + 1), minlength=nmax + 2)[1:]
    exp_ = np.array([(1 - Ph) ** (m - 1) * Ph for m in range(1, nmax + 1)] + [(1 - Ph) ** nmax]) * len(g)
    assert stats.chi2.sf(((obs - exp_) ** 2 / exp_).sum(), len(exp_) - 1) > 1e-3
    assert abs(g.mean() - 1 / Ph) < 5 * math.sqrt((1 - Ph) / Ph**2 / len(g))
    assert O.tp_gap(1.0, 123) == 1 and O.tp_gap(1.5, 123) == 1
    assert O.tp_gap(0.0, 123) == 2**31 - 1


@pytest.mark.parametrize("tp_mode", [0, 1])
def test_tp_thermalizes_to_gas_temperature(tp_mode):
    """Hard-sphere Al-Ar collisions relax the Al velocity distribution to a
    Maxwellian at the gas temperature: <v_x^2> = kT/M_Al (both collision
    modes; the thinned candidates need P^ <= 1, hence the shorter step)."""
    n, p, T = 40_000, 5.0, 300.0
    rng = np.random.default_rng(4)
    orc = O.Oracle(prm(L=1e6, ncell=1024, p=p, Tg=T, sigma_tp=3e-19, tp_mode=tp_mode), 1, 1, n)
    load(orc, 2, np.full(n, 512.0) + rng.uniform(-1, 1, n), _mono(n, math.sqrt(2 * 5 * QE / MAL), rng))
    if tp_mode == 1:
        orc.tp_step(300, 1e-6)        # P ~ 0.2 per step: ~60 collisions per atom
    else:
        orc.tp_step(3000, 1e-7)       # P^ <= 0.25 per step
    assert orc.counters()["numerics"] == 0
    tp = orc.get_species(2)
    ref = KB * T / MAL
    for comp in ("vx", "vy", "vz"):
        assert abs((tp[comp]**2).mean() / ref - 1) < 0.03


def test_tp_deposition_histograms_and_grid_moments():
    """TP diagnostics (Sec. 'Wall Interactions' and 'Limitations and
    Constraints' of the TPM): an atom that reaches an electrode is binned by
    its energy 1/2 M_Al |v|^2 (0.5 eV bins on [0, 300)) and its angle to the
    normal (1-degree bins) at that electrode; the grid moments of the atoms
    in flight give a mean-velocity moment equal to density times a uniform
    drift, and the density w n / L of a uniform load.  No gas: no collision."""
    N, L, w, dt = 32, 0.02, 1e12, 1e-9
    E = np.array([1.3, 47.6, 299.9, 12.2, 150.1])          # eV
    th = np.array([2.5, 45.3, 80.1, 10.7, 70.7])           # degrees from the normal
    out = np.array([1.0, 1.0, 1.0, -1.0, -1.0])            # three toward x = L, two toward x = 0
    sp = np.sqrt(2 * E * QE / MAL)
    n, u = 200_000, 500.0
    rng = np.random.default_rng(41)
    xi = np.concatenate([np.where(out > 0, N - 1e-4, 1e-4), rng.uniform(0.1, N - 0.1, n)])
    vx = np.concatenate([out * sp * np.cos(np.radians(th)), np.full(n, u)])
    vy = np.concatenate([sp * np.sin(np.radians(th)), rng.standard_normal(n) * 300.0])
    orc = O.Oracle(prm(L=L, ncell=N, w=w, p=0.0), 1, 1, n + 8)
    load(orc, 2, xi, [vx, vy, 0 * vy])
    orc.tp_step(3, dt)
    c = orc.counters()
    assert c["tp_dep_r"] == 3 and c["tp_dep_l"] == 2 and c["tp_coll"] == 0
    for side, bins, angs in (("r", [2, 95, 599], [2, 45, 80]), ("l", [24, 300], [10, 70])):
        he, ha = orc.diag("sputter_e_" + side), orc.diag("sputter_ang_" + side)
        assert he.shape == (600,) and ha.shape == (90,)
        assert np.nonzero(he)[0].tolist() == bins and he.sum() == len(bins)
        assert np.nonzero(ha)[0].tolist() == angs and ha.sum() == len(angs)
    dens, mom = orc.diag("tp_dens"), orc.diag("tp_vx")
    assert (dens > 0).all()
    assert np.allclose(mom, dens * u, rtol=1e-12, atol=0)
    n0 = w * n / (L * (N - 0.2) / N)                       # the loaded span is (0.1, N - 0.1) cells
    assert abs(dens[2:N - 1].mean() / n0 - 1) < 4 / math.sqrt(n)


# ------------------------------------------------------------------ conservation, diagnostics
def test_charge_and_particle_conservation_over_steps():
    """Every step: sum of deposits = 2^32 x alive particles per species;
    ionisation creates equal numbers of electrons and ions."""
    prmd = prm(L=0.025, ncell=128, p=3.0, V0=100.0, w=1.25e12 * 10, dt=1.0 / 13.56e6 / 400)
    orc = O.Oracle(prmd, 12_000, 12_000)
    orc.init_species(0, 2000, 2.0)
    orc.init_species(1, 2000, 0.026)
    orc.field()
    for _ in range(40):
        orc.step(5)
        f = orc.get_field()
        c = orc.counters()
        assert int(f["q_e"].sum()) == 2**32 * c["n_e"]
        assert int(f["q_i"].sum()) == 2**32 * c["n_i"]
        assert c["n_e"] + c["imp_e_l"] + c["imp_e_r"] == 2000 + c["ionizations"]
        assert c["n_i"] + c["imp_i_l"] + c["imp_i_r"] == 2000 + c["ionizations"]


@pytest.mark.parametrize("sigma_tp", [0.0, 3e-19])
def test_sputter_to_test_particle_coupling(sigma_tp):
    """The one-way coupling of the two modules (Sec. "Simulation Scenario",
    Fig. 3; Sec. "Wall Interactions" of the TPM): ion impacts launch atoms,
    and the atoms are advanced by a TP step of tp_every PIC steps after every
    tp_every-th PIC step (sub-cycling).  Two waves of 300 eV Ar+ impacts, at
    steps 0 and 505 on both electrodes of a 1 mm gap, no field, no charged
    collisions before the walls.  At every check: TP steps = PIC steps //
    tp_every; atoms launched (sputtered) = deposited at either electrode + in
    flight; and with sigma_tp = 0 (ballistic) every atom in flight sits
    exactly k sub-cycle flights v_x tp_every dt from its electrode, k the TP
    steps since its wave."""
    N, L, dt, every = 64, 1e-3, 1e-9, 10
    n = 20_000
    orc = O.Oracle(prm(L=L, ncell=N, p=0.5, sputter=1, tp_every=every, sigma_tp=sigma_tp, dt=dt,
                       V0=0.0, w=0.0, seed=17), 1, 2 * n, 2 * n)
    sp = math.sqrt(2 * 300.0 * QE / MAR)
    rng = np.random.default_rng(17)

    def wave(tag):
        xi = np.concatenate([rng.uniform(1e-3, 2e-3, n), N - rng.uniform(1e-3, 2e-3, n)])
        vx = np.concatenate([np.full(n, -sp), np.full(n, sp)])
        ids = (np.arange(2 * n, dtype=np.uint64) + np.uint64(tag)) | np.uint64(1 << 62)
        load(orc, 1, xi, [vx, np.zeros(2 * n), np.zeros(2 * n)], ids)

    dx = L / N
    wave(0)
    orc.step(505)
    m1 = orc.tp_step_index                                  # TP steps before the second wave
    wave(1 << 20)
    for chunk in (95, 400, 1000):
        orc.step(chunk)
        c = orc.counters()
        assert orc.tp_step_index == orc.step_index // every
        launched = c["sputtered_l"] + c["sputtered_r"]
        assert launched > 0.25 * 4 * n
        assert launched == c["tp_dep_l"] + c["tp_dep_r"] + c["n_tp"]
        if sigma_tp == 0.0:
            assert c["tp_coll"] == 0
            tp = orc.get_species(2)
            wall = np.where(tp["vx"] > 0, 0.0, float(N))
            k = (tp["xi"] - wall) * dx / (tp["vx"] * every * dt)
            m = orc.tp_step_index
            ok = (np.abs(k - m) < 1e-6) | (np.abs(k - (m - m1)) < 1e-6)
            assert ok.all(), k[~ok][:5]
        else:
            assert c["tp_coll"] > 0
    assert c["tp_dep_l"] + c["tp_dep_r"] > 0.2 * launched
    for side in "lr":
        assert orc.diag("sputter_e_" + side).sum() == c["tp_dep_" + side]
        assert orc.diag("sputter_ang_" + side).sum() == c["tp_dep_" + side]


def test_density_diagnostic_normalisation():
    """Uniform loading gives <n> = w N / L at every node, including the
    half-volume electrode nodes."""
    n, N, L = 400_000, 64, 0.02
    w = 1e15 * L / n
    orc = O.Oracle(prm(L=L, ncell=N, w=w, dt=1e-13), n, 1)
    orc.init_species(0, n, 0.01)
    orc.field()
    orc.step(1)
    ne = orc.diag("n_e")
    per = n / N
    assert abs(ne[1:N].mean() / 1e15 - 1) < 4 / math.sqrt(n)
    assert abs(ne[0] / 1e15 - 1) < 5 / math.sqrt(per / 2)
    assert abs(ne[N] / 1e15 - 1) < 5 / math.sqrt(per / 2)


def test_flux_diagnostic_is_density_times_drift():
    """The particle flux profile (Sec. 'Simulation Results') is the time
    average of n <v_x>: with every electron drifting at u through a
    field-free gap, Gamma = n u at every node, exactly up to the weights'
    2^-32 rounding, at every node -- the depleted upstream electrode and the
    half-volume ends included -- and for either sign of u."""
    n, N, L, dt = 100_000, 64, 0.02, 1e-11
    w = 1e15 * L / n
    rng = np.random.default_rng(31)
    for u in (2.0e5, -3.0e5):
        orc = O.Oracle(prm(L=L, ncell=N, w=w, dt=dt), n, 1)
        vt = rng.standard_normal((2, n)) * 1e5
        load(orc, 0, rng.uniform(0.0, N, n), [np.full(n, u), vt[0], vt[1]])
        for _ in range(5):
            orc.set_field(np.zeros(N + 1))
            orc.step(1)
        ne, ge = orc.diag("n_e"), orc.diag("gamma_e")
        assert (ne > 0).all()
        assert np.allclose(ge, ne * u, rtol=1e-8, atol=0)
        assert orc.counters()["imp_e_l" if u < 0 else "imp_e_r"] > 0


def test_time_averaged_vacuum_potential_closed_form():
    """Time-averaged potential (Sec. 'Simulation Results'; reading: the
    average of the states after steps 1 ... n): in an empty gap the solution
    of Eq. poisson is the vacuum profile V(t)(1 - x/L), so the average is
    (1 - x/L) V0 sum_{l=1..n} sin(l th) / n, th = 2 pi f dt, and the sine sum
    has the closed form sin(n th/2) sin((n+1) th/2) / sin(th/2)."""
    P, f, V0, N = 400, 13.56e6, 100.0, 16
    th = 2 * math.pi / P
    for n in (1, 37, 100, 400):
        orc = O.Oracle(prm(V0=V0, f=f, dt=1.0 / f / P, ncell=N, L=0.02), 1, 1)
        orc.field()
        orc.step(n)
        mean_sin = math.sin(n * th / 2) * math.sin((n + 1) * th / 2) / math.sin(th / 2) / n
        want = (1.0 - np.arange(N + 1) / N) * V0 * mean_sin
        assert np.allclose(orc.diag("phi"), want, rtol=0, atol=1e-9 * V0)


# ------------------------------------------------------------------ source waveform and external circuit
def test_two_harmonic_waveform_extremes_and_mean():
    """Sec. 'Simulation Scenario': V0 [cos(wt + phase) + cos(2wt)] with phase
    0 peaks at 2 V0 (t = 0) and bottoms at -9/8 V0 (where cos wt = -1/4),
    the asymmetry the electrical asymmetry effect rests on; both it and the
    sine have zero mean over a period, and the sine peaks at V0."""
    n, f, V0 = 40000, 13.56e6, 300.0
    for waveform, vmax, vmin in ((1, 2.0 * V0, -1.125 * V0), (0, V0, -V0)):
        orc = O.Oracle(prm(V0=V0, f=f, dt=1.0 / f / n, waveform=waveform, ncell=8), 1, 1)
        v = np.array([orc.source_voltage(l) for l in range(n)])
        assert v.max() == pytest.approx(vmax, rel=1e-12)
        assert v.min() == pytest.approx(vmin, rel=1e-7)
        assert abs(v.mean()) < 1e-9 * V0
    orc = O.Oracle(prm(V0=V0, f=f, dt=1.0 / f / n, waveform=1, phase=math.pi / 2, ncell=8), 1, 1)
    assert orc.source_voltage(0) == pytest.approx(V0, rel=1e-12)      # -sin(0) + cos(0)


def test_series_capacitor_vacuum_divider():
    """No charge in the gap: the blocking capacitor c and the vacuum gap
    eps0/L (per unit area) in series divide the source voltage, phi_0 =
    V c / (c + eps0/L), and the field is uniform, phi_0/L."""
    L, N, f = 0.02, 64, 13.56e6
    for ratio in (0.25, 1.0, 7.0):
        cb = ratio * EPS0 / L
        orc = O.Oracle(prm(L=L, ncell=N, V0=100.0, f=f, dt=1.0 / f / 400, circuit=1, cb=cb, w=1e10), 4, 4)
        orc.step_index = 37
        orc.field()
        phi0 = orc.source_voltage(37) * cb / (cb + EPS0 / L)
        fld = orc.get_field()
        assert fld["phi"][0] == pytest.approx(phi0, rel=1e-13)
        assert np.allclose(fld["E"], phi0 / L, rtol=1e-11, atol=0)
        assert np.allclose(fld["phi"], phi0 * (1.0 - np.arange(N + 1) / N), rtol=0, atol=1e-12 * abs(phi0))


def _small_discharge(**kw):
    f = 13.56e6
    p = prm(L=0.025, p=3.0, Tg=300.0, f=f, V0=100.0, w=1e15 * 0.025 / 3000, dt=1.0 / f / 400, ncell=64,
            seed=11, diag_every=10)
    p.update(kw)
    orc = O.Oracle(p, 20000, 20000, 1)
    orc.init_species(0, 3000, 2.0)
    orc.init_species(1, 3000, 0.026)
    orc.field()
    return orc


def test_infinite_blocking_capacitance_is_the_ideal_source():
    """c -> infinity shorts the capacitor: 40 steps with the circuit and
    c = inf leave exactly the state of the ideal source on the electrode."""
    a = _small_discharge(circuit=1, cb=math.inf, waveform=1)
    b = _small_discharge(circuit=0, waveform=1)
    a.step(40)
    b.step(40)
    for s in (0, 1):
        ga, gb = a.get_species(s), b.get_species(s)
        for k in ("xi", "vx", "vy", "vz", "id"):
            assert np.array_equal(ga[k], gb[k]), (s, k)
    assert np.array_equal(a.get_field()["E"], b.get_field()["E"])


def test_circuit_surface_charge_balance():
    """Gauss's law at the driven electrode, eps0 E_0 = sigma = q + w, with w
    the charge of the ions minus the electrons absorbed there: c = 0 is a
    floating electrode (q = 0, so eps0 E_0 = w); a finite c obeys the loop
    phi_0 = V - q/c.  Checked after several steps with wall losses."""
    for cb in (0.0, 3.0 * EPS0 / 0.025):
        orc = _small_discharge(circuit=1, cb=cb)
        for _ in range(3):
            orc.step(15)
            c = orc.counters()
            w = QE * orc.prm["w"] * (c["imp_i_l"] - c["imp_e_l"])
            fld = orc.get_field()
            sigma = EPS0 * fld["E"][0]
            scale = EPS0 * np.abs(fld["E"]).max() + abs(w)
            q = sigma - w
            if cb == 0.0:
                assert abs(q) <= 1e-10 * scale
            else:
                V = orc.source_voltage(orc.step_index)
                assert fld["phi"][0] == pytest.approx(V - q / cb, abs=1e-9 * max(abs(V), abs(fld["phi"][0])))
        assert c["imp_e_l"] + c["imp_i_l"] > 0


# ------------------------------------------------------------------ event-driven TP flight
def test_mean_relative_speed_against_quadrature():
    """<|v - w|> over a Maxwellian of most probable speed c, by numerical
    integration over the partner's speed and angle, against the closed form
    and its small-s series the event-driven flight uses for nu(v)."""
    from scipy import integrate
    c = 352.0
    for s in (0.0, 5e-4, 2e-3, 0.3, 1.0, 2.5, 8.0):
        v = s * c

        def inner(u):
            # angle average of |v - w| for |w| = u, in closed form over cos(theta)
            if v == 0.0:
                return u
            a, b = abs(v - u), v + u
            return (b**3 - a**3) / (6.0 * v * u) if u > 0 else v

        num, _ = integrate.quad(lambda u: inner(u) * 4 * math.pi * u * u * math.exp(-u * u / (c * c))
                                / (math.pi * c * c) ** 1.5, 0.0, 12 * c + v, limit=200, epsabs=0, epsrel=1e-12)
        assert O.mean_rel_speed(v, c) == pytest.approx(num, rel=1e-9), s


def test_flux_weighted_partner_sampler():
    """Collision partners of an atom at speed v are drawn with density
    |v - w| f(w)/<|v - w|>, so the mean relative speed over them is
    <|v - w|^2>/<|v - w|> = (v^2 + 3c^2/2)/<|v - w|>, and the proposals
    used per partner are geometric with mean (|v| + 2c/sqrt(pi))/<|v - w|>."""
    T = 300.0
    c = math.sqrt(2 * KB * T / MAR)
    for vm in (50.0, 600.0, 4000.0):
        v = np.array([0.6, -0.48, 0.64]) * vm
        n = 40_000
        g, tries = np.zeros(n), np.zeros(n)
        for e in range(n):
            w, t = O.tpf_partner(99, 7 | (2 << 62), e, T, v)
            g[e] = np.linalg.norm(v - w)
            tries[e] = t
        gbar = O.mean_rel_speed(vm, c)
        want = (vm * vm + 1.5 * c * c) / gbar
        assert abs(g.mean() - want) < 4.5 * g.std() / math.sqrt(n)
        mt = (vm + 2 * c / math.sqrt(math.pi)) / gbar
        assert abs(tries.mean() - mt) < 4.5 * tries.std() / math.sqrt(n)
        assert tries.max() <= 64


def test_event_driven_flight_without_gas_is_ballistic():
    """No gas (p = 0): every atom flies straight to the wall it heads for and
    sticks there with its launch energy; each cell crossed whole collects
    dx/|v_x| of residence time, so the cells away from the launch point all
    hold the same time, the sum over the atoms of dx/|v_x|."""
    n, N, L = 20_000, 64, 0.05
    rng = np.random.default_rng(3)
    orc = O.Oracle(prm(L=L, ncell=N, p=0.0, Tg=300.0, sigma_tp=3e-19), 1, 1, n)
    v = _mono(n, 2000.0, rng)
    xi = rng.uniform(0.2, 0.8, n) * N
    load(orc, 2, xi, v)
    assert orc.tp_flight(10) == 0
    c = orc.counters()
    right = v[0] > 0
    assert c["tp_dep_r"] == int(right.sum()) and c["tp_dep_l"] == n - int(right.sum())
    E = 0.5 * MAL * (v ** 2).sum(0) / QE
    h = np.histogram(E[right], bins=600, range=(0.0, 300.0))[0]
    assert np.array_equal(orc.diag("sputter_e_r"), h.astype(float))
    t = orc.diag("tpf_time")
    dx = L / N
    full = np.ones(N, bool)
    full[int(0.2 * N):int(0.8 * N) + 1] = False
    want_r = (dx / np.abs(v[0][right])).sum()
    want_l = (dx / np.abs(v[0][~right])).sum()
    for j in np.nonzero(full)[0]:
        want = want_r if j > 0.5 * N else want_l
        assert t[j] == pytest.approx(want, rel=1e-10), j
    path = np.where(right, N - xi, xi) * dx
    assert t.sum() == pytest.approx((path / np.abs(v[0])).sum(), rel=1e-10)


def test_event_driven_uncollided_fraction_in_cold_gas():
    """A mono-energetic beam along +x into a cold gas (relative speed = the
    atom's speed) crosses the gap without a collision with probability
    exp(-n sigma L): the atoms that stick at the far wall in their first
    event."""
    n, N, L, ngas, sig, T = 200_000, 128, 0.03, 1.2e20, 3e-19, 1e-3
    orc = O.Oracle(prm(L=L, ncell=N, p=ngas * KB * T, Tg=T, sigma_tp=sig), 1, 1, n)
    v = np.zeros((3, n))
    v[0] = 3000.0
    load(orc, 2, np.full(n, 1e-6), v)
    orc.tp_flight(1)
    P = math.exp(-ngas * sig * L)
    got = orc.counters()["tp_dep_r"]
    assert abs(got - n * P) < 4.5 * math.sqrt(n * P * (1 - P))


@pytest.mark.parametrize("tp_mode", [0, 1])
def test_event_driven_flight_agrees_with_the_per_step_test(tp_mode):
    """The two TP transport schemes of the oracle, written independently --
    the per-step collision test (orc_tp_step, dt = 5 ns, nu dt < 1e-3; with
    thinned candidates, tp_mode 0, and with the literal test, tp_mode 1) and
    the event-driven flight -- give the same energetic arrivals (> 2 eV) at
    the far electrode from a 300 eV-ion source: count within 4.5 standard
    deviations, energy distribution by a two-sample KS test."""
    n, N, L = 3000, 64, 0.02
    P = prm(L=L, ncell=N, p=0.5, Tg=300.0, sigma_tp=3e-19, seed=21, tp_mode=tp_mode)
    a = O.Oracle(P, 1, 1, n)
    b = O.Oracle(P, 1, 1, n)
    a.tp_launch(n, 300.0)
    b.tp_launch(n, 300.0)
    a.tp_step(6000, 5e-9)                        # 30 us: energetic atoms have arrived
    b.tp_flight(100_000)
    edges = np.arange(601) * 0.5
    ha, hb = a.diag("sputter_e_r"), b.diag("sputter_e_r")
    sel = edges[:-1] >= 2.0
    na, nb = ha[sel].sum(), hb[sel].sum()
    assert na > 300 and abs(na - nb) < 4.5 * math.sqrt(na + nb)
    ca, cb = np.cumsum(ha[sel]) / na, np.cumsum(hb[sel]) / nb
    D = np.abs(ca - cb).max()
    pval = stats.kstwobign.sf(D * math.sqrt(na * nb / (na + nb)))
    assert pval > 1e-3, (pval, na, nb)
    assert b.counters()["tp_dep_l"] + b.counters()["tp_dep_r"] == n


# ------------------------------------------------------------------ hypothesis checks
def test_width_to_peak_and_rms_angle_closed_forms():
    """Sec. 'Hypotheses validation' measures: the full width at half maximum
    of a sampled Gaussian peak is 2 sqrt(2 ln 2) sigma to a bin; a box of W
    bins starting at bin b0 has width W bins over a peak at bin b0 (its
    first fullest bin); the rms angle of a one-bin histogram is the bin
    centre, and of a flat one over [0, 90) deg it is sqrt(sum (b + 1/2)^2 / 90)."""
    nb, emax = 512, 600.0
    bw = emax / nb
    c = (np.arange(nb) + 0.5) * bw
    for E0, sig in ((300.0, 12.0), (80.0, 3.0)):
        h = np.exp(-0.5 * ((c - E0) / sig) ** 2) * 1e6
        r = O.width_to_peak(h, emax)
        pk = (np.argmax(h) + 0.5) * bw
        assert abs(r * pk - 2 * math.sqrt(2 * math.log(2)) * sig) <= 1.01 * bw
    h = np.zeros(nb)
    h[100:117] = 5.0
    assert O.width_to_peak(h, emax) == pytest.approx(17 / 100.5, rel=1e-15)
    one = np.zeros(90)
    one[3] = 7
    assert O.rms_angle(one) == pytest.approx(3.5, rel=1e-15)
    flat = np.ones(90)
    assert O.rms_angle(flat) == pytest.approx(math.sqrt(sum((b + 0.5) ** 2 for b in range(90)) / 90), rel=1e-14)
    assert O.width_to_peak(np.zeros(nb), emax) == 0.0 and O.rms_angle(np.zeros(90)) == 0.0


def test_hypotheses_read_the_run_diagnostics():
    """orc_hypotheses combines the run's diagnostics as defined: the ion
    energy distributions' width-to-peak, the energy-summed IEADF's rms
    angle, and the largest averaged n_i and TP density over the gas density."""
    orc = _small_discharge(sputter=1, V0=300.0, tp_every=10)
    orc.step(400)
    h = orc.hypotheses()
    for el, side in ((0, "l"), (1, "r")):
        assert h[el] == pytest.approx(O.width_to_peak(orc.diag("iedf_" + side), 600.0), rel=1e-15)
        ang = orc.diag("ieadf_" + side).reshape(128, 90).sum(0)
        assert h[2 + el] == pytest.approx(O.rms_angle(ang), rel=1e-15)
    ngas = orc.derived()["n_gas"]
    assert h[4] == pytest.approx(orc.diag("n_i").max() / ngas, rel=1e-15)
    assert h[5] == pytest.approx(orc.diag("tp_dens").max() / ngas, rel=1e-15)
    assert 0.0 < h[4] < 1e-3


# ------------------------------------------------------------------ VHS / M1 test-particle collisions
def test_vhs_reference_diameter_of_argon():
    """Eq. referencediameter turns argon's tabulated viscosity into its
    tabulated VHS diameter (tests/golden/vhs_argon_bird1994.txt)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "vhs_argon_bird1994.txt"))
            if l.strip() and not l.startswith("#")]
    mu, T, om, m, d, tol = map(float, rows[0])
    assert abs(O.vhs_dref(mu, T, om, m * AMU) / d - 1.0) < tol


def test_vhs_cross_section_law():
    """Eq. maximumimpactparameter: sigma = pi b_max^2 falls as g^(1 - 2 omega);
    omega = 1/2 is the hard sphere of diameter d_ref (Gamma(2) = 1); M1 takes
    d_ref sqrt(4/3), so 4/3 of the VHS cross section."""
    d = 4.17e-10
    vhs = O.Oracle(prm(tp_model=1, dref=d, omega=0.81, tref=273.0), 1, 1, 1)
    m1 = O.Oracle(prm(tp_model=2, dref=d, omega=0.81, tref=273.0), 1, 1, 1)
    hs = O.Oracle(prm(tp_model=1, dref=d, omega=0.5, tref=273.0), 1, 1, 1)
    for g in (50.0, 700.0, 5000.0):
        assert vhs.tp_sigma(2 * g) / vhs.tp_sigma(g) == pytest.approx(2 ** (1 - 2 * 0.81), rel=1e-12)
        assert m1.tp_sigma(g) == pytest.approx(4.0 / 3.0 * vhs.tp_sigma(g), rel=1e-12)
        assert hs.tp_sigma(g) == pytest.approx(math.pi * d * d, rel=1e-14)
    mr = MAL * MAR / (MAL + MAR)
    g = 1234.0
    bmax2 = d * d * (2 * KB * 273.0 / (mr * g * g)) ** (0.81 - 0.5) / special.gamma(2.5 - 0.81)
    assert vhs.tp_sigma(g) == pytest.approx(math.pi * bmax2, rel=1e-12)


def test_scattering_angle_laws():
    """Sec. 'Binary Interactions': VHS scatters isotropically (cos chi
    uniform on [-1, 1]); M1 deflects by chi = pi (1 - b/b_max) with b =
    b_max sqrt(R), so P(chi <= x) = 1 - (1 - x/pi)^2; both keep |g|."""
    rng = np.random.default_rng(8)
    g = np.array([-0.3, 0.8, 0.52])
    gh = g / np.linalg.norm(g)
    n = 20000
    words = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64)
    for model, cdf in ((1, lambda x: (1 - np.cos(x)) / 2), (2, lambda x: 1 - (1 - x / np.pi) ** 2)):
        chi = np.empty(n)
        for i in range(n):
            dvec = O.tp_scatter(model, g, int(words[i, 0]), int(words[i, 1]))
            assert abs(np.linalg.norm(dvec) - 1.0) < 1e-12
            chi[i] = math.acos(max(-1.0, min(1.0, float(dvec @ gh))))
        assert stats.kstest(chi, cdf).pvalue > 1e-3, model


def test_vhs_uncollided_fraction_in_cold_gas():
    """A mono-energetic beam into a cold gas under the VHS law: the flight
    with candidates at a majorant rate and null events keeps the atoms that
    never collide at probability exp(-n sigma(v0) L); they reach the far
    electrode along the normal (the first angle bin; an isotropic deflection
    lands there with probability 8e-5)."""
    n, N, L, ngas, T = 100_000, 128, 0.03, 1.2e20, 1e-3
    v0 = 2400.0
    orc = O.Oracle(prm(L=L, ncell=N, p=ngas * KB * T, Tg=T, tp_model=1, dref=4.17e-10, omega=0.81, tref=273.0),
                   1, 1, n)
    v = np.zeros((3, n))
    v[0] = v0
    load(orc, 2, np.full(n, 1e-6), v)
    assert orc.tp_flight(100_000) == 0
    got = orc.diag("sputter_ang_r")[0]            # still along the normal: never scattered
    P = math.exp(-ngas * orc.tp_sigma(v0) * L)
    assert abs(got - n * P) < 4.5 * math.sqrt(n * P * (1 - P))


@pytest.mark.parametrize("tp_mode", [0, 1])
@pytest.mark.parametrize("model", [1, 2])
def test_vhs_and_m1_flights_agree_with_the_per_step_test(model, tp_mode):
    """Under the VHS and M1 laws the event-driven flight (majorant rate, null
    events, gamma-distributed partner speeds) and the per-step test (both
    modes) give the same energetic arrivals at the far electrode from a
    300 eV-ion source."""
    n, N, L = 3000, 64, 0.02
    P = prm(L=L, ncell=N, p=0.5, Tg=300.0, seed=23, tp_model=model, dref=4.17e-10, omega=0.81, tref=273.0,
            tp_mode=tp_mode)
    a = O.Oracle(P, 1, 1, n)
    b = O.Oracle(P, 1, 1, n)
    a.tp_launch(n, 300.0)
    b.tp_launch(n, 300.0)
    a.tp_step(6000, 5e-9)
    b.tp_flight(100_000)
    edges = np.arange(601) * 0.5
    ha, hb = a.diag("sputter_e_r"), b.diag("sputter_e_r")
    sel = edges[:-1] >= 2.0
    na, nb = ha[sel].sum(), hb[sel].sum()
    assert na > 300 and abs(na - nb) < 4.5 * math.sqrt(na + nb)
    D = np.abs(np.cumsum(ha[sel]) / na - np.cumsum(hb[sel]) / nb).max()
    assert stats.kstwobign.sf(D * math.sqrt(na * nb / (na + nb))) > 1e-3
    assert b.counters()["tp_dep_l"] + b.counters()["tp_dep_r"] == n


# ------------------------------------------------------------------ tabulated electron cross sections
def test_cross_section_table_interpolation_against_numpy():
    """Linear interpolation of an LXcat-style table (constant beyond the
    ends) against numpy.interp on random tables and energies, including the
    table points themselves and energies outside it."""
    rng = np.random.default_rng(12)
    for n in (2, 7, 300):
        E = np.sort(rng.uniform(0.0, 200.0, n))
        E = np.unique(E)
        sg = rng.uniform(0.0, 1e-19, E.size)
        eps = np.concatenate([rng.uniform(-10.0, 250.0, 400), E])
        got = np.array([O.xs_interp(E, sg, e) for e in eps])
        assert np.allclose(got, np.interp(eps, E, sg), rtol=1e-14, atol=0.0)


def test_constant_cross_section_table_gives_the_collision_rate():
    """A table holding a constant elastic cross section (excitation and
    ionisation tables zero): nu_max is n sigma v(eps_max), and electrons at
    speed v collide per step with probability (1 - exp(-nu_max dt)) n sigma
    v / nu_max."""
    N, dt, n, p = 64, 2e-11, 200_000, 3.0
    orc = O.Oracle(prm(L=1.0, ncell=N, p=p, Tg=300.0, dt=dt, V0=50.0), n + 10, 10)
    E = np.array([0.0, 1000.0])
    orc.set_cross_section(0, E, [2.5e-19, 2.5e-19])
    orc.set_cross_section(1, E, [0.0, 0.0])
    orc.set_cross_section(2, E, [0.0, 0.0])
    ngas = p / (KB * 300.0)
    eps_max = 2 * 50.0 + 100.0
    assert orc.derived()["nu_max_e"] == pytest.approx(ngas * 2.5e-19 * math.sqrt(2 * eps_max * QE / ME), rel=1e-14)
    v = math.sqrt(2 * 10.0 * QE / ME)
    rng = np.random.default_rng(5)
    load(orc, 0, rng.uniform(10, 50, n), _mono(n, v, rng))
    orc.set_field(np.zeros(N + 1))
    orc.step(1)
    num = orc.derived()["nu_max_e"]
    pexp = (1.0 - math.exp(-num * dt)) * ngas * 2.5e-19 * v / num   # candidate, then elastic
    got = orc.counters()["elastic"]
    assert abs(got - n * pexp) < 4.5 * math.sqrt(n * pexp)
    assert orc.counters()["excitation"] == 0 and orc.counters()["ionizations"] == 0
