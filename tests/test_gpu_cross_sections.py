"""Tabulated e-Ar cross sections (pic_set_cross_section) against the
oracle's tables: the same nu_max, and one MCC step from identical Philox
words with the same collisions and post-collision states (tolerances of the
analytic collision test in test_gpu_parity.py)."""
import math

import numpy as np
import pytest

from paper_1607_04069_gb300 import workloads as W

from helpers import gpu_discharge, match, oracle_for

pytestmark = pytest.mark.gpu

QE, ME = 1.602176634e-19, 9.1093837015e-31

# LXcat-like shapes: an elastic cross section with a minimum near 0.3 eV, and
# excitation and ionisation tables that start at their thresholds
TABLES = {
    0: ([0.0, 0.1, 0.3, 0.6, 1.0, 3.0, 10.0, 15.0, 30.0, 100.0, 1000.0],
        [7e-20, 1.5e-20, 2e-21, 6e-21, 1.4e-20, 5e-20, 1.5e-19, 1.4e-19, 8e-20, 3e-20, 5e-21]),
    1: ([11.5, 12.0, 15.0, 20.0, 30.0, 60.0, 1000.0], [0.0, 2e-22, 4e-21, 8e-21, 1e-20, 7e-21, 1e-21]),
    2: ([15.8, 17.0, 20.0, 30.0, 50.0, 100.0, 1000.0], [0.0, 2e-21, 6e-21, 1.8e-20, 2.8e-20, 3e-20, 1.2e-20]),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield


def test_tables_give_the_oracles_collisions():
    ncell = 256
    cfg = W.ccp_small(n_per_species=1000)
    cfg.update(n_cells=ncell, pressure_pa=3.0, rf_volt_v=100.0, pos_precision=32, sort_every_e=0,
               sort_every_i=0, n_e0=0, n_i0=0, cap_e=400_000, cap_i=400_000, gap_m=1.0, dt=1e-10)
    d = gpu_discharge(cfg)
    orc = oracle_for(cfg, cap=400_000)
    nu0 = d.derived()["nu_max_e"]
    e = W.random_particles(100_000, ncell, 0, math.sqrt(20 * QE / ME), 5, 32)
    d.set_species(0, e["pos"], e["vx"], e["vy"], e["vz"], e["id"])
    orc.set_species(0, e["xi"], e["vx"].astype(np.float64), e["vy"].astype(np.float64),
                    e["vz"].astype(np.float64), e["id"])
    for q, (E, s) in TABLES.items():
        d.set_cross_section(q, E, s)
        orc.set_cross_section(q, E, s)
    assert d.derived()["nu_max_e"] == pytest.approx(orc.derived()["nu_max_e"], rel=1e-12)
    E0 = np.zeros(ncell + 1)
    d.set_field(E0)
    orc.set_field(E0)
    d.step(1)
    d.sync()
    orc.step(1)
    c, oc = d.counters(), orc.counters()
    for k in ("elastic", "excitation", "ionizations"):
        assert c[k] == oc[k], (k, c[k], oc[k])
    assert c["elastic"] > 500 and c["excitation"] > 20 and c["ionizations"] > 5
    for s in (0, 1):
        g, o, only_g, only_o = match(d.get_species(s), orc.get_species(s))
        assert len(only_g) == 0 and len(only_o) == 0
        vg = np.stack([g["vx"], g["vy"], g["vz"]]).astype(np.float64)
        vo = np.stack([o["vx"], o["vy"], o["vz"]])
        ng, no = np.linalg.norm(vg, axis=0), np.linalg.norm(vo, axis=0)
        # energies (a threshold subtraction cancels, so not speeds), FP32 rounding of the pre-collision one
        m = ME if s == 0 else 39.948 * 1.66053906660e-27
        Eg, Eo = 0.5 * m * ng**2 / QE, 0.5 * m * no**2 / QE
        assert (np.abs(Eg - Eo) <= 2e-6 * (2 * Eo + 40.0)).all()
        ok = no > 0
        assert (np.linalg.norm(vg[:, ok] / ng[ok] - vo[:, ok] / no[ok], axis=0) <= 1e-5).all()
    for q in TABLES:                              # back to the analytic form
        d.set_cross_section(q, [], [])
    assert d.derived()["nu_max_e"] == pytest.approx(nu0, rel=1e-15)
    d.close()
