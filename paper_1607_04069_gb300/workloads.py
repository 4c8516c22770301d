"""Workload definitions and seeded synthetic inputs.

This module holds parameter sets and numpy random generators only -- no step
of the method.  It is the one module that both the CUDA path's tests/bench
and the oracle's tests draw their inputs from.

Workloads (shaped like the paper's capacitive argon sputtering discharge,
Sec. "Simulation Scenario", with the sizes of the benchmark configurations):

* ``ccp_small``   -- 25 mm gap, 128 cells, 13.56 MHz 100 V sine, 3 Pa,
  300 K, 20k e- + 20k Ar+, dt = T_RF/400, 64-bit positions, no sputtering.
* ``ccp_sputter`` -- 50 mm gap, 1024 cells, 300 V, 0.5 Pa, dt = T_RF/3000,
  2M e- + 2M Ar+, 32-bit positions, sputtering on, TP sub-cycled x40.
* ``tp_transport`` -- 100M Al atoms from a 300 eV mono-energetic Ar+ source,
  50 mm gap, hard spheres (3e-19 m^2) in 0.5 Pa / 300 K Ar, dt_tp = 1 ns.
* ``batched``     -- many independent discharges of uneven size stepped
  together, and ``poisson_arrivals`` for a stream of such requests.
"""
from __future__ import annotations

import math

import numpy as np

F_RF = 13.56e6
T_RF = 1.0 / F_RF


def ccp_small(n_per_species: int = 20_000, seed: int = 1235) -> dict:
    n0 = 1e15
    L = 0.025
    return dict(name="ccp_small: 25mm/128 cells/100V/3Pa, 20k+20k, dt=T_RF/400, fp64 x",
                gap_m=L, pressure_pa=3.0, gas_temp_k=300.0, rf_freq_hz=F_RF, rf_volt_v=100.0,
                n_cells=128, weight=n0 * L / n_per_species, dt=T_RF / 400,
                n_e0=n_per_species, n_i0=n_per_species, te0_ev=2.0, ti0_ev=0.026, seed=seed,
                pos_precision=64, sputter_enable=0, tp_every=0, tp_dt=1e-9,
                sigma_tp=3e-19, diag_every=10, steps_per_period=400, periods=20)


def ccp_sputter(n_per_species: int = 2_000_000, seed: int = 1236, n_cells: int = 1024) -> dict:
    n0 = 4e15
    L = 0.05
    return dict(name="ccp_sputter: 50mm/1024 cells/300V/0.5Pa, 2M+2M, dt=T_RF/3000, u32 x",
                gap_m=L, pressure_pa=0.5, gas_temp_k=300.0, rf_freq_hz=F_RF, rf_volt_v=300.0,
                n_cells=n_cells, weight=n0 * L / n_per_species, dt=T_RF / 3000,
                n_e0=n_per_species, n_i0=n_per_species, te0_ev=2.0, ti0_ev=0.026, seed=seed,
                pos_precision=32, sputter_enable=1, tp_every=40, tp_dt=40 * T_RF / 3000,
                sigma_tp=3e-19, diag_every=10, steps_per_period=3000, periods=10)


def tp_transport(n_atoms: int = 100_000_000, seed: int = 1237) -> dict:
    return dict(name="tp_transport: 100M Al atoms, 50mm/1024 cells, 0.5Pa 300K Ar, dt=1ns",
                gap_m=0.05, pressure_pa=0.5, gas_temp_k=300.0, rf_freq_hz=F_RF, rf_volt_v=300.0,
                n_cells=1024, weight=1.0, dt=T_RF / 3000, n_e0=0, n_i0=0, te0_ev=2.0,
                ti0_ev=0.026, seed=seed, pos_precision=32, sputter_enable=0, tp_every=0,
                tp_dt=1e-9, sigma_tp=3e-19, diag_every=10, n_atoms=n_atoms, e_ion_ev=300.0)


def batched(n_discharges: int = 256, seed: int = 1238, n_min: int = 50_000, n_max: int = 2_000_000,
            steps_per_period: int = 3000) -> list[dict]:
    """Independent discharges of uneven size for one batched launch: cell
    counts 256-2048 (powers of two), 50k-2M superparticles per species
    (log-uniform), 0.3-5 Pa (log-uniform), 50-500 V, gap 25-50 mm, all at
    13.56 MHz with one dt = T_RF / steps_per_period, 32-bit positions, no
    sputtering.  Density 2e15 m^-3 at load (dx < lambda_D = 0.235 mm at
    2 eV, w_p dt = 0.06); member k has seed 10^6 + k."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_discharges):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        n_cells = int(2 ** rng.integers(8, 12))
        L = float(rng.uniform(0.025, 0.05))
        p = float(math.exp(rng.uniform(math.log(0.3), math.log(5.0))))
        V = float(rng.uniform(50.0, 500.0))
        out.append(dict(name=f"member {k}: {L * 1e3:.1f} mm/{n_cells} cells/{V:.0f} V/{p:.2f} Pa, {n}+{n}",
                        gap_m=L, pressure_pa=p, gas_temp_k=300.0, rf_freq_hz=F_RF, rf_volt_v=V,
                        n_cells=n_cells, weight=2e15 * L / n, dt=T_RF / steps_per_period, n_e0=n, n_i0=n,
                        te0_ev=2.0, ti0_ev=0.026, seed=10**6 + k, pos_precision=32, sputter_enable=0,
                        tp_every=0, tp_dt=1e-9, sigma_tp=3e-19, diag_every=10, sort_every_e=400,
                        sort_every_i=400, steps_per_period=steps_per_period))
    return out


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson stream of the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def oracle_params(cfg: dict) -> dict:
    """Map a workload dict onto the oracle's parameter names."""
    return dict(L=cfg["gap_m"], p=cfg["pressure_pa"], Tg=cfg["gas_temp_k"], f=cfg["rf_freq_hz"],
                V0=cfg["rf_volt_v"], w=cfg["weight"], dt=cfg["dt"], te0=cfg["te0_ev"],
                ti0=cfg["ti0_ev"], tp_dt=cfg["tp_dt"], sigma_tp=cfg["sigma_tp"], seed=cfg["seed"],
                ncell=cfg["n_cells"], sputter=cfg["sputter_enable"], tp_every=cfg["tp_every"],
                diag_every=cfg["diag_every"], waveform=cfg.get("waveform", 0), circuit=cfg.get("circuit", 0),
                phase=cfg.get("rf_phase", 0.0), cb=cfg.get("c_block", math.inf),
                dref=cfg.get("tp_dref", 0.0), omega=cfg.get("tp_omega", 0.5), tref=cfg.get("tp_tref", 273.0),
                tp_model=cfg.get("tp_model", 0), coll_mode=cfg.get("coll_mode", 0),
                tp_mode=cfg.get("tp_mode", 0))


# ------------------------------------------------------------- particle sets
TAG = {0: 0, 1: 1 << 62, 2: 2 << 62}


def fixed_positions(rng: np.random.Generator, n: int) -> np.ndarray:
    """32-bit fixed-point positions over the gap, never 0 (0 marks a removed slot)."""
    return rng.integers(1, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


def random_particles(n: int, n_cells: int, species: int, v_scale: float, seed: int,
                     pos_precision: int = 32) -> dict:
    """Uniform positions and Gaussian velocities of scale ``v_scale`` (m/s),
    float32 velocities, sequential tagged ids.  Positions are returned both
    in the storage form of the requested precision and in cell units
    (float64, exact for the fixed-point form)."""
    rng = np.random.default_rng(seed)
    if pos_precision == 32:
        pos = fixed_positions(rng, n)
        xi = pos.astype(np.float64) * (n_cells / 2.0**32)
    else:
        xi = rng.uniform(0.0, n_cells, size=n)
        xi = np.where(xi <= 0.0, 0.5, xi)
        pos = xi.copy()
    v = (rng.standard_normal((3, n)) * v_scale).astype(np.float32)
    ids = (np.arange(n, dtype=np.uint64) | np.uint64(TAG[species]))
    return dict(pos=pos, xi=xi, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=ids)


def thermal_speed(T_eV: float, mass_kg: float) -> float:
    """sqrt(kT/m) for a temperature given in eV -- an input scale, not a step."""
    return math.sqrt(T_eV * 1.602176634e-19 / mass_kg)
