"""FP64 CPU oracle of the 1d3v PIC/MCC cycle and of test-particle transport.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``.  The product path
(``paper_1607_04069_gb300``) never imports this package, and this package
never imports the product path.  The C source ``pic_oracle.c`` is the
definition; this module only compiles it with gcc and marshals numpy arrays.

Paper: Trieschmann, Schmidt & Mussenbrock, arXiv:1607.04069, Sec. "Kinetic
Particle Simulation", "Particle-In-Cell Scheme" and "Test Particle Method".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# counter slots of orc_counters (same order as the enum in pic_oracle.c)
COUNTERS = ["n_e", "n_i", "n_tp", "imp_e_l", "imp_e_r", "imp_i_l", "imp_i_r", "ionizations",
            "sputtered_l", "sputtered_r", "tp_dep_l", "tp_dep_r", "numerics", "elastic",
            "excitation", "cx", "iso", "tp_coll", "capacity"]

DIAG = {"phi": 0, "n_e": 1, "n_i": 2, "gamma_e": 3, "gamma_i": 4, "eedf": 5, "iedf_l": 6,
        "iedf_r": 7, "ieadf_l": 8, "ieadf_r": 9, "sputter_e_l": 10, "sputter_e_r": 11,
        "sputter_ang_l": 12, "sputter_ang_r": 13, "tp_dens": 14, "tp_vx": 15, "tpf_time": 16,
        "tpf_vx": 17}

E, I, TP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, -O2,
    no FMA contraction so every product and sum rounds as written)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Mirror of ``orc_params`` in pic_oracle.c."""
    _fields_ = [("L", C.c_double), ("p", C.c_double), ("Tg", C.c_double), ("f", C.c_double),
                ("V0", C.c_double), ("w", C.c_double), ("dt", C.c_double),
                ("te0", C.c_double), ("ti0", C.c_double), ("tp_dt", C.c_double),
                ("sigma_tp", C.c_double), ("seed", C.c_uint64), ("ncell", C.c_int32),
                ("sputter", C.c_int32), ("tp_every", C.c_int32), ("diag_every", C.c_int32),
                ("waveform", C.c_int32), ("circuit", C.c_int32), ("phase", C.c_double), ("cb", C.c_double),
                ("dref", C.c_double), ("omega", C.c_double), ("tref", C.c_double), ("tp_model", C.c_int32),
                ("coll_mode", C.c_int32), ("tp_mode", C.c_int32), ("pad2", C.c_int32)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, u32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_double
            sig = {
                "orc_philox": (None, [vp, vp, vp]),
                "orc_sigma_e": (None, [dbl, vp]),
                "orc_sigma_i": (dbl, [dbl]),
                "orc_yield": (dbl, [dbl]),
                "orc_emit": (None, [dbl, dbl, dbl, dbl, dbl, vp]),
                "orc_deposit": (None, [vp, i64, i32, vp]),
                "orc_poisson": (None, [i32, dbl, dbl, vp, vp, dbl, vp, vp]),
                "orc_create": (vp, [C.POINTER(Params), i64, i64, i64]),
                "orc_destroy": (None, [vp]),
                "orc_derived": (None, [vp, vp]),
                "orc_init_species": (None, [vp, C.c_int, i64, dbl]),
                "orc_init_species_range": (None, [vp, C.c_int, i64, i64, dbl]),
                "orc_step_particles": (None, [vp]),
                "orc_step_field": (None, [vp]),
                "orc_set_deposit": (None, [vp, vp, vp]),
                "orc_solve": (None, [vp]),
                "orc_tp_launch_ids": (None, [vp, i64, dbl, i64]),
                "orc_set_species": (C.c_int, [vp, C.c_int, i64, vp, vp, vp, vp, vp]),
                "orc_get_species": (i64, [vp, C.c_int, i64, vp, vp, vp, vp, vp]),
                "orc_field": (None, [vp]),
                "orc_get_field": (None, [vp, vp, vp, vp, vp]),
                "orc_set_field": (None, [vp, vp]),
                "orc_counters": (None, [vp, vp]),
                "orc_step": (None, [vp, i64]),
                "orc_tp_step": (None, [vp, i64, dbl]),
                "orc_tp_launch": (None, [vp, i64, dbl]),
                "orc_diag": (i64, [vp, C.c_int, vp, i64]),
                "orc_reset_averages": (None, [vp]),
                "orc_get_step": (u32, [vp]),
                "orc_set_step": (None, [vp, u32]),
                "orc_get_tp_step": (u32, [vp]),
                "orc_gap": (u32, [dbl, u32]),
                "orc_tp_gap": (u32, [dbl, u32]),
                "orc_source_voltage": (dbl, [vp, u32]),
                "orc_mean_rel_speed": (dbl, [dbl, dbl]),
                "orc_tpf_partner": (C.c_int, [C.c_uint64, C.c_uint64, u32, dbl, vp, vp]),
                "orc_tp_flight": (i64, [vp, i64]),
                "orc_width_to_peak": (dbl, [vp, C.c_int, dbl]),
                "orc_tp_sigma": (dbl, [vp, dbl]),
                "orc_xs_interp": (dbl, [vp, vp, i64, dbl]),
                "orc_set_cross_section": (C.c_int, [vp, C.c_int, i64, vp, vp]),
                "orc_vhs_dref": (dbl, [dbl, dbl, dbl, dbl]),
                "orc_tp_scatter": (None, [C.c_int, vp, u32, u32, vp]),
                "orc_rms_angle": (dbl, [vp, C.c_int]),
                "orc_hypotheses": (None, [vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def gap(lam, w):
    """Steps from one null-collision candidate to the next for nu_max dt =
    lam, from the Philox word w (geometric law, see orc_gap)."""
    return int(lib().orc_gap(float(lam), int(w) & 0xffffffff))


def tp_gap(Ph, w):
    """TP steps from one collision candidate to the next at the per-step
    candidate probability Ph, from the Philox word w (geometric law)."""
    return int(lib().orc_tp_gap(float(Ph), int(w) & 0xffffffff))


def mean_rel_speed(v, c):
    """<|v - w|> of a particle of speed v in a Maxwellian gas of most probable speed c."""
    return float(lib().orc_mean_rel_speed(float(v), float(c)))


def tpf_partner(seed, atom_id, e, Tg, v):
    """Collision partner of event e of an atom with velocity v (flux-weighted
    Maxwellian sample); returns (w, proposals used)."""
    vv = np.ascontiguousarray(v, dtype=np.float64)
    w = np.zeros(3)
    t = lib().orc_tpf_partner(int(seed), int(atom_id), int(e), float(Tg), _p(vv), _p(w))
    return w, int(t)


def xs_interp(E, sigma, eps):
    """Tabulated cross section at eps: linear between points, constant outside."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    return float(lib().orc_xs_interp(_p(E), _p(sg), E.size, float(eps)))


def vhs_dref(mu_ref, t_ref, omega, mass):
    """VHS reference diameter from the viscosity at T_ref (Eq. referencediameter)."""
    return float(lib().orc_vhs_dref(float(mu_ref), float(t_ref), float(omega), float(mass)))


def tp_scatter(model, g, r1, r2):
    """Unit direction of the post-collision relative velocity (0/1 isotropic, 2 M1)."""
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_tp_scatter(int(model), _p(gg), int(r1) & 0xffffffff, int(r2) & 0xffffffff, _p(out))
    return out


def width_to_peak(h, emax):
    """Full width at half maximum over the peak energy of a histogram on [0, emax]."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    return float(lib().orc_width_to_peak(_p(h), h.size, float(emax)))


def rms_angle(h):
    """Root mean square angle (deg) of a 1-degree angle histogram."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    return float(lib().orc_rms_angle(_p(h), h.size))


def sigma_e(eps):
    out = np.zeros(3)
    lib().orc_sigma_e(float(eps), _p(out))
    return out


def sigma_i(eps):
    return lib().orc_sigma_i(float(eps))


def sputter_yield(E):
    return lib().orc_yield(float(E))


def emit(uE, uT, uP, Emax, direction=1.0):
    out = np.zeros(3)
    lib().orc_emit(float(uE), float(uT), float(uP), float(Emax), float(direction), _p(out))
    return out


def deposit(xi, ncell):
    """CIC deposit of positions given in cell units; int64[ncell+1] result."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    q = np.zeros(ncell + 1, dtype=np.int64)
    lib().orc_deposit(_p(xi), xi.size, int(ncell), _p(q))
    return q


def poisson(ncell, dx, w, q_i, q_e, v_left):
    q_i = np.ascontiguousarray(q_i, dtype=np.int64)
    q_e = np.ascontiguousarray(q_e, dtype=np.int64)
    phi = np.zeros(ncell + 1)
    E = np.zeros(ncell + 1)
    lib().orc_poisson(int(ncell), float(dx), float(w), _p(q_i), _p(q_e), float(v_left),
                      _p(phi), _p(E))
    return phi, E


# ---------------------------------------------------------------- simulation
class Oracle:
    """One discharge in the oracle.  ``prm`` is a dict with the keys of
    :class:`Params` (SI units, temperatures of the initial loading in eV)."""

    def __init__(self, prm: dict, cap_e: int, cap_i: int, cap_tp: int = 0):
        self.prm = dict(prm)
        P = Params()
        for name, _ in Params._fields_:
            setattr(P, name, prm.get(name, 0))
        self._P = P
        self.ncell = int(prm["ncell"])
        self.h = lib().orc_create(C.byref(P), int(cap_e), int(cap_i), int(cap_tp))
        self.cap = [int(cap_e), int(cap_i), int(cap_tp)]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def derived(self):
        out = np.zeros(8)
        lib().orc_derived(self.h, _p(out))
        keys = ["n_gas", "dx", "nu_max_e", "nu_max_i", "p_max_e", "p_max_i", "eps_max", "lambda"]
        return dict(zip(keys, out.tolist()))

    def init_species(self, s, n, T_eV, first=0):
        """The initial loading of particles first .. first + n - 1 (ids tag | k)."""
        lib().orc_init_species_range(self.h, int(s), int(first), int(n), float(T_eV))

    def step_particles(self):
        """First half of a cycle: push, walls, collisions, charge assignment of the own particles."""
        lib().orc_step_particles(self.h)

    def step_field(self):
        """Second half: field solve from the deposit, time averages, coupled TP step."""
        lib().orc_step_field(self.h)

    def solve(self):
        """Field solve of the current step from the deposit held."""
        lib().orc_solve(self.h)

    def set_deposit(self, q_e, q_i):
        """Replace the deposit the next field solve uses (int64[ncell+1] each)."""
        a = np.ascontiguousarray(q_e, dtype=np.int64)
        b = np.ascontiguousarray(q_i, dtype=np.int64)
        lib().orc_set_deposit(self.h, _p(a), _p(b))

    def set_species(self, s, xi, vx, vy, vz, ids):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xi, vx, vy, vz)]
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        rc = lib().orc_set_species(self.h, int(s), ids.size, *[_p(a) for a in arrs], _p(ids))
        if rc != 0:
            raise ValueError("capacity exceeded")

    def get_species(self, s):
        cap = self.cap[s]
        out = [np.zeros(cap) for _ in range(4)]
        ids = np.zeros(cap, dtype=np.uint64)
        n = lib().orc_get_species(self.h, int(s), cap, *[_p(a) for a in out], _p(ids))
        return {"xi": out[0][:n], "vx": out[1][:n], "vy": out[2][:n], "vz": out[3][:n],
                "id": ids[:n]}

    def field(self):
        lib().orc_field(self.h)

    def get_field(self):
        n = self.ncell + 1
        E, phi = np.zeros(n), np.zeros(n)
        qe, qi = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
        lib().orc_get_field(self.h, _p(E), _p(phi), _p(qe), _p(qi))
        return {"E": E, "phi": phi, "q_e": qe, "q_i": qi}

    def set_field(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        lib().orc_set_field(self.h, _p(E))

    def counters(self):
        out = np.zeros(len(COUNTERS), dtype=np.int64)
        lib().orc_counters(self.h, _p(out))
        return dict(zip(COUNTERS, out.tolist()))

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def tp_step(self, n, dt_tp):
        lib().orc_tp_step(self.h, int(n), float(dt_tp))

    def tp_launch(self, n, E_ion, first_id=None):
        """Atoms of a mono-energetic source; first_id: ids first_id .. first_id + n - 1
        (default: after the atoms launched before)."""
        if first_id is None:
            lib().orc_tp_launch(self.h, int(n), float(E_ion))
        else:
            lib().orc_tp_launch_ids(self.h, int(n), float(E_ion), int(first_id))

    def tp_flight(self, max_events):
        """Event-driven flight of every live TP atom, at most max_events
        events each; returns the atoms still alive."""
        return int(lib().orc_tp_flight(self.h, int(max_events)))

    def diag(self, kind):
        k = DIAG[kind] if isinstance(kind, str) else int(kind)
        cap = 128 * 90 + 16
        out = np.zeros(max(cap, self.ncell + 1))
        n = lib().orc_diag(self.h, k, _p(out), out.size)
        return out[:n].copy()

    def reset_averages(self):
        lib().orc_reset_averages(self.h)

    def set_cross_section(self, process, E, sigma):
        """Tabulate e-Ar process 0/1/2 (elastic, excitation, ionisation); E in eV,
        sigma in m^2; empty arrays restore the analytic form."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        if lib().orc_set_cross_section(self.h, int(process), E.size, _p(E), _p(sg)) != 0:
            raise ValueError("bad cross-section table")

    def tp_sigma(self, g):
        """TP collision cross section at relative speed g (m^2)."""
        return float(lib().orc_tp_sigma(self.h, float(g)))

    def hypotheses(self):
        """dE/E_max left/right, rms impact angle left/right (deg), max n_Ar+/n_Ar, max n_Al/n_Ar."""
        out = np.zeros(6)
        lib().orc_hypotheses(self.h, _p(out))
        return out

    def source_voltage(self, l):
        """Source voltage at step l (before any series capacitor)."""
        return float(lib().orc_source_voltage(self.h, int(l)))

    @property
    def step_index(self):
        return int(lib().orc_get_step(self.h))

    @step_index.setter
    def step_index(self, l):
        lib().orc_set_step(self.h, int(l))

    @property
    def tp_step_index(self):
        return int(lib().orc_get_tp_step(self.h))
