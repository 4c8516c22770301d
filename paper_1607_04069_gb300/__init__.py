"""GB300 engine for the PIC/MCC + test-particle hot path of arXiv:1607.04069.

A thin ctypes binding of the C ABI in ``include/pic_gb300.h``: argument
marshalling only -- every step of the method runs in the CUDA kernels of
``_build/libpic_gb300.so``.  There is no CPU fallback: if the library is not
built, every entry point raises.  PyTorch supplies streams and the device
buffers of the stateless operations.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads  # noqa: F401  (input recipes, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic_gb300.so")
_lib = None

SPECIES = {"e": 0, "i": 1, "tp": 2}
DIAG = {"phi": 0, "n_e": 1, "n_i": 2, "gamma_e": 3, "gamma_i": 4, "v_e": 5, "v_i": 6, "eedf": 7,
        "iedf_l": 8, "iedf_r": 9, "ieadf_l": 10, "ieadf_r": 11, "sputter_e_l": 12,
        "sputter_e_r": 13, "sputter_ang_l": 14, "sputter_ang_r": 15, "tp_dens": 16, "tp_v": 17,
        "E": 18, "phi_now": 19, "tpf_time": 20, "tpf_vx": 21}
COUNTERS = ["n_e_slots", "n_i_slots", "n_tp_slots", "step", "tp_step", "imp_e_l", "imp_e_r",
            "imp_i_l", "imp_i_r", "ionizations", "sputtered_l", "sputtered_r", "tp_dep_l",
            "tp_dep_r", "numerics", "elastic", "excitation", "cx", "iso", "tp_coll", "capacity"]
KERNEL = {"step": 0, "tp": 1, "compact": 2}


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class PicParams(C.Structure):
    """Mirror of ``pic_params``."""
    _fields_ = [("gap_m", C.c_double), ("pressure_pa", C.c_double), ("gas_temp_k", C.c_double),
                ("rf_freq_hz", C.c_double), ("rf_volt_v", C.c_double), ("weight", C.c_double),
                ("dt", C.c_double), ("te0_ev", C.c_double), ("ti0_ev", C.c_double),
                ("tp_dt", C.c_double), ("sigma_tp", C.c_double), ("n_e0", C.c_int64),
                ("n_i0", C.c_int64), ("cap_e", C.c_int64), ("cap_i", C.c_int64),
                ("cap_tp", C.c_int64), ("seed", C.c_uint64), ("n_cells", C.c_int32),
                ("pos_precision", C.c_int32), ("sputter_enable", C.c_int32),
                ("tp_every", C.c_int32), ("diag_every", C.c_int32), ("sort_every_e", C.c_int32),
                ("sort_every_i", C.c_int32), ("sort_every_tp", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("strict", C.c_int32), ("waveform", C.c_int32),
                ("circuit", C.c_int32), ("rf_phase", C.c_double), ("c_block", C.c_double),
                ("tp_model", C.c_int32), ("tp_mode", C.c_int32), ("tp_dref", C.c_double),
                ("tp_omega", C.c_double), ("tp_tref", C.c_double), ("id_offset", C.c_int64)]


class ServerOpts(C.Structure):
    """Mirror of ``pic_server_opts``."""
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("min_periods", C.c_int32), ("max_periods", C.c_int32),
                ("tol", C.c_double), ("batched", C.c_int32), ("graphs", C.c_int32),
                ("chunks_per_period", C.c_int32), ("criterion", C.c_int32), ("window_periods", C.c_int32),
                ("pad", C.c_int32)]


class RequestInfo(C.Structure):
    """Mirror of ``pic_request_info``."""
    _fields_ = [("id", C.c_int64), ("state", C.c_int32), ("periods", C.c_int32), ("t_arrival", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("change", C.c_double),
                ("bytes", C.c_int64), ("particles", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["state"] = REQUEST_STATES[self.state]
        return d


class ServerStats(C.Structure):
    """Mirror of ``pic_server_stats``."""
    _fields_ = [("queued", C.c_int64), ("running", C.c_int64), ("done", C.c_int64), ("bytes_used", C.c_int64),
                ("budget", C.c_int64), ("chunks", C.c_int64), ("steps", C.c_int64),
                ("particle_steps", C.c_double), ("busy_s", C.c_double)]


REQUEST_STATES = ["queued", "running", "converged", "max_periods", "rejected", "failed"]


class TpSource(C.Structure):
    _fields_ = [("n", C.c_int64), ("e_ion_ev", C.c_double), ("first_id", C.c_int64)]


def lib():
    """Load the engine library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA engine library missing ({LIB_PATH}); build it with "
                              "`python -m paper_1607_04069_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl, pi64 = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.POINTER(C.c_int64)
        sig = {
            "pic_params_default": [C.POINTER(PicParams)],
            "pic_create": [C.POINTER(PicParams), vp, C.POINTER(vp)],
            "pic_step": [vp, i64],
            "pic_sync": [vp],
            "pic_exchange_slot": [vp, C.POINTER(vp), pi64],
            "pic_test_wait_timeout": [vp, C.c_int],
            "pic_diag": [vp, C.c_int, vp, i64, pi64],
            "pic_reset_averages": [vp],
            "pic_counters": [vp, vp, i64, pi64],
            "pic_get_species": [vp, C.c_int, i64, vp, vp, vp, vp, vp, pi64],
            "pic_set_species": [vp, C.c_int, i64, vp, vp, vp, vp, vp, C.c_int],
            "pic_get_field": [vp, vp, vp, vp, vp],
            "pic_set_field": [vp, vp],
            "tp_launch": [vp, C.POINTER(TpSource)],
            "tp_step": [vp, i64, pi64],
            "tp_flight": [vp, i64, pi64],
            "pic_hypotheses": [vp, vp],
            "pic_set_cross_section": [vp, C.c_int, i64, vp, vp],
            "pic_compact": [vp, C.c_int],
            "pic_timing": [vp, C.c_int],
            "pic_kernel_time": [vp, C.c_int, C.POINTER(dbl), pi64],
            "pic_derived": [vp, vp],
            "pic_trace": [vp, C.c_int],
            "pic_trace_read": [vp, vp, i64, pi64],
            "pic_op_deposit": [vp, C.c_int, i64, i32, vp, vp],
            "pic_op_poisson": [vp, vp, i32, dbl, dbl, dbl, vp, vp, vp],
            "pic_op_sort_noalloc": [C.c_int, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "pic_batch_create": [vp, C.POINTER(vp)],
            "pic_batch_add": [vp, C.POINTER(PicParams), C.POINTER(C.c_int)],
            "pic_batch_remove": [vp, C.c_int],
            "pic_batch_ctx": [vp, C.c_int, C.POINTER(vp)],
            "pic_batch_set_target": [vp, i64],
            "pic_batch_set_chunk": [vp, i64],
            "pic_batch_step": [vp, i64],
            "pic_batch_sync": [vp],
            "pic_batch_graphs": [vp, C.c_int],
            "pic_batch_timing": [vp, C.c_int, C.POINTER(dbl), pi64],
            "pic_batch_autotune": [vp, vp, C.c_int, i64, pi64],
            "pic_state_bytes": [C.POINTER(PicParams), pi64],
            "pic_server_opts_default": [C.POINTER(ServerOpts)],
            "pic_server_create": [C.POINTER(ServerOpts), C.POINTER(vp)],
            "pic_server_clock": [vp, C.POINTER(dbl)],
            "pic_server_submit": [vp, C.POINTER(PicParams), dbl, pi64],
            "pic_server_info": [vp, i64, C.POINTER(RequestInfo)],
            "pic_server_wait": [vp, i64, dbl, C.POINTER(RequestInfo)],
            "pic_server_error": [vp, i64, C.c_char_p, i64],
            "pic_server_result": [vp, i64, C.c_int, vp, i64, pi64],
            "pic_server_forget": [vp, i64],
            "pic_server_status": [vp, C.POINTER(ServerStats)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        for name in ("pic_destroy", "pic_batch_destroy", "pic_server_destroy"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = None
        L.pic_strerror.argtypes = [C.c_int]
        L.pic_strerror.restype = C.c_char_p
        L.pic_vhs_dref.argtypes = [dbl, dbl, dbl, dbl]
        L.pic_vhs_dref.restype = dbl
        L.pic_last_error.argtypes = []
        L.pic_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        L = lib()
        raise PicError(rc, f"{L.pic_strerror(rc).decode()}: {L.pic_last_error().decode()}")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _CudaArray:
    """A device buffer owned by the library, exposed to torch through the
    CUDA array interface (no copy, no ownership)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _device_view(ptr, n, dtype):
    """A torch tensor that aliases n elements at device address ptr."""
    import torch
    typestr = {torch.int64: "<i8", torch.float64: "<f8"}[dtype]
    t = torch.as_tensor(_CudaArray(ptr, n, typestr))
    if t.data_ptr() != int(ptr) or t.device.type != "cuda":
        raise RuntimeError("torch copied the library's buffer instead of viewing it")
    return t


def default_params() -> PicParams:
    p = PicParams()
    _check(lib().pic_params_default(C.byref(p)))
    return p


def params_from_workload(cfg: dict, **over) -> PicParams:
    """Fill a PicParams from a workload dict (see ``workloads``)."""
    p = default_params()
    for name, _ in PicParams._fields_:
        if name in cfg:
            setattr(p, name, cfg[name])
    for k, v in over.items():
        setattr(p, k, v)
    return p


class Discharge:
    """One discharge on the current CUDA device (``pic_create`` .. ``pic_destroy``)."""

    def __init__(self, params, stream=None):
        if isinstance(params, dict):
            params = params_from_workload(params)
        self.params = params
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        _check(lib().pic_create(C.byref(params), C.c_void_p(self.stream), C.byref(h)))
        self.h = h
        self.n_cells = params.n_cells

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib().pic_destroy(self.h)
            self.h = None

    __del__ = close

    def step(self, n=1):
        _check(lib().pic_step(self.h, int(n)))

    def sync(self):
        _check(lib().pic_sync(self.h))

    def diag(self, kind) -> np.ndarray:
        k = DIAG[kind] if isinstance(kind, str) else int(kind)
        n = C.c_int64()
        _check(lib().pic_diag(self.h, k, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        _check(lib().pic_diag(self.h, k, _ptr(out), out.size, C.byref(n)))
        return out

    def reset_averages(self):
        _check(lib().pic_reset_averages(self.h))

    def hypotheses(self) -> dict:
        """The paper's checks of its modelling assumptions (``pic_hypotheses``)."""
        out = np.zeros(6)
        _check(lib().pic_hypotheses(self.h, _ptr(out)))
        keys = ["dE_over_E_l", "dE_over_E_r", "rms_angle_l_deg", "rms_angle_r_deg", "n_ion_over_n_gas",
                "n_al_over_n_gas"]
        return dict(zip(keys, out.tolist()))

    def counters(self) -> dict:
        out = np.zeros(64, dtype=np.int64)
        n = C.c_int64()
        _check(lib().pic_counters(self.h, _ptr(out), out.size, C.byref(n)))
        return dict(zip(COUNTERS, out[: n.value].tolist()))

    def get_species(self, s) -> dict:
        s = SPECIES.get(s, s)
        n = C.c_int64()
        _check(lib().pic_get_species(self.h, s, 0, None, None, None, None, None, C.byref(n)))
        m = n.value
        xi = np.zeros(m)
        v = [np.zeros(m, dtype=np.float32) for _ in range(3)]
        ids = np.zeros(m, dtype=np.uint64)
        _check(lib().pic_get_species(self.h, s, m, _ptr(xi), *[_ptr(a) for a in v], _ptr(ids),
                                     C.byref(n)))
        return {"xi": xi, "vx": v[0], "vy": v[1], "vz": v[2], "id": ids}

    def set_species(self, s, pos, vx, vy, vz, ids, keep_field=False):
        s = SPECIES.get(s, s)
        p64 = self.params.pos_precision == 64 and s != 2
        pos = np.ascontiguousarray(pos, dtype=np.float64 if p64 else np.uint32)
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (vx, vy, vz)]
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        _check(lib().pic_set_species(self.h, s, pos.size, _ptr(pos), *[_ptr(a) for a in arrs],
                                     _ptr(ids), int(bool(keep_field))))

    def get_field(self) -> dict:
        n = self.n_cells + 1
        E, phi = np.zeros(n), np.zeros(n)
        qe, qi = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
        _check(lib().pic_get_field(self.h, _ptr(E), _ptr(phi), _ptr(qe), _ptr(qi)))
        return {"E": E, "phi": phi, "q_e": qe, "q_i": qi}

    def set_field(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        _check(lib().pic_set_field(self.h, _ptr(E)))

    def tp_launch(self, n, e_ion_ev, first_id=-1):
        """Atoms of a mono-energetic source; first_id >= 0 gives them the ids
        first_id .. first_id + n - 1 (one rank's share of a split source)."""
        src = TpSource(int(n), float(e_ion_ev), int(first_id))
        _check(lib().tp_launch(self.h, C.byref(src)))

    def exchange_slot(self):
        """The device int64 block of the current step that ranks sharing one
        discharge sum in place before the next step (``pic_exchange_slot``),
        as a torch tensor viewing the context's memory.  The block rotates
        with the step: ask for it after every step."""
        import torch
        ptr, n = C.c_void_p(), C.c_int64()
        _check(lib().pic_exchange_slot(self.h, C.byref(ptr), C.byref(n)))
        views = self.__dict__.setdefault("_views", {})
        if ptr.value not in views:
            views[ptr.value] = _device_view(ptr.value, n.value, torch.int64)
        return views[ptr.value]

    def test_wait_timeout(self, enable=True):
        """Make the TP step's first bounded wait of one warp run out
        (``pic_test_wait_timeout``; for tests)."""
        _check(lib().pic_test_wait_timeout(self.h, int(bool(enable))))

    def tp_step(self, n=1, count_alive=True):
        a = C.c_int64()
        _check(lib().tp_step(self.h, int(n), C.byref(a) if count_alive else None))
        return a.value if count_alive else None

    def tp_flight(self, max_events=1_000_000):
        """Event-driven flight of the test particles, at most max_events
        events per atom; returns the atoms still in flight."""
        a = C.c_int64()
        _check(lib().tp_flight(self.h, int(max_events), C.byref(a)))
        return a.value

    def set_cross_section(self, process, energy_ev, sigma_m2):
        """Tabulated e-Ar cross section of process 0/1/2 (``pic_set_cross_section``);
        empty arrays restore the analytic form."""
        E = np.ascontiguousarray(energy_ev, dtype=np.float64)
        sg = np.ascontiguousarray(sigma_m2, dtype=np.float64)
        _check(lib().pic_set_cross_section(self.h, int(process), E.size, _ptr(E), _ptr(sg)))

    def compact(self, s):
        _check(lib().pic_compact(self.h, SPECIES.get(s, s)))

    def timing(self, enable=True):
        _check(lib().pic_timing(self.h, int(bool(enable))))

    def kernel_time(self, kind="step"):
        ms, n = C.c_double(), C.c_int64()
        _check(lib().pic_kernel_time(self.h, KERNEL.get(kind, kind), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def trace(self, enable=True):
        _check(lib().pic_trace(self.h, int(bool(enable))))

    def trace_read(self) -> np.ndarray:
        """Per-CTA phase stamps of the last step launch, shape (grid, 16)."""
        n = C.c_int64()
        _check(lib().pic_trace_read(self.h, None, 0, C.byref(n)))
        out = np.zeros(n.value, dtype=np.uint64)
        _check(lib().pic_trace_read(self.h, _ptr(out), out.size, C.byref(n)))
        return out.reshape(-1, 16)

    def derived(self) -> dict:
        out = np.zeros(8)
        _check(lib().pic_derived(self.h, _ptr(out)))
        keys = ["n_gas", "dx", "nu_max_e", "nu_max_i", "p_max_e", "p_max_i", "eps_max", "lambda"]
        return dict(zip(keys, out.tolist()))


class Batch:
    """Independent discharges stepped together, one step launch for all of
    them (``pic_batch_*``).  Members share dt and diag_every, use 32-bit
    positions and a whole number of steps per RF period."""

    def __init__(self, stream=None, particles_per_cta=None, particles_per_chunk=None):
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        _check(lib().pic_batch_create(C.c_void_p(self.stream), C.byref(h)))
        self.h = h
        self._params = {}
        if particles_per_cta is not None:
            _check(lib().pic_batch_set_target(self.h, int(particles_per_cta)))
        if particles_per_chunk is not None:
            self.set_chunk(particles_per_chunk)

    def set_chunk(self, particles_per_chunk):
        """Resident CTAs taking chunks of this many particles (0: one CTA per slot)."""
        _check(lib().pic_batch_set_chunk(self.h, int(particles_per_chunk)))

    def add(self, params) -> int:
        if isinstance(params, dict):
            params = params_from_workload(params)
        slot = C.c_int()
        _check(lib().pic_batch_add(self.h, C.byref(params), C.byref(slot)))
        self._params[slot.value] = params
        return slot.value

    def remove(self, slot):
        _check(lib().pic_batch_remove(self.h, int(slot)))
        self._params.pop(int(slot), None)

    def member(self, slot) -> Discharge:
        """A view of the member in ``slot`` (diagnostics, counters, particles);
        the batch owns it and steps it."""
        h = C.c_void_p()
        _check(lib().pic_batch_ctx(self.h, int(slot), C.byref(h)))
        d = Discharge.__new__(Discharge)
        d.h, d._owned, d.stream = h, False, self.stream
        d.params = self._params[int(slot)]
        d.n_cells = d.params.n_cells
        return d

    def step(self, n=1):
        _check(lib().pic_batch_step(self.h, int(n)))

    def sync(self):
        _check(lib().pic_batch_sync(self.h))

    def graphs(self, enable=True):
        _check(lib().pic_batch_graphs(self.h, int(bool(enable))))

    def timing(self, enable=True):
        """Turn launch timing on or off; returns (ms, steps) recorded since the last call."""
        ms, n = C.c_double(), C.c_int64()
        _check(lib().pic_batch_timing(self.h, int(bool(enable)), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def autotune(self, candidates=None, steps_each=20) -> int:
        """Pick the particles-per-CTA division by timing real steps; returns it."""
        best = C.c_int64()
        if candidates:
            arr = (C.c_int64 * len(candidates))(*[int(c) for c in candidates])
            _check(lib().pic_batch_autotune(self.h, C.cast(arr, C.c_void_p), len(candidates), int(steps_each),
                                            C.byref(best)))
        else:
            _check(lib().pic_batch_autotune(self.h, None, 0, int(steps_each), C.byref(best)))
        return best.value

    def close(self):
        if getattr(self, "h", None):
            lib().pic_batch_destroy(self.h)
            self.h = None

    __del__ = close


def vhs_dref(mu_ref, t_ref, omega, mass_kg) -> float:
    """VHS reference diameter from a viscosity (``pic_vhs_dref``)."""
    return float(lib().pic_vhs_dref(float(mu_ref), float(t_ref), float(omega), float(mass_kg)))


def state_bytes(params) -> int:
    """Device bytes a discharge with these parameters holds (``pic_state_bytes``)."""
    if isinstance(params, dict):
        params = params_from_workload(params)
    n = C.c_int64()
    _check(lib().pic_state_bytes(C.byref(params), C.byref(n)))
    return n.value


class Server:
    """Request loop running discharges to periodic steady state (``pic_server_*``).
    Its worker thread owns the device work; every method is thread-safe."""

    def __init__(self, **opts):
        o = ServerOpts()
        _check(lib().pic_server_opts_default(C.byref(o)))
        for k, v in opts.items():
            setattr(o, k, v)
        h = C.c_void_p()
        _check(lib().pic_server_create(C.byref(o), C.byref(h)))
        self.h = h
        self.opts = o

    def clock(self) -> float:
        t = C.c_double()
        _check(lib().pic_server_clock(self.h, C.byref(t)))
        return t.value

    def submit(self, params, t_arrival=-1.0) -> int:
        if isinstance(params, dict):
            params = params_from_workload(params)
        rid = C.c_int64()
        _check(lib().pic_server_submit(self.h, C.byref(params), float(t_arrival), C.byref(rid)))
        return rid.value

    def info(self, rid) -> dict:
        i = RequestInfo()
        _check(lib().pic_server_info(self.h, int(rid), C.byref(i)))
        return i.as_dict()

    def wait(self, rid, timeout=-1.0) -> dict:
        i = RequestInfo()
        _check(lib().pic_server_wait(self.h, int(rid), float(timeout), C.byref(i)))
        return i.as_dict()

    def error(self, rid) -> str:
        buf = C.create_string_buffer(512)
        _check(lib().pic_server_error(self.h, int(rid), buf, len(buf)))
        return buf.value.decode()

    def result(self, rid, what) -> np.ndarray:
        k = {"n_e": 0, "n_i": 1, "phi": 2}.get(what, what)
        n = C.c_int64()
        _check(lib().pic_server_result(self.h, int(rid), int(k), None, 0, C.byref(n)))
        out = np.zeros(n.value)
        _check(lib().pic_server_result(self.h, int(rid), int(k), _ptr(out), out.size, C.byref(n)))
        return out

    def forget(self, rid):
        _check(lib().pic_server_forget(self.h, int(rid)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().pic_server_status(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().pic_server_destroy(self.h)
            self.h = None

    __del__ = close


# ------------------------------------------------------------------ stateless ops (torch buffers)
def _cuda_operands(tensors, names):
    """Every operand a contiguous tensor on one CUDA device; returns that device."""
    dev = None
    for t, name in zip(tensors, names):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError(f"{name} is on {t.device}, the other operands on {dev}")
    return dev


def op_deposit(pos, n_cells: int, q=None, stream=None):
    """Linear charge assignment of device positions ``pos`` (torch uint32 /
    int32 fixed point or float64 cell units) into int64 ``q`` (returned)."""
    import torch
    if pos.dtype not in (torch.int32, torch.uint32, torch.float64):
        raise ValueError("pos must be int32/uint32 (fixed point) or float64 (cell units)")
    prec = 64 if pos.dtype == torch.float64 else 32
    if q is None:
        q = torch.zeros(n_cells + 1, dtype=torch.int64, device=pos.device)
    if q.dtype != torch.int64 or q.numel() < n_cells + 1:
        raise ValueError("q must be an int64 tensor of at least n_cells + 1 elements")
    dev = _cuda_operands((pos, q), ("pos", "q"))
    with torch.cuda.device(dev):
        _check(lib().pic_op_deposit(C.c_void_p(pos.data_ptr()), prec, pos.numel(), int(n_cells),
                                    C.c_void_p(q.data_ptr()), C.c_void_p(_stream_handle(stream))))
    return q


def op_poisson(q_i, q_e, n_cells: int, dx: float, weight: float, v_left: float, stream=None):
    """Field solve from device int64 node counts; returns (phi, E) float64 tensors."""
    import torch
    for name, q in (("q_i", q_i), ("q_e", q_e)):
        if q.dtype != torch.int64 or q.numel() < n_cells + 1:
            raise ValueError(f"{name} must be an int64 tensor of at least n_cells + 1 elements")
    dev = _cuda_operands((q_i, q_e), ("q_i", "q_e"))
    phi = torch.empty(n_cells + 1, dtype=torch.float64, device=dev)
    E = torch.empty_like(phi)
    with torch.cuda.device(dev):
        _check(lib().pic_op_poisson(C.c_void_p(q_i.data_ptr()), C.c_void_p(q_e.data_ptr()),
                                    int(n_cells), float(dx), float(weight), float(v_left),
                                    C.c_void_p(phi.data_ptr()), C.c_void_p(E.data_ptr()),
                                    C.c_void_p(_stream_handle(stream))))
    return phi, E


def op_sort_noalloc(pos, vx, vy, vz, ids, n_cells: int, pos_out, vx_out, vy_out, vz_out, ids_out,
                    n_out=None, stream=None):
    """Counting sort by cell of device particle arrays into caller-owned
    outputs, allocating no device memory (the library's static scratch holds
    up to 4096 cells).  ``n_out``: optional device int64 tensor receiving the
    number of particles kept.  Calls whose work may overlap on the GPU race on
    the shared scratch and must be ordered by the caller."""
    import torch
    if pos.dtype not in (torch.int32, torch.uint32, torch.float64):
        raise ValueError("pos must be int32/uint32 (fixed point) or float64 (cell units)")
    if pos_out.dtype != pos.dtype:
        raise ValueError("pos_out must have the dtype of pos")
    for name, a in (("vx", vx), ("vy", vy), ("vz", vz), ("vx_out", vx_out), ("vy_out", vy_out),
                    ("vz_out", vz_out)):
        if a.dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
    for name, a in (("ids", ids), ("ids_out", ids_out)):
        if a.dtype not in (torch.int64, torch.uint64):
            raise ValueError(f"{name} must be a 64-bit integer tensor")
    if n_out is not None and (n_out.dtype != torch.int64 or n_out.numel() < 1):
        raise ValueError("n_out must be an int64 tensor of at least one element")
    prec = 64 if pos.dtype == torch.float64 else 32
    n = pos.numel()
    for a in (vx, vy, vz, ids, pos_out, vx_out, vy_out, vz_out, ids_out):
        if a.numel() < n:
            raise ValueError("every particle array needs room for pos.numel() slots")
    ops = [pos, vx, vy, vz, ids, pos_out, vx_out, vy_out, vz_out, ids_out] + ([] if n_out is None else [n_out])
    names = ["pos", "vx", "vy", "vz", "ids", "pos_out", "vx_out", "vy_out", "vz_out", "ids_out", "n_out"]
    dev = _cuda_operands(ops, names)
    with torch.cuda.device(dev):          # the static scratch of that device
        _check(lib().pic_op_sort_noalloc(prec, n, int(n_cells), *[C.c_void_p(a.data_ptr()) for a in
                                         (pos, vx, vy, vz, ids, pos_out, vx_out, vy_out, vz_out, ids_out)],
                                         None if n_out is None else C.c_void_p(n_out.data_ptr()),
                                         C.c_void_p(_stream_handle(stream))))
