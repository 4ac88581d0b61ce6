"""ctypes binding of libadi (include/adi.h): argument marshalling only.

Every step of the ADI path runs inside the library's CUDA kernels.  There is no CPU
fallback: if the library cannot be loaded (not built, or no CUDA device) the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads

ADI_CFD = 0
ADI_MFD = 1
ADI_FP32 = 0
ADI_FP64 = 1
ADI_SOLVER_LINE = 0
ADI_SOLVER_CHUNKED = 1
ADI_SOLVER_FACTORED = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadi.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p


class AdiRequest(ctypes.Structure):
    """adi_request (include/adi.h)."""
    _fields_ = [("method", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("c_field", _dp), ("u0", _dp), ("v0", _dp), ("w0", _dp),
                ("nsteps", ctypes.c_int), ("has_source", ctypes.c_int),
                ("src_i", ctypes.c_int), ("src_j", ctypes.c_int),
                ("src_amp", ctypes.c_double), ("src_f0", ctypes.c_double),
                ("src_tdelay", ctypes.c_double)]


ADI_REQ_PENDING, ADI_REQ_RUNNING, ADI_REQ_DONE, ADI_REQ_FAILED = 0, 1, 2, 3

_SIGS = {
    "adi_abi_version": ([], ctypes.c_int),
    "adi_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "adi_state_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "adi_create": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                    ctypes.c_double, _dp, _dp, _dp, _dp, ctypes.c_int], ctypes.c_int),
    "adi_set_source": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                        ctypes.c_double], ctypes.c_int),
    "adi_set_stream": ([_vp, _vp], ctypes.c_int),
    "adi_set_solver": ([_vp, ctypes.c_int], ctypes.c_int),
    "adi_get_solver": ([_vp], ctypes.c_int),
    "adi_get_scan_reach": ([_vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_autotune": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp], ctypes.c_int),
    "adi_selftest_wait_timeout": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)],
                                  ctypes.c_int),
    "adi_batch_submit": ([ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                          ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_batch_poll": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_fixed_point": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp,
                         _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int, ctypes.c_double,
                         ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _dp], ctypes.c_int),
    "adi_set_harmonic": ([_vp, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "adi_fma_peak": ([ctypes.c_int, _dp], ctypes.c_int),
    "adi_set_sponge": ([_vp, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "adi_set_launch": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "adi_get_launch": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_set_fields_f32": ([_vp, _fp, _fp, _fp], ctypes.c_int),
    "adi_read_fields_f32": ([_vp, _fp, _fp, _fp], ctypes.c_int),
    "adi_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "adi_sync": ([_vp], ctypes.c_int),
    "adi_read_fields": ([_vp, _dp, _dp, _dp], ctypes.c_int),
    "adi_set_fields": ([_vp, _dp, _dp, _dp], ctypes.c_int),
    "adi_check_finite": ([_vp], ctypes.c_int),
    "adi_get_time": ([_vp, ctypes.POINTER(ctypes.c_longlong), _dp], ctypes.c_int),
    "adi_destroy": ([_vp], ctypes.c_int),
    "adi_batch_create": ([ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int], ctypes.c_int),
    "adi_batch_set_stream": ([_vp, _vp], ctypes.c_int),
    "adi_batch_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "adi_batch_sync": ([_vp], ctypes.c_int),
    "adi_batch_half_step": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "adi_batch_destroy": ([_vp], ctypes.c_int),
    "adi_batch_set_timing": ([_vp, ctypes.c_int], ctypes.c_int),
    "adi_batch_solve_time": ([_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_step_static": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                         ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "adi_server_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "adi_server_create": ([ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int],
                          ctypes.c_int),
    "adi_server_submit": ([_vp, ctypes.POINTER(AdiRequest), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_server_tick": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "adi_server_status": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp], ctypes.c_int),
    "adi_server_result": ([_vp, ctypes.c_int, _dp, _dp, _dp], ctypes.c_int),
    "adi_server_used_bytes": ([_vp], ctypes.c_size_t),
    "adi_server_destroy": ([_vp], ctypes.c_int),
}


class AdiError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().adi_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (code %d)" % (what, msg, code))


def lib():
    """Loads libadi (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build
        _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libadi.so is missing: the CUDA extension was not built")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, what: str):
    if rc != 0:
        raise AdiError(rc, what)


def _arr(a, shape):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a, a.ctypes.data_as(_dp)


def fma_peak(precision):
    """adi_fma_peak: the device's measured FMA throughput (flop/s) in FP64 or FP32."""
    out = ctypes.c_double(0.0)
    _check(lib().adi_fma_peak(int(precision), ctypes.byref(out)), "adi_fma_peak")
    return out.value


def step_static(method, nx, ny, h, dt, precision, c, u, v, w, u_out, v_out, w_out, stream=0):
    """adi_step_static on device pointers (ints): one step into caller-owned device buffers."""
    _check(lib().adi_step_static(method, nx, ny, h, dt, precision, c, u, v, w, u_out, v_out, w_out,
                                 stream or None), "adi_step_static")


def state_bytes(method, nx, ny, precision=ADI_FP32) -> int:
    return int(lib().adi_state_bytes(method, nx, ny, precision))


def selftest_wait_timeout(polls):
    """adi_selftest_wait_timeout: (gave_up, cycles) of a bounded wait that nothing completes."""
    g = ctypes.c_int(0)
    c = ctypes.c_longlong(0)
    _check(lib().adi_selftest_wait_timeout(int(polls), ctypes.byref(g), ctypes.byref(c)), "adi_selftest_wait_timeout")
    return bool(g.value), int(c.value)


def batch_submit(sims, nsteps):
    """adi_batch_submit: advance each simulation by its own step count as one asynchronous
    batch; returns the ticket (poll it with batch_poll)."""
    n = len(sims)
    hs = (_vp * n)(*[s.handle for s in sims])
    st = (ctypes.c_int * n)(*[int(k) for k in nsteps])
    t = ctypes.c_int(0)
    _check(lib().adi_batch_submit(hs, st, n, ctypes.byref(t)), "adi_batch_submit")
    return t.value


def batch_poll(ticket):
    """adi_batch_poll: True once the ticket's steps have all finished (never blocks)."""
    d = ctypes.c_int(0)
    _check(lib().adi_batch_poll(int(ticket), ctypes.byref(d)), "adi_batch_poll")
    return bool(d.value)


def fixed_point(method, nx, ny, h, dt, c, u, v, w, nsteps, t0=0.0, source=None, kmax=6, eps=0.0,
                precision=ADI_FP32):
    """adi_fixed_point: nsteps PR steps with the paper's fixed-point stage solver (Eq. 9).
    Returns (U, V, W, sweeps, device_ms); the inputs are not modified."""
    su, sv, sw = workloads.shapes(method, nx, ny)
    c, cp = _arr(c, su)
    U = np.array(u, dtype=np.float64, order="C", copy=True)
    V = np.array(v, dtype=np.float64, order="C", copy=True)
    W = np.array(w, dtype=np.float64, order="C", copy=True)
    for a, s in ((U, su), (V, sv), (W, sw)):
        if a.shape != tuple(s):
            raise ValueError("expected shape %s, got %s" % (s, a.shape))
    src = None if source is None else np.array(source, dtype=np.float64)
    sweeps = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(lib().adi_fixed_point(method, nx, ny, h, dt, cp, U.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                                 W.ctypes.data_as(_dp), int(nsteps), float(t0),
                                 src.ctypes.data_as(_dp) if src is not None else None, int(kmax), float(eps),
                                 precision, ctypes.byref(sweeps), ctypes.byref(ms)), "adi_fixed_point")
    return U, V, W, int(sweeps.value), float(ms.value)


class Sim:
    """One simulation resident on the current CUDA device (see adi_create)."""

    def __init__(self, method, nx, ny, h, dt, c, u0=None, v0=None, w0=None,
                 precision=ADI_FP32, solver=None):
        self.method, self.nx, self.ny, self.h, self.dt = method, nx, ny, h, dt
        self.precision = precision
        su, sv, sw = workloads.shapes(method, nx, ny)
        self.shapes = (su, sv, sw)
        c, cp = _arr(c, su)
        u0, up = _arr(u0, su)
        v0, vp = _arr(v0, sv)
        w0, wp = _arr(w0, sw)
        h_ = _vp()
        _check(lib().adi_create(ctypes.byref(h_), method, nx, ny, h, dt, cp, up, vp, wp,
                                precision), "adi_create")
        self._h = h_
        if solver is not None:
            self.set_solver(solver)

    @property
    def handle(self):
        return self._h

    def set_source(self, is_, js, amp, f0, tdelay):
        _check(lib().adi_set_source(self._h, is_, js, amp, f0, tdelay), "adi_set_source")

    def set_harmonic(self, B=None, F=None, omega=0.0, phase_b=0.0, phase_f=0.0):
        """adi_set_harmonic: walls B cos(omega t + phase_b), forcing F cos(omega t + phase_f)
        (arrays of U's shape); B=None returns to time-independent walls."""
        su = self.shapes[0]
        B, bp = _arr(B, su)
        F, fp = _arr(F, su)
        _check(lib().adi_set_harmonic(self._h, bp, fp, float(omega), float(phase_b), float(phase_f)),
               "adi_set_harmonic")

    def set_sponge(self, width, a):
        """adi_set_sponge: Cerjan absorbing layers `width` cells wide with strength `a`
        (width 0 or a 0 removes them)."""
        _check(lib().adi_set_sponge(self._h, float(width), float(a)), "adi_set_sponge")

    def set_stream(self, stream_ptr):
        _check(lib().adi_set_stream(self._h, _vp(stream_ptr)), "adi_set_stream")

    def set_solver(self, solver):
        _check(lib().adi_set_solver(self._h, int(solver)), "adi_set_solver")

    @property
    def solver(self):
        return lib().adi_get_solver(self._h)

    @property
    def scan_reach(self):
        """adi_get_scan_reach: the factored solver's largest chunk-joining reach (0 otherwise)."""
        r = ctypes.c_int()
        _check(lib().adi_get_scan_reach(self._h, ctypes.byref(r)), "adi_get_scan_reach")
        return r.value

    def autotune(self, trials=2, force=False):
        """adi_autotune: times every usable solver on this simulation's own state (restored
        afterwards) and keeps the fastest.  Returns (chosen solver, {solver: ms per step})."""
        chosen = ctypes.c_int(-1)
        ms = (ctypes.c_double * 3)()
        _check(lib().adi_autotune(self._h, int(trials), 1 if force else 0, ctypes.byref(chosen), ms),
               "adi_autotune")
        return chosen.value, {k: ms[k] for k in range(3) if ms[k] >= 0}

    def set_launch(self, lines_per_cta=0, ring_depth=0):
        """adi_set_launch: the factored solver's lines per CTA and staging ring depth (0 = auto)."""
        _check(lib().adi_set_launch(self._h, int(lines_per_cta), int(ring_depth)), "adi_set_launch")

    def launch(self):
        """adi_get_launch: (lines_per_cta cap, ring depth cap), 0 = automatic."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().adi_get_launch(self._h, ctypes.byref(a), ctypes.byref(b)), "adi_get_launch")
        return a.value, b.value

    def step(self, n=1):
        _check(lib().adi_step(self._h, int(n)), "adi_step")

    def sync(self):
        _check(lib().adi_sync(self._h), "adi_sync")

    def read(self):
        su, sv, sw = self.shapes
        U, V, W = np.empty(su), np.empty(sv), np.empty(sw)
        _check(lib().adi_read_fields(self._h, U.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                                     W.ctypes.data_as(_dp)), "adi_read_fields")
        return U, V, W

    def set_fields(self, U=None, V=None, W=None):
        su, sv, sw = self.shapes
        U, up = _arr(U, su)
        V, vp = _arr(V, sv)
        W, wp = _arr(W, sw)
        _check(lib().adi_set_fields(self._h, up, vp, wp), "adi_set_fields")

    def read_into(self, U, V, W):
        """adi_read_fields into caller-provided float64 C-contiguous arrays."""
        _check(lib().adi_read_fields(self._h, U.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                                     W.ctypes.data_as(_dp)), "adi_read_fields")

    def read_into_f32(self, U, V, W):
        """adi_read_fields_f32 into caller-provided float32 C-contiguous arrays."""
        for a, shp in zip((U, V, W), self.shapes):
            if a is not None:
                assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.shape == tuple(shp)
        p = [a.ctypes.data_as(_fp) if a is not None else None for a in (U, V, W)]
        _check(lib().adi_read_fields_f32(self._h, *p), "adi_read_fields_f32")

    def set_fields_f32(self, U=None, V=None, W=None):
        """adi_set_fields_f32 from float32 C-contiguous arrays (None keeps a field)."""
        p = []
        for a, shp in zip((U, V, W), self.shapes):
            if a is None:
                p.append(None)
                continue
            assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.shape == tuple(shp)
            p.append(a.ctypes.data_as(_fp))
        _check(lib().adi_set_fields_f32(self._h, *p), "adi_set_fields_f32")

    def check_finite(self):
        return lib().adi_check_finite(self._h)

    def time(self):
        s = ctypes.c_longlong()
        t = ctypes.c_double()
        _check(lib().adi_get_time(self._h, ctypes.byref(s), ctypes.byref(t)), "adi_get_time")
        return s.value, t.value

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            if _lib.adi_destroy(self._h) != 6:  # ADI_EBUSY: still in a batch; keep the handle
                self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A group of simulations advanced by one launch per half step (adi_batch_*)."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (_vp * len(self.sims))(*[s.handle for s in self.sims])
        b = _vp()
        _check(lib().adi_batch_create(ctypes.byref(b), arr, len(self.sims)), "adi_batch_create")
        self._b = b

    def set_stream(self, stream_ptr):
        _check(lib().adi_batch_set_stream(self._b, _vp(stream_ptr)), "adi_batch_set_stream")

    def step(self, n=1):
        _check(lib().adi_batch_step(self._b, int(n)), "adi_batch_step")

    def sync(self):
        _check(lib().adi_batch_sync(self._b), "adi_batch_sync")

    def set_timing(self, enable=True):
        _check(lib().adi_batch_set_timing(self._b, 1 if enable else 0), "adi_batch_set_timing")

    def solve_time(self, stage):
        """(summed ms, count) of the line-solve launches of `stage` recorded since the last query."""
        ms, n = ctypes.c_double(), ctypes.c_int()
        _check(lib().adi_batch_solve_time(self._b, int(stage), ctypes.byref(ms), ctypes.byref(n)),
               "adi_batch_solve_time")
        return ms.value, n.value

    def half_step(self, stage, write_natural=False):
        _check(lib().adi_batch_half_step(self._b, int(stage), 1 if write_natural else 0),
               "adi_batch_half_step")

    def close(self):
        if getattr(self, "_b", None) is not None and _lib is not None:
            _lib.adi_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop on the current device (adi_server_*): FIFO admission by HBM budget,
    admitted simulations advanced together as one batch, re-formed as they join and leave."""

    def __init__(self, hbm_budget, precision=ADI_FP32, quantum=100, max_active=64):
        h = _vp()
        _check(lib().adi_server_create(ctypes.byref(h), int(hbm_budget), precision, int(quantum),
                                       int(max_active)), "adi_server_create")
        self._s = h
        self._keep = {}

    def submit(self, method, nx, ny, h, dt, c, nsteps, U=None, V=None, W=None, source=None):
        su, sv, sw = workloads.shapes(method, nx, ny)
        c, cp = _arr(c, su)
        U, up = _arr(U, su)
        V, vp = _arr(V, sv)
        W, wp = _arr(W, sw)
        r = AdiRequest(method=method, nx=nx, ny=ny, h=h, dt=dt, c_field=cp, u0=up, v0=vp, w0=wp,
                       nsteps=int(nsteps), has_source=0)
        if source is not None:
            r.has_source = 1
            r.src_i, r.src_j, r.src_amp, r.src_f0, r.src_tdelay = source
        t = ctypes.c_int()
        _check(lib().adi_server_submit(self._s, ctypes.byref(r), ctypes.byref(t)), "adi_server_submit")
        self._keep[t.value] = (method, nx, ny)
        return t.value

    def tick(self):
        nr, npd = ctypes.c_int(), ctypes.c_int()
        _check(lib().adi_server_tick(self._s, ctypes.byref(nr), ctypes.byref(npd)), "adi_server_tick")
        return nr.value, npd.value

    def status(self, ticket):
        st = ctypes.c_int()
        ts, t0, t1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().adi_server_status(self._s, int(ticket), ctypes.byref(st), ctypes.byref(ts),
                                       ctypes.byref(t0), ctypes.byref(t1)), "adi_server_status")
        return st.value, ts.value, t0.value, t1.value

    def result(self, ticket):
        method, nx, ny = self._keep[ticket]
        su, sv, sw = workloads.shapes(method, nx, ny)
        U, V, W = np.empty(su), np.empty(sv), np.empty(sw)
        _check(lib().adi_server_result(self._s, int(ticket), U.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                                       W.ctypes.data_as(_dp)), "adi_server_result")
        return U, V, W

    def used_bytes(self):
        return int(lib().adi_server_used_bytes(self._s))

    def close(self):
        if getattr(self, "_s", None) is not None and _lib is not None:
            _lib.adi_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_bytes(method, nx, ny, precision=ADI_FP32) -> int:
    return int(lib().adi_server_bytes(method, nx, ny, precision))

