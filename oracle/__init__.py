"""Plain FP64 CPU oracle for the Peaceman-Rachford ADI step (arXiv 2006.07583).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg (and its ``--impl reference`` arm) may import this package.  It shares
no code with the CUDA path in ``paper_2006_07583_gb300``; the only common module is the
seeded input generator ``paper_2006_07583_gb300.workloads``, which holds none of the
method's arithmetic.

The C implementation (``adi_oracle.c``) follows Sec. 2 of the paper: Eqs. 4-10 for the
compact-FD (CFD) scheme, Eq. 12 and Algorithm 2 for the mimetic (MFD) scheme, App. A/B for
the operators.  Every exported function is pinned by a test under ``tests/`` (operator
exactness on polynomials, dense LU, the dense 2-D Kronecker step, time reversal, the exact
standing wave and its convergence rate).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

CFD = 0
MFD = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, OpenMP) into ``oracle/_build/liboracle.so``."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        ):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
            )
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_operator.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.oracle_operator.restype = ctypes.c_int
        lib.oracle_line_solve.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp, dp,
            ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int,
        ]
        lib.oracle_line_solve.restype = ctypes.c_int
        lib.oracle_run.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
            dp, dp, dp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double,
            ctypes.c_int, ctypes.POINTER(ctypes.c_int),
        ]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run_harmonic.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
            dp, dp, dp, ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
            ctypes.c_double, ctypes.c_double,
        ]
        lib.oracle_run_harmonic.restype = ctypes.c_int
        lib.oracle_run_sponge.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
            dp, dp, dp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
            ctypes.c_int,
        ]
        lib.oracle_run_sponge.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def field_shapes(method: int, nx: int, ny: int):
    """Shapes of (U, V, W) -- also the shape of kappa, which lives where U does."""
    if method == CFD:
        s = (ny + 1, nx + 1)
        return s, s, s
    return (ny + 2, nx + 2), (ny + 2, nx + 1), (ny + 1, nx + 2)


def operator(which: str, N: int, h: float) -> np.ndarray:
    """1-D operator matrix: 'P', 'Q', 'Pbar', 'Qbar' (App. A) or 'D', 'G' (App. B)."""
    codes = {"P": (0, (N + 1, N + 1)), "Q": (1, (N + 1, N + 1)), "Pbar": (2, (N - 1, N - 1)),
             "Qbar": (3, (N - 1, N + 1)), "D": (4, (N, N + 1)), "G": (5, (N + 1, N + 2))}
    code, shape = codes[which]
    out = np.zeros(shape, dtype=np.float64)
    rc = _load().oracle_operator(code, N, h, _ptr(out))
    if rc:
        raise ValueError("oracle_operator failed (N >= 8 required)")
    return out


def line_solve(method, N, h, alpha, beta, a, vm, ub0=0.0, ub1=0.0, dense=False):
    """Exact solve of one coupled line system (Eq. 8 / Eq. 10); returns (ubar, v)."""
    np_ = N - 1 if method == CFD else N
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    vm = np.ascontiguousarray(vm, dtype=np.float64)
    assert alpha.shape == (np_,) and a.shape == (np_,) and vm.shape == (N + 1,)
    ub = np.zeros(np_)
    v = np.zeros(N + 1)
    rc = _load().oracle_line_solve(method, N, h, _ptr(alpha), beta, _ptr(a), _ptr(vm),
                                   ub0, ub1, _ptr(ub), _ptr(v), 1 if dense else 0)
    if rc:
        raise RuntimeError("oracle_line_solve failed: %d" % rc)
    return ub, v


def run(method, nx, ny, h, dt, kappa, U, V, W, nsteps, t0=0.0, source=None, kmax=0,
        eps=0.0, threads=1, return_sweeps=False):
    """Advances copies of (U, V, W) by ``nsteps`` PR steps; returns the new (U, V, W).

    source: None or (is, js, amp, f0, tdelay), a Ricker point source f = s(t)/h^2 at U[is, js].
    kmax: 0 = exact line solves; > 0 = the paper's fixed-point iteration (Eq. 9).
    return_sweeps: also return an (nsteps, 2) int array with the sweeps each stage took in
    the fixed-point mode (zeros for exact solves).
    """
    su, sv, sw = field_shapes(method, nx, ny)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    V = np.array(V, dtype=np.float64, order="C", copy=True)
    W = np.array(W, dtype=np.float64, order="C", copy=True)
    assert kappa.shape == su and U.shape == su and V.shape == sv and W.shape == sw
    src = None
    if source is not None:
        src = np.array(source, dtype=np.float64)
    sweeps = np.zeros((max(int(nsteps), 1), 2), dtype=np.int32)
    rc = _load().oracle_run(method, nx, ny, h, dt, _ptr(kappa), _ptr(U), _ptr(V), _ptr(W),
                            int(nsteps), float(t0), _ptr(src) if src is not None else None,
                            int(kmax), float(eps), int(threads),
                            sweeps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc:
        raise RuntimeError("oracle_run failed: %d" % rc)
    if return_sweeps:
        return U, V, W, sweeps[:int(nsteps)].copy()
    return U, V, W


def run_harmonic(method, nx, ny, h, dt, kappa, U, V, W, nsteps, B, F=None, omega=1.0,
                 phase_b=0.0, phase_f=0.0, t0=0.0, source=None, kmax=0, eps=0.0, threads=1,
                 sponge=None):
    """run() with time-harmonic Dirichlet data u = B cos(omega t + phase_b) on U's walls and
    forcing f = F cos(omega t + phase_f) at the interior pressure points (Eq. 11's problem).
    U must hold the walls at t0.  sponge: None or (width, a), the absorbing layers of
    run_sponge after every step."""
    su, sv, sw = field_shapes(method, nx, ny)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    V = np.array(V, dtype=np.float64, order="C", copy=True)
    W = np.array(W, dtype=np.float64, order="C", copy=True)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert kappa.shape == su and U.shape == su and V.shape == sv and W.shape == sw
    assert B.shape == su
    Fp = None
    if F is not None:
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == su
        Fp = _ptr(F)
    src = None if source is None else np.array(source, dtype=np.float64)
    rc = _load().oracle_run_harmonic(method, nx, ny, h, dt, _ptr(kappa), _ptr(U), _ptr(V),
                                     _ptr(W), int(nsteps), float(t0),
                                     _ptr(src) if src is not None else None, _ptr(B), Fp,
                                     float(omega), float(phase_b), float(phase_f), int(kmax),
                                     float(eps), int(threads),
                                     float(sponge[0]) if sponge else 0.0,
                                     float(sponge[1]) if sponge else 0.0)
    if rc:
        raise RuntimeError("oracle_run_harmonic failed: %d" % rc)
    return U, V, W


def run_sponge(method, nx, ny, h, dt, kappa, U, V, W, nsteps, width, a, t0=0.0, source=None,
               threads=1):
    """run() with Cerjan absorbing layers: after every step the fields at points within
    `width` cells of a wall (distance delta) are multiplied by exp(-(a (width - delta))^2);
    the pressure's own wall values are left alone."""
    su, sv, sw = field_shapes(method, nx, ny)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    V = np.array(V, dtype=np.float64, order="C", copy=True)
    W = np.array(W, dtype=np.float64, order="C", copy=True)
    assert kappa.shape == su and U.shape == su and V.shape == sv and W.shape == sw
    src = None if source is None else np.array(source, dtype=np.float64)
    rc = _load().oracle_run_sponge(method, nx, ny, h, dt, _ptr(kappa), _ptr(U), _ptr(V), _ptr(W),
                                   int(nsteps), float(t0), _ptr(src) if src is not None else None,
                                   float(width), float(a), int(threads))
    if rc:
        raise RuntimeError("oracle_run_sponge failed: %d" % rc)
    return U, V, W


def num_threads() -> int:
    return _load().oracle_num_threads()


def trimmed_mean(rates) -> float:
    """Average of convergence rates after dropping the highest and the lowest value
    (the averaging rule of Tables 4-5)."""
    r = sorted(float(x) for x in rates)
    return float(np.mean(r[1:-1]))


def rates(errors, Ns):
    """Empirical convergence rates log(e1/e2)/log(N2/N1) between consecutive grids."""
    return [float(np.log(errors[i] / errors[i + 1]) / np.log(Ns[i + 1] / Ns[i]))
            for i in range(len(errors) - 1)]
