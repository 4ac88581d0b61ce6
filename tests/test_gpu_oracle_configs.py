"""GPU against the FP64 oracle at the workloads' own sizes and step counts.

* Config 1 (standing wave, 100 x 100 cells, dt = 0.5 h) at its full 200 steps, FP64 and FP32,
  with the bars of tests/amplification.py: the per-step rounding difference of two correct
  implementations, carried forward by the growth the oracle measures on this very problem.
  MFD (a neutral step) keeps the short-run bars (1e-12, 1e-4).  CFD's growing modes widen the
  FP64 bar to about 4e-8 and make the FP32 bar uninformative (about 0.7).  Both FP64 runs and the
  FP32 MFD run are also held to the exact solution (the Crank-Nicolson phase-error bound that the
  oracle meets).  The FP32 CFD run is not: the growing modes amplify FP32 rounding about 5e5
  times over these 200 steps, which leaves it about 1e-2 from the exact solution -- a property
  of the scheme that any FP32 implementation shares; FP32 CFD is held to 1e-4 of the oracle only
  over 50 steps (test_gpu_parity.py).
* A mixed batch (CFD and MFD, square and rectangular, a split-line member 4700 x 24, a member
  with a Ricker source) against the oracle member by member: FP64 <= 1e-12, FP32 <= 1e-4.
* Config 2 (MFD, 1001 x 1001 cells, layered medium, 15 Hz Ricker) over its first 5 steps
  against the oracle on all host cores: FP64 pressure relative L2 <= 1e-12 (the target's
  metric), velocities relative L2 <= 1e-11, max difference <= 1e-11 of max |field| everywhere;
  FP32 relative L2 <= 1e-4.  In SI units (h = 5 m, c up to 5000 m/s) the pressure and velocity
  unknowns of a line differ in scale by about 1e7 and the line systems have a 2-norm condition
  number of about 4e6, so two FP64 eliminations in different orders differ by a few 1e-12 in
  the velocities (measured 4e-12 for v) while the pressure stays within 1e-12.
* A 4096-wide strip of the bench workload (the bench's 4096-cell x-lines with their seismic
  speeds, 48 rows) against the oracle, both schemes, FP64 and FP32.
* The bench configuration itself (4096 x 4096, one CFD and one MFD simulation, batched, the
  default solver): time reversal, a property of the exact PR step at any size (J S J = S^-1 with
  J flipping the velocities): n steps, flip, n steps, flip gives back the initial fields, to the
  FP64 bar or to 2n times the FP32 bar of one step (1e-4 relative L2).
"""
import math

import numpy as np
import pytest

import oracle
from amplification import bars, growth
from paper_2006_07583_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CFD, MFD = wl.CFD, wl.MFD


@pytest.fixture(scope="module")
def adi():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_07583_gb300 import adi as _adi

    _adi.lib()
    return _adi


def _max_rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _l2_rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _threads():
    return max(1, oracle.num_threads())


# ---------------------------------------------------------------------------------------
# Config 1 at its 200 steps
# ---------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c1_bars():
    N = 100
    out = {}
    for m in (CFD, MFD):
        U, V, W = wl.standing_wave(m, N, 0.0)
        gm, gl = growth(m, N, N, 1.0 / N, 0.5 / N, wl.unit_kappa(m, N, N), U, V, W, 200)
        out[m] = bars(gm, gl, 200)
    return out


@pytest.mark.parametrize("method", [CFD, MFD])
def test_config1_200_steps_vs_oracle(adi, c1_bars, method):
    N, steps = 100, 200
    h = 1.0 / N
    dt = 0.5 * h
    U, V, W = wl.standing_wave(method, N, 0.0)
    c = wl.unit_kappa(method, N, N)
    O = oracle.run(method, N, N, h, dt, c, U, V, W, steps, threads=_threads())
    b64, b32 = c1_bars[method]
    G = {}
    for prec in (adi.ADI_FP64, adi.ADI_FP32):
        s = adi.Sim(method, N, N, h, dt, c, U, V, W, precision=prec)
        s.step(steps)
        G[prec] = s.read()
        s.close()
    for g, o in zip(G[adi.ADI_FP64], O):
        assert _max_rel(g, o) <= b64, (_max_rel(g, o), b64)
    for g, o in zip(G[adi.ADI_FP32], O):
        assert _l2_rel(g, o) <= b32, (_l2_rel(g, o), b32)
    # accuracy against the exact solution: within the trapezoidal phase-error bound,
    # (omega dt)^3 / 12 per step with omega = sqrt(2) pi (the oracle meets it too)
    Ue, _, _ = wl.standing_wave(method, N, steps * dt)
    bound = (math.sqrt(2) * math.pi * dt) ** 3 / 12 * steps
    assert np.max(np.abs(O[0] - Ue)) < 1.2 * bound
    assert np.max(np.abs(G[adi.ADI_FP64][0] - Ue)) < 1.2 * bound
    if method == MFD:
        assert np.max(np.abs(G[adi.ADI_FP32][0] - Ue)) < 1.2 * bound


# ---------------------------------------------------------------------------------------
# A mixed batch, member by member against the oracle
# ---------------------------------------------------------------------------------------

def _random_case(method, nx, ny, seed):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    h = 1.0 / max(nx, ny)
    c = rng.uniform(0.6, 1.4, su)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    return h, 0.8 * h / c.max(), c, U, V, W


# (method, nx, ny, source)
MIX = [(CFD, 20, 31, None), (MFD, 33, 17, None), (CFD, 64, 64, (30, 20, 0.7, 12.0, 0.01)),
       (MFD, 16, 50, None), (MFD, 4700, 24, (12, 2400, 0.5, 15.0, 0.0)), (CFD, 130, 90, None),
       (MFD, 97, 211, (100, 50, 1.1, 9.0, 0.02))]


@pytest.mark.parametrize("precision", [1, 0])
def test_mixed_batch_members_vs_oracle(adi, precision):
    steps = 3
    cases = [_random_case(m, nx, ny, seed=200 + k) for k, (m, nx, ny, _) in enumerate(MIX)]
    sims = []
    for (m, nx, ny, src), (h, dt, c, U, V, W) in zip(MIX, cases):
        s = adi.Sim(m, nx, ny, h, dt, c, U, V, W, precision=precision)
        if src is not None:
            s.set_source(*src)
        sims.append(s)
    b = adi.Batch(sims)
    b.step(steps)
    b.sync()
    got = [s.read() for s in sims]
    b.close()
    for s in sims:
        s.close()
    for (m, nx, ny, src), (h, dt, c, U, V, W), g in zip(MIX, cases, got):
        O = oracle.run(m, nx, ny, h, dt, c ** 2, U, V, W, steps, source=src, threads=_threads())
        for x, o in zip(g, O):
            if precision == 1:
                assert _max_rel(x, o) <= 1e-12, (m, nx, ny, _max_rel(x, o))
            else:
                assert _l2_rel(x, o) <= 1e-4, (m, nx, ny, _l2_rel(x, o))


# ---------------------------------------------------------------------------------------
# Config 2's first steps, and a 4096-wide strip of the bench workload
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [1, 0])
def test_config2_1001_first_steps_vs_oracle(adi, precision):
    sp = wl.seismic_spec(MFD, 1001, 1001, 5, h=5.0, seed=1)
    su, sv, sw = wl.shapes(MFD, 1001, 1001)
    rng = np.random.default_rng(17)
    # a nonzero start, so that every line carries data from the first step on
    (ux, uy), (vx, vy), (wx, wy) = wl.point_coords(MFD, 1001, 1001, 1.0 / 1001)
    U = np.outer(np.sin(3 * np.pi * uy), np.sin(2 * np.pi * ux)) * rng.uniform(0.5, 1.5)
    V = np.outer(np.sin(np.pi * vy), np.cos(4 * np.pi * vx)) * 0.3
    W = np.zeros(sw)
    U[0, :] = U[-1, :] = 0.0
    U[:, 0] = U[:, -1] = 0.0
    src = sp.source.as_tuple()
    s = adi.Sim(MFD, 1001, 1001, sp.h, sp.dt, sp.c, U, V, W, precision=precision)
    s.set_source(*src)
    s.step(sp.steps)
    G = s.read()
    s.close()
    O = oracle.run(MFD, 1001, 1001, sp.h, sp.dt, sp.c ** 2, U, V, W, sp.steps, source=src,
                   threads=_threads())
    for k, (g, o) in enumerate(zip(G, O)):
        if precision == 1:
            assert _l2_rel(g, o) <= (1e-12 if k == 0 else 1e-11), (k, _l2_rel(g, o))
            assert _max_rel(g, o) <= 1e-11, (k, _max_rel(g, o))
        else:
            assert _l2_rel(g, o) <= 1e-4


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("precision", [1, 0])
def test_bench_strip_4096_vs_oracle(adi, method, precision):
    """48 rows of the 4096 x 4096 bench workload through its source: the same 4096-cell
    x-lines, speeds and time step as the bench, with the bench's Ricker source."""
    full = wl.seismic_spec(method, 4096, 4096, 3, h=5.0, seed=1 if method == CFD else 2)
    rows = 48
    r0 = full.source.is_ - rows // 2
    su, sv, sw = wl.shapes(method, 4096, rows)
    c = np.ascontiguousarray(full.c[r0:r0 + su[0], :])
    src = (full.source.is_ - r0, full.source.js, full.source.amp, full.source.f0,
           full.source.tdelay)
    rng = np.random.default_rng(5 + method)
    U = rng.standard_normal(su) * 1e-3
    V = rng.standard_normal(sv) * 1e-3
    W = rng.standard_normal(sw) * 1e-3
    steps = 3
    s = adi.Sim(method, 4096, rows, full.h, full.dt, c, U, V, W, precision=precision)
    assert s.solver == adi.ADI_SOLVER_FACTORED
    s.set_source(*src)
    s.step(steps)
    G = s.read()
    s.close()
    O = oracle.run(method, 4096, rows, full.h, full.dt, c ** 2, U, V, W, steps, source=src,
                   threads=_threads())
    for g, o in zip(G, O):
        if precision == 1:
            assert _max_rel(g, o) <= 1e-12
        else:
            assert _l2_rel(g, o) <= 1e-4


# ---------------------------------------------------------------------------------------
# The bench configuration: time reversal at 4096 x 4096
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [1, 0])
def test_bench_config_time_reversal(adi, precision):
    """n steps forward, velocities flipped, n steps, flipped back: the initial fields return
    (no source: a time-dependent source is not reversible).  FP64 to 1e-10 of max |field|;
    FP32 to 2n x 1e-4 relative L2 (each of the 2n steps may add the FP32 bar of one step)."""
    side, n = 4096, 2
    sims, starts = [], []
    rng = np.random.default_rng(23)
    for method, seed in ((CFD, 1), (MFD, 2)):
        sp = wl.seismic_spec(method, side, side, n, h=5.0, seed=seed)
        (ux, uy), (vx, vy), (wx, wy) = wl.point_coords(method, side, side, 1.0 / side)

        def smooth(x, y, k):
            a = rng.standard_normal(3)
            return sum(a[i] * np.outer(np.sin((i + 1) * np.pi * y), np.sin((i + k) * np.pi * x))
                       for i in range(3))

        U, V, W = smooth(ux, uy, 1), smooth(vx, vy, 2), smooth(wx, wy, 3)
        U[0, :] = U[-1, :] = 0.0
        U[:, 0] = U[:, -1] = 0.0
        sims.append(adi.Sim(method, side, side, sp.h, sp.dt, sp.c, U, V, W, precision=precision))
        starts.append((U, V, W))
    b = adi.Batch(sims)
    b.step(n)
    b.sync()
    b.close()
    for s in sims:
        U, V, W = s.read()
        s.set_fields(U, -V, -W)
    b = adi.Batch(sims)
    b.step(n)
    b.sync()
    b.close()
    for s, (U0, V0, W0) in zip(sims, starts):
        U, V, W = s.read()
        s.close()
        for got, want in ((U, U0), (-V, V0), (-W, W0)):
            if precision == 1:
                assert _max_rel(got, want) <= 1e-10
            else:
                assert _l2_rel(got, want) <= 2 * n * 1e-4, _l2_rel(got, want)
