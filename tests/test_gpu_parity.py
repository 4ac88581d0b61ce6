"""GPU parity: libadi (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs, element by element.

Tolerances (the precision policy of the path):
  * FP64 GPU vs oracle: max |difference| <= 1e-12 * max |field| per field.  The two sides
    solve the same exact line systems with different elimination orders (block Thomas
    with FP64 boundary tables vs banded partial pivoting), so they agree to rounding.
  * FP32 GPU vs oracle: relative L2 error of the pressure <= 1e-4 after the case's step
    count (velocity likewise, relative to its own norm).
The CFD scheme's PR step has spectral radius ~1.06-1.10 (its boundary closure is not
energy stable; pinned on the oracle side in test_oracle_stability.py), so any two correct
implementations drift apart geometrically: CFD cases are compared at step counts where
that amplification stays below ~20 (FP64) / ~20 (FP32); MFD (spectral radius 1) is
compared over the full 200 steps.
"""
import numpy as np
import pytest

import oracle
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


def _random_case(method, nx, ny, seed, dirichlet=True):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    h = 1.0 / max(nx, ny)
    c = rng.uniform(0.6, 1.4, su)
    U = rng.standard_normal(su)
    if not dirichlet:
        U[0, :] = U[-1, :] = 0.0; U[:, 0] = U[:, -1] = 0.0
    V = rng.standard_normal(sv)
    W = rng.standard_normal(sw)
    dt = 0.8 * h / c.max()
    return h, dt, c, U, V, W


def _run_both(adi, method, nx, ny, h, dt, c, U, V, W, steps, precision, src=None, solver=None):
    sim = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=precision, solver=solver)
    if src is not None:
        sim.set_source(*src)
    sim.step(steps)
    G = sim.read()
    sim.close()
    O = oracle.run(method, nx, ny, h, dt, c ** 2, U, V, W, steps, source=src)
    return G, O


# exact-solution case: 101x101 nodes / 100x100 cells, c = 1, dt = 0.5 h
SW_STEPS = {CFD: 50, MFD: 200}


@pytest.mark.parametrize("method", [CFD, MFD])
def test_standing_wave_fp64(adi, method):
    N = 100
    h = 1.0 / N
    dt = 0.5 * h
    steps = SW_STEPS[method]
    U, V, W = wl.standing_wave(method, N, 0.0)
    c = wl.unit_kappa(method, N, N)
    G, O = _run_both(adi, method, N, N, h, dt, c, U, V, W, steps, adi.ADI_FP64)
    for g, o in zip(G, O):
        assert _max_rel(g, o) <= 1e-12
    Ue, _, _ = wl.standing_wave(method, N, steps * dt)
    assert np.max(np.abs(G[0] - Ue)) < 2e-4


@pytest.mark.parametrize("method", [CFD, MFD])
def test_standing_wave_fp32(adi, method):
    N = 100
    h = 1.0 / N
    dt = 0.5 * h
    U, V, W = wl.standing_wave(method, N, 0.0)
    c = wl.unit_kappa(method, N, N)
    G, O = _run_both(adi, method, N, N, h, dt, c, U, V, W, SW_STEPS[method], adi.ADI_FP32)
    assert _l2_rel(G[0], O[0]) <= 1e-4
    assert _l2_rel(G[1], O[1]) <= 1e-4
    assert _l2_rel(G[2], O[2]) <= 1e-4


# sizes spanning the MFD block remainder (N - 8) mod 3 = 0, 1, 2, the minimum size, and
# rectangles
SIZES = [(16, 16), (17, 23), (18, 16), (40, 29), (61, 64)]


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_random_fields_dirichlet_fp64(adi, method, nx, ny, solver):
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=nx * 100 + ny + method)
    G, O = _run_both(adi, method, nx, ny, h, dt, c, U, V, W, 3, adi.ADI_FP64, solver=solver)
    for g, o in zip(G, O):
        assert _max_rel(g, o) <= 1e-12


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("nx,ny", [(16, 16), (45, 38)])
def test_random_fields_fp32(adi, method, nx, ny, solver):
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=7 + nx + method)
    G, O = _run_both(adi, method, nx, ny, h, dt, c, U, V, W, 5, adi.ADI_FP32, solver=solver)
    for g, o in zip(G, O):
        assert _l2_rel(g, o) <= 1e-4


@pytest.mark.parametrize("method", [CFD, MFD])
def test_point_source_fp64(adi, method):
    nx, ny = 48, 40
    spec = wl.seismic_spec(method, nx, ny, steps=30, h=5.0, seed=4)
    src = spec.source.as_tuple()
    su, sv, sw = wl.shapes(method, nx, ny)
    Z = [np.zeros(s) for s in (su, sv, sw)]
    G, O = _run_both(adi, method, nx, ny, spec.h, spec.dt, spec.c, Z[0], Z[1], Z[2], 30,
                     adi.ADI_FP64, src=src)
    assert np.max(np.abs(O[0])) > 0
    for g, o in zip(G, O):
        assert _max_rel(g, o) <= 1e-12


@pytest.mark.parametrize("method", [CFD, MFD])
def test_steps_in_pieces_equal_one_call(adi, method):
    """adi_step(3) == adi_step(1) x 3 (graph replay vs direct launches), bit for bit."""
    nx, ny = 24, 20
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=3)
    a = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP32)
    b = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP32)
    a.step(3)
    for _ in range(3):
        b.step(1)
    for x, y in zip(a.read(), b.read()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone(adi, precision):
    """Each simulation gives the same result alone and inside a mixed batch."""
    specs = [(CFD, 20, 31), (MFD, 33, 17), (CFD, 64, 64), (MFD, 16, 50)]
    cases = [_random_case(m, nx, ny, seed=k) for k, (m, nx, ny) in enumerate(specs)]
    alone, batched = [], []
    for (m, nx, ny), (h, dt, c, U, V, W) in zip(specs, cases):
        s = adi.Sim(m, nx, ny, h, dt, c, U, V, W, precision=precision)
        s.step(4)
        alone.append(s.read())
        s.close()
    sims = [adi.Sim(m, nx, ny, h, dt, c, U, V, W, precision=precision)
            for (m, nx, ny), (h, dt, c, U, V, W) in zip(specs, cases)]
    batch = adi.Batch(sims)
    batch.step(4)
    batch.sync()
    for s, ref in zip(sims, alone):
        got = s.read()
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
    batch.close()


def test_invalid_arguments_rejected(adi):
    su, sv, sw = wl.shapes(CFD, 16, 16)
    c = np.ones(su)
    with pytest.raises(adi.AdiError) as e:
        adi.Sim(CFD, 15, 16, 0.1, 0.01, np.ones(wl.shapes(CFD, 15, 16)[0]))
    assert e.value.code == 1
    bad = c.copy(); bad[3, 3] = -1.0
    with pytest.raises(adi.AdiError):
        adi.Sim(CFD, 16, 16, 0.1, 0.01, bad)
    nan = np.zeros(su); nan[2, 2] = np.nan
    with pytest.raises(adi.AdiError):
        adi.Sim(CFD, 16, 16, 0.1, 0.01, c, nan)
    s = adi.Sim(CFD, 16, 16, 0.1, 0.01, c)
    with pytest.raises(adi.AdiError):
        s.set_source(0, 5, 1.0, 10.0, 0.1)  # boundary point
    with pytest.raises(adi.AdiError):
        s.step(-1)
    assert s.check_finite() == 0
    s.close()


def test_nonfinite_detected(adi):
    """A field driven to overflow is reported as ADI_ENONFINITE by the device scan."""
    su, sv, sw = wl.shapes(MFD, 16, 16)
    U = np.zeros(su); U[5, 5] = 1e300  # finite in FP64, overflows to inf in the FP32 state
    s = adi.Sim(MFD, 16, 16, 0.1, 0.05, np.ones(su), U, precision=adi.ADI_FP32)
    s.step(2)
    assert s.check_finite() == 4
    s.close()


# multi-chunk lines.  Chunked solver: chunks of <= 32 (CFD) / 16 (MFD) blocks with separators.
# Factored solver: chunks of exactly 8 (CFD) / 2 or 3 (MFD) blocks, the remainder absorbed by
# the line ends; these sizes give every remainder, idle trailing threads, lines spanning 1, 2
# and more warps, and the longest lines of the bench (4096 cells: 512 and 480 threads per line,
# the three-block MFD chunks).
MULTI = [(CFD, 230, 171), (MFD, 260, 197), (CFD, 97, 400), (MFD, 53, 311), (CFD, 400, 150),
         (MFD, 500, 97), (CFD, 4096, 19), (MFD, 4096, 17), (MFD, 3500, 24)]


@pytest.mark.parametrize("solver", [1, 2])
@pytest.mark.parametrize("method,nx,ny", MULTI)
def test_multichunk_fp64_vs_oracle(adi, method, nx, ny, solver):
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=nx + ny)
    G, O = _run_both(adi, method, nx, ny, h, dt, c, U, V, W, 2, adi.ADI_FP64, solver=solver)
    for g, o in zip(G, O):
        assert _max_rel(g, o) <= 1e-12


@pytest.mark.parametrize("solver", [1, 2])
@pytest.mark.parametrize("method,nx,ny", MULTI)
def test_multichunk_fp32_vs_oracle(adi, method, nx, ny, solver):
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=3 * nx + ny)
    G, O = _run_both(adi, method, nx, ny, h, dt, c, U, V, W, 4, adi.ADI_FP32, solver=solver)
    for g, o in zip(G, O):
        assert _l2_rel(g, o) <= 1e-4


@pytest.mark.parametrize("method", [CFD, MFD])
def test_solvers_agree_seismic_with_source(adi, method):
    """Thread-per-line and chunked solvers on a layered medium with a Ricker source."""
    spec = wl.seismic_spec(method, 300, 280, steps=20, h=5.0, seed=9)
    out = []
    for solver in (adi.ADI_SOLVER_LINE, adi.ADI_SOLVER_CHUNKED, adi.ADI_SOLVER_FACTORED):
        s = adi.Sim(method, spec.nx, spec.ny, spec.h, spec.dt, spec.c, precision=adi.ADI_FP64,
                    solver=solver)
        assert s.solver == solver
        s.set_source(*spec.source.as_tuple())
        s.step(20)
        out.append(s.read())
        s.close()
    for ref in out[1:]:
        for a, b in zip(out[0], ref):
            assert _max_rel(a, b) <= 1e-12


@pytest.mark.parametrize("method", [CFD, MFD])
def test_set_fields_restart_matches_continuous_run(adi, method):
    """Reading the fields, loading them back (adi_set_fields) and continuing equals an
    uninterrupted FP64 run to rounding (the carried state is rebuilt from the fields)."""
    nx, ny = 70, 66
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=12)
    a = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    b = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    a.step(6)
    b.step(3)
    b.set_fields(*b.read())
    b.step(3)
    for x, y in zip(a.read(), b.read()):
        assert _max_rel(x, y) <= 1e-12


# Lines longer than one CTA's chunks (about 4330 CFD nodes / 4320 MFD cells) are split into
# sub-lines that each own a span of chunks and solve a halo of the scan reach around it.  A
# grid 4700 cells wide and 24 high has split x-lines and ordinary y-lines, small enough for
# the oracle.
@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("precision", [1, 0])
def test_split_lines_vs_oracle(adi, method, precision):
    nx, ny = 4700, 24
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=40 + method)
    steps = 2 if method == CFD else 4
    src = (ny // 2, 2400, 0.5, 15.0, 0.0)
    sim = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=precision)
    assert sim.solver == adi.ADI_SOLVER_FACTORED  # split x-lines, not a fallback
    sim.set_source(*src)
    sim.step(steps)
    G = sim.read()
    sim.close()
    O = oracle.run(method, nx, ny, h, dt, c ** 2, U, V, W, steps, source=src)
    for g, o in zip(G, O):
        if precision == 1:
            assert _max_rel(g, o) <= 1e-12
        else:
            assert _l2_rel(g, o) <= 1e-4


def test_set_fields_rejects_nonfinite_and_keeps_state(adi):
    """adi_set_fields checks its host inputs on the device before touching the state: a NaN
    or Inf in any field gives ADI_EINVAL and the fields read exactly as before."""
    method, nx, ny = CFD, 40, 30
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=91)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP32)
    s.step(3)
    before = s.read()
    for k, bad in ((0, np.nan), (1, np.inf), (2, -np.inf)):
        fields = [f.copy() for f in before]
        fields[k][3, 4] = bad
        with pytest.raises(adi.AdiError) as e:
            s.set_fields(*fields)
        assert e.value.code == 1  # ADI_EINVAL
        for a, b in zip(s.read(), before):
            assert np.array_equal(a, b)
    s.set_fields(*before)  # finite inputs are accepted
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fp32_host_field_calls(adi, precision):
    """adi_set_fields_f32 / adi_read_fields_f32: the same state as the FP64 calls on values that
    FP32 holds exactly, reads equal to the FP64 read rounded to FP32, and a NaN input rejected
    with the fields untouched."""
    method, nx, ny = MFD, 45, 38
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=515)
    U32, V32, W32 = (x.astype(np.float32) for x in (U, V, W))
    a = adi.Sim(method, nx, ny, h, dt, c, precision=precision)
    b = adi.Sim(method, nx, ny, h, dt, c, precision=precision)
    a.set_fields(*(x.astype(np.float64) for x in (U32, V32, W32)))
    b.set_fields_f32(U32, V32, W32)
    a.step(3)
    b.step(3)
    ra = a.read()
    for x, y in zip(ra, b.read()):
        assert np.array_equal(x, y)
    out = [np.empty(s, dtype=np.float32) for s in b.shapes]
    b.read_into_f32(*out)
    for x, y in zip(out, ra):
        assert np.array_equal(x, y.astype(np.float32))
    bad = [o.copy() for o in out]
    bad[1][2, 3] = np.nan
    with pytest.raises(adi.AdiError) as e:
        b.set_fields_f32(*bad)
    assert e.value.code == 1
    for x, y in zip(b.read(), ra):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.mark.parametrize("method", [CFD, MFD])
def test_source_set_after_steps_follows_the_clock(adi, method):
    """A Ricker source switched on after some source-free steps is evaluated at the simulation's
    own time (the device step clock follows the step count), as the oracle started at t0."""
    nx, ny = 40, 36
    h, dt, c, U, V, W = _random_case(method, nx, ny, seed=77)
    src = (ny // 2, nx // 2, 2.0, 9.0, 0.03)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    s.step(5)
    s.set_source(*src)
    s.step(4)
    G = s.read()
    s.close()
    O = oracle.run(method, nx, ny, h, dt, c ** 2, U, V, W, 5)
    O = oracle.run(method, nx, ny, h, dt, c ** 2, *O, 4, t0=5 * dt, source=src)
    for g, o in zip(G, O):
        assert _max_rel(g, o) <= 1e-12
