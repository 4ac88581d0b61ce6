"""A simulation's FP32 trajectory does not depend on how its steps are grouped into calls or on
what shares a launch with it: the results are bit-identical.

* n steps in one call equal n calls of one step with the fields read after each.  The last
  step of a call also writes the natural fields; the carried values are formed by the same
  operations whether it does or not.  Every solver, both methods, with a point source.
* A batch that mixes a simulation whose lines need the full log-depth chunk-joining scans
  (reach above 32 chunks, at a time step far beyond the seismic one) with simulations whose
  lines take the windowed scans: each member ends exactly where it ends alone, both in a
  synchronous batch and in an asynchronous one with per-member step counts.  Each launch
  group picks its scans from its own simulation's reach.
"""
import time

import numpy as np
import pytest

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


def _fields(method, nx, ny, seed):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    return rng.uniform(0.7, 1.3, su), rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("method,nx,ny", [(CFD, 150, 97), (MFD, 131, 160)])
def test_one_call_equals_single_steps_with_reads(adi, method, nx, ny, solver):
    c, U, V, W = _fields(method, nx, ny, seed=nx + ny + solver)
    h = 1.0 / max(nx, ny)
    dt = 0.9 * h / c.max()
    src = (ny // 2, nx // 3, 1.0, 9.0, 0.02)

    def make():
        s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP32, solver=solver)
        s.set_source(*src)
        return s

    a = make()
    a.step(6)
    A = a.read()
    a.close()
    b = make()
    for _ in range(6):
        b.step(1)
        B = b.read()
    b.close()
    for x, y in zip(A, B):
        assert np.array_equal(x, y)


def _full_scan_sim(adi, method, nx, ny, seed):
    """A factored FP32 simulation whose lines need the full scans: the smallest of a list of
    growing time steps whose reach exceeds 32 chunks."""
    c, U, V, W = _fields(method, nx, ny, seed)
    h = 1.0 / max(nx, ny)
    for k in (4.0, 16.0, 64.0, 256.0, 1024.0):
        s = adi.Sim(method, nx, ny, h, k * h / c.max(), c, U, V, W, precision=adi.ADI_FP32,
                    solver=adi.ADI_SOLVER_FACTORED)
        if s.scan_reach > 32:
            return (method, nx, ny, h, k * h / c.max(), c, U, V, W)
        s.close()
    raise AssertionError("no time step in the list gives a reach above 32")


def _members(adi):
    full = _full_scan_sim(adi, CFD, 330, 70, seed=3)
    out = [full]
    for k, (m, nx, ny) in enumerate([(CFD, 300, 64), (MFD, 210, 150), (CFD, 90, 200)]):
        c, U, V, W = _fields(m, nx, ny, seed=40 + k)
        h = 1.0 / max(nx, ny)
        out.append((m, nx, ny, h, 0.8 * h / c.max(), c, U, V, W))
    return out


def _make(adi, spec):
    m, nx, ny, h, dt, c, U, V, W = spec
    s = adi.Sim(m, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP32, solver=adi.ADI_SOLVER_FACTORED)
    s.set_source(ny // 2, nx // 2, 1.0, 7.0, 0.01)
    return s


def test_full_and_windowed_scans_in_one_batch_equal_alone(adi):
    specs = _members(adi)
    reach = []
    for sp in specs:
        s = _make(adi, sp)
        reach.append(s.scan_reach)
        s.close()
    assert reach[0] > 32 and all(0 < r <= 32 for r in reach[1:]), reach
    steps = 5
    alone = []
    for sp in specs:
        s = _make(adi, sp)
        s.step(steps)
        alone.append(s.read())
        s.close()
    sims = [_make(adi, sp) for sp in specs]
    b = adi.Batch(sims)
    b.step(steps)
    b.sync()
    for s, ref in zip(sims, alone):
        for x, y in zip(s.read(), ref):
            assert np.array_equal(x, y)
    b.close()
    for s in sims:
        s.close()


def test_full_and_windowed_scans_in_an_async_batch_equal_alone(adi):
    specs = _members(adi)
    nsteps = [4, 1, 6, 3]
    sims = [_make(adi, sp) for sp in specs]
    t = adi.batch_submit(sims, nsteps)
    deadline = time.time() + 60
    while not adi.batch_poll(t):
        assert time.time() < deadline
        time.sleep(0.001)
    for sp, s, n in zip(specs, sims, nsteps):
        r = _make(adi, sp)
        r.step(n)
        for x, y in zip(s.read(), r.read()):
            assert np.array_equal(x, y)
        r.close()
        s.close()
