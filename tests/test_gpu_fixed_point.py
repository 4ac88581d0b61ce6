"""The paper's fixed-point stage solver on the GPU (adi_fixed_point: Eq. 9, Algorithms 3-4,
with the convergence test on the device) against the oracle's fixed-point mode (oracle.run
with kmax > 0) on the same seeded inputs, and its limit: with enough sweeps the iteration
reaches the exact line solves of the default path.

Tolerances: FP64 max |difference| <= 1e-12 x max |field|; FP32 relative L2 <= 1e-4 per field.
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


def _case(method, nx, ny, seed, cfl):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    h = 1.0 / max(nx, ny)
    c = rng.uniform(0.6, 1.4, su)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    return h, cfl * h / c.max(), c, U, V, W


def _check(got, want, precision):
    for g, o in zip(got, want):
        if precision == 1:
            assert np.max(np.abs(g - o)) <= 1e-12 * max(np.max(np.abs(o)), 1e-300)
        else:
            assert np.linalg.norm(g - o) <= 1e-4 * np.linalg.norm(o)


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("precision", [1, 0])
def test_fixed_sweeps_vs_oracle(adi, method, precision):
    nx, ny = 40, 33
    h, dt, c, U, V, W = _case(method, nx, ny, 60 + method, 0.6)
    steps, kmax = 3, 6
    src = (ny // 2, nx // 3, 0.5, 15.0, 0.0)
    Ug, Vg, Wg, sweeps, _ = adi.fixed_point(method, nx, ny, h, dt, c, U, V, W, steps, source=src, kmax=kmax,
                                            eps=0.0, precision=precision)
    O = oracle.run(method, nx, ny, h, dt, c ** 2, U, V, W, steps, source=src, kmax=kmax, eps=0.0)
    assert sweeps == 2 * steps * kmax
    _check((Ug, Vg, Wg), O, precision)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_stops_at_eps_like_the_oracle(adi, method):
    nx, ny = 36, 30
    h, dt, c, U, V, W = _case(method, nx, ny, 70 + method, 0.4)
    steps, kmax, eps = 2, 40, 1e-7
    Ug, Vg, Wg, sweeps, _ = adi.fixed_point(method, nx, ny, h, dt, c, U, V, W, steps, kmax=kmax, eps=eps,
                                            precision=1)
    O = oracle.run(method, nx, ny, h, dt, c ** 2, U, V, W, steps, kmax=kmax, eps=eps)
    assert 2 * steps * 2 < sweeps < 2 * steps * kmax  # stopped by the test, after a few sweeps
    _check((Ug, Vg, Wg), O, 1)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_many_sweeps_reach_the_exact_line_solves(adi, method):
    nx, ny = 48, 40
    h, dt, c, U, V, W = _case(method, nx, ny, 80 + method, 0.2)
    steps = 3
    Ug, Vg, Wg, _, _ = adi.fixed_point(method, nx, ny, h, dt, c, U, V, W, steps, kmax=80, eps=0.0, precision=1)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    s.step(steps)
    exact = s.read()
    s.close()
    for g, o in zip((Ug, Vg, Wg), exact):
        assert np.max(np.abs(g - o)) <= 1e-10 * np.max(np.abs(o))


def test_rejects_bad_arguments(adi):
    h, dt, c, U, V, W = _case(CFD, 20, 20, 1, 0.5)
    with pytest.raises(adi.AdiError):
        adi.fixed_point(CFD, 20, 20, h, dt, c, U, V, W, 1, kmax=0)
    with pytest.raises(adi.AdiError):
        adi.fixed_point(CFD, 20, 20, h, dt, c, U, V, W, 1, source=(0, 5, 1.0, 15.0, 0.0))
