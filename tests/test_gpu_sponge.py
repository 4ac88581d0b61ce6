"""GPU parity of the absorbing layers (adi_set_sponge; Cerjan damping, Sec. 2.1) against the
oracle's damped mode: FP64 <= 1e-12 of max |field|, FP32 relative L2 <= 1e-4, every solver,
square and rectangular grids, with a Ricker source, with time-harmonic walls, inside a batch
(equal to the member alone), and switched off again.  Plus the physics at scale: a pulse in a
1024^2 FP32 grid loses its energy in the layers.
"""
import math

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


def _case(method, nx, ny, seed):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    h = 1.0 / max(nx, ny)
    c = rng.uniform(0.6, 1.4, su)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    return h, 0.8 * h / c.max(), c, U, V, W


def _check(G, O, precision):
    for g, o in zip(G, O):
        if precision == 1:
            assert _max_rel(g, o) <= 1e-12, _max_rel(g, o)
        else:
            assert _l2_rel(g, o) <= 1e-4, _l2_rel(g, o)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("method,nx,ny", [(CFD, 40, 31), (MFD, 33, 45), (CFD, 230, 97), (MFD, 120, 260)])
def test_sponge_vs_oracle(adi, method, nx, ny, solver, precision):
    h, dt, c, U, V, W = _case(method, nx, ny, seed=3 * nx + ny + method)
    width, a = 8.5, 0.12
    src = (ny // 2, nx // 3, 0.8, 13.0, 0.01)
    steps = 4
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=precision, solver=solver)
    s.set_source(*src)
    s.set_sponge(width, a)
    s.step(steps)
    G = s.read()
    s.close()
    O = oracle.run_sponge(method, nx, ny, h, dt, c ** 2, U, V, W, steps, width, a, source=src,
                          threads=max(1, oracle.num_threads()))
    _check(G, O, precision)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_sponge_with_harmonic_walls(adi, method):
    """Layers and time-harmonic walls together: after each step the walls are set, the damping
    spares them, and the oracle does the same (harmonic step, then damping)."""
    nx, ny = 36, 30
    h, dt, c, U, V, W = _case(method, nx, ny, seed=71 + method)
    rng = np.random.default_rng(5)
    su = wl.shapes(method, nx, ny)[0]
    B = rng.standard_normal(su)
    om, pb, pf = 6.0, 0.2, 0.0
    U[0, :] = B[0, :] * math.cos(pb); U[-1, :] = B[-1, :] * math.cos(pb)
    U[:, 0] = B[:, 0] * math.cos(pb); U[:, -1] = B[:, -1] * math.cos(pb)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    s.set_harmonic(B, None, om, pb, pf)
    s.set_sponge(6.0, 0.2)
    s.step(3)
    G = s.read()
    s.close()
    O = oracle.run_harmonic(method, nx, ny, h, dt, c ** 2, U, V, W, 3, B, None, om, pb, pf,
                            sponge=(6.0, 0.2))
    _check(G, O, 1)


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_with_sponge_member_equals_alone(adi, precision):
    specs = [(CFD, 30, 41, True), (MFD, 50, 20, False), (MFD, 33, 33, True), (CFD, 64, 17, False)]
    cases = [_case(m, nx, ny, seed=120 + k) for k, (m, nx, ny, _) in enumerate(specs)]

    def make(k):
        (m, nx, ny, sp), (h, dt, c, U, V, W) = specs[k], cases[k]
        s = adi.Sim(m, nx, ny, h, dt, c, U, V, W, precision=precision)
        if sp:
            s.set_sponge(7.0, 0.1)
        return s

    alone = []
    for k in range(len(specs)):
        s = make(k)
        s.step(5)
        alone.append(s.read())
        s.close()
    sims = [make(k) for k in range(len(specs))]
    b = adi.Batch(sims)
    b.step(5)
    b.sync()
    for s, ref in zip(sims, alone):
        for x, y in zip(s.read(), ref):
            assert np.array_equal(x, y)
    b.close()
    for s in sims:
        s.close()


def test_sponge_off_again(adi):
    method, nx, ny = CFD, 30, 26
    h, dt, c, U, V, W = _case(method, nx, ny, seed=61)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=adi.ADI_FP64)
    s.set_sponge(5.0, 0.3)
    s.step(2)
    s.set_sponge(0.0, 0.0)
    s.step(3)
    G = s.read()
    s.close()
    O = oracle.run_sponge(method, nx, ny, h, dt, c ** 2, U, V, W, 2, 5.0, 0.3)
    O = oracle.run(method, nx, ny, h, dt, c ** 2, *O, 3, t0=2 * dt)
    _check(G, O, 1)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_pulse_energy_absorbed_at_1024(adi, method):
    """A Gaussian pulse at the centre of a 1024^2 unit-speed grid (FP32, dt = 0.5 h): with
    layers 100 cells wide its energy falls below 1 % once the pulse has crossed them (2000
    steps = t 0.98).  Without layers MFD keeps its energy within 10 %; CFD is not run without
    layers here: its growing boundary modes (about 0.1/h per unit time) would overflow FP32 at
    this size, while the layers damp them along with the pulse."""
    N = 1024
    h = 1.0 / N
    su, sv, sw = wl.shapes(method, N, N)
    (ux, uy), _, _ = wl.point_coords(method, N, N, h)
    X, Y = np.meshgrid(ux, uy)
    U = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.02 ** 2))
    U[0, :] = U[-1, :] = 0.0
    U[:, 0] = U[:, -1] = 0.0

    def energy(F):
        return 0.5 * h * h * (np.sum(F[0][1:-1, 1:-1] ** 2) + np.sum(F[1] ** 2) + np.sum(F[2] ** 2))

    E0 = energy((U, np.zeros(sv), np.zeros(sw)))
    out = {}
    for layers in ((False, True) if method == MFD else (True,)):
        s = adi.Sim(method, N, N, h, 0.5 * h, np.ones(su), U, precision=adi.ADI_FP32)
        if layers:
            s.set_sponge(100.0, 0.015)
        s.step(2000)
        out[layers] = energy(s.read()) / E0
        s.close()
    if method == MFD:
        assert 0.9 < out[False] < 1.1, out
    assert out[True] < 0.01, out


@pytest.mark.parametrize("precision", [1, 0])
def test_sponge_split_lines_vs_oracle(adi, precision):
    """4700-cell x-lines (split into sub-lines by the factored solver) with absorbing layers."""
    method, nx, ny = CFD, 4700, 24
    h, dt, c, U, V, W = _case(method, nx, ny, seed=4747)
    s = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=precision)
    assert s.solver == adi.ADI_SOLVER_FACTORED
    s.set_sponge(30.0, 0.04)
    s.step(2)
    G = s.read()
    s.close()
    O = oracle.run_sponge(method, nx, ny, h, dt, c ** 2, U, V, W, 2, 30.0, 0.04,
                          threads=max(1, oracle.num_threads()))
    _check(G, O, precision)
