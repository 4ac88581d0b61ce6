"""Pins of the oracle's absorbing layers (Cerjan's damping, named in Sec. 2.1): after every
full step the fields at points within `width` cells of a wall are multiplied by
g = exp(-(a (width - delta))^2), delta the point's distance to the nearest wall in cells.

* a = 0 or width = 0 is the plain step, bit for bit.
* One damped step is the plain step followed by g, with g evaluated here from the mesh
  coordinates of the input generator (CFD nodes; MFD cell centres and faces).
* Energy: a Gaussian pulse in a unit-speed medium keeps its discrete energy (within 10 %)
  without layers; with layers 20 cells wide the energy falls below 1 % once the pulse has
  crossed them, and the wave reflected by the walls reaches the centre at least 50 times
  weaker.
* Before the pulse reaches the layers the damped and plain runs agree.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import CFD, MFD
from paper_2006_07583_gb300 import workloads as wl


def _pulse(method, N):
    h = 1.0 / N
    su, sv, sw = wl.shapes(method, N, N)
    (ux, uy), _, _ = wl.point_coords(method, N, N, h)
    X, Y = np.meshgrid(ux, uy)
    U = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.04 ** 2))
    U[0, :] = U[-1, :] = 0.0
    U[:, 0] = U[:, -1] = 0.0
    return h, np.ones(su), U, np.zeros(sv), np.zeros(sw)


def _energy(F, h):
    U, V, W = F
    return 0.5 * h * h * (np.sum(U[1:-1, 1:-1] ** 2) + np.sum(V ** 2) + np.sum(W ** 2))


@pytest.mark.parametrize("method", [CFD, MFD])
def test_no_damping_is_the_plain_step(method):
    rng = np.random.default_rng(3 + method)
    nx, ny = 20, 17
    su, sv, sw = wl.shapes(method, nx, ny)
    k = rng.uniform(0.5, 1.5, su)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    A = oracle.run(method, nx, ny, 0.05, 0.03, k, U, V, W, 3)
    for width, a in ((0.0, 0.3), (6.0, 0.0)):
        B = oracle.run_sponge(method, nx, ny, 0.05, 0.03, k, U, V, W, 3, width, a)
        for x, y in zip(A, B):
            np.testing.assert_array_equal(x, y)


def _g(x, y, nx, ny, width, a):
    """The damping factor at points (x, y) given in cells."""
    d = np.minimum(np.minimum(x, nx - x), np.minimum(y, ny - y))
    return np.where(d < width, np.exp(-(a * (width - d)) ** 2), 1.0)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_one_step_is_plain_step_times_profile(method):
    rng = np.random.default_rng(11 + method)
    nx, ny = 24, 19
    width, a = 5.5, 0.2
    su, sv, sw = wl.shapes(method, nx, ny)
    k = rng.uniform(0.5, 1.5, su)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    A = oracle.run(method, nx, ny, 0.05, 0.03, k, U, V, W, 1)
    B = oracle.run_sponge(method, nx, ny, 0.05, 0.03, k, U, V, W, 1, width, a)
    coords = wl.point_coords(method, nx, ny, 1.0)  # in cells
    for f, (x, y) in enumerate(coords):
        X, Y = np.meshgrid(x, y)
        g = _g(X, Y, nx, ny, width, a)
        want = A[f] * g
        if f == 0:  # the pressure's wall values are Dirichlet data, never damped
            want[0, :] = A[0][0, :]; want[-1, :] = A[0][-1, :]
            want[:, 0] = A[0][:, 0]; want[:, -1] = A[0][:, -1]
        np.testing.assert_allclose(B[f], want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_layers_absorb_the_pulse(method):
    N = 100
    h, k, U, V, W = _pulse(method, N)
    dt = 0.5 * h
    E0 = _energy((U, V, W), h)
    th = max(1, oracle.num_threads())
    for steps in (100, 200):
        P = oracle.run(method, N, N, h, dt, k, U, V, W, steps, threads=th)
        S = oracle.run_sponge(method, N, N, h, dt, k, U, V, W, steps, 20.0, 0.075, threads=th)
        assert 0.9 < _energy(P, h) / E0 < 1.1
        if steps == 200:
            assert _energy(S, h) / E0 < 0.01
            # the wave reflected by the walls, back at the centre
            assert abs(S[0][N // 2, N // 2]) * 50 < abs(P[0][N // 2, N // 2])


@pytest.mark.parametrize("method", [CFD, MFD])
def test_interior_unchanged_before_the_pulse_arrives(method):
    N = 100
    h, k, U, V, W = _pulse(method, N)
    P = oracle.run(method, N, N, h, 0.5 * h, k, U, V, W, 10)
    S = oracle.run_sponge(method, N, N, h, 0.5 * h, k, U, V, W, 10, 20.0, 0.075)
    for x, y in zip(P, S):
        assert np.max(np.abs(x - y)) < 1e-8 * np.max(np.abs(P[0]))
