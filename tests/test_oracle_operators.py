"""Pins of the oracle's 1-D operators (App. A and App. B) and of its line solver.

The operators are pinned by what the mathematics fixes, not by retyping coefficients:
every row of a fourth-order operator differentiates polynomials of degree <= 4 exactly and
fails on degree 5.  A wrong coefficient, a dropped 1/h, a wrong mirror sign or a shifted
column fails one of these checks.
"""
import numpy as np
import pytest

import oracle
from oracle import CFD, MFD


def _poly(k, x):
    return x ** k


def _dpoly(k, x):
    return k * x ** (k - 1) if k > 0 else np.zeros_like(x)


@pytest.mark.parametrize("N", [8, 16, 37])
def test_cfd_full_operator_exact_to_degree_4(N):
    h = 1.0 / N
    x = np.arange(N + 1) * h
    P, Q = oracle.operator("P", N, h), oracle.operator("Q", N, h)
    for k in range(5):
        res = P @ _dpoly(k, x) - Q @ _poly(k, x)
        assert np.max(np.abs(res)) < 1e-9 * max(1.0, k * N), (k, res)
    res5 = P @ _dpoly(5, x) - Q @ _poly(5, x)
    # the boundary closures are fourth order, not fifth
    assert np.max(np.abs(res5)) > 1e-6


@pytest.mark.parametrize("N", [8, 16, 37])
def test_cfd_reduced_operator_exact_to_degree_4(N):
    h = 1.0 / N
    x = np.arange(N + 1) * h
    Pb, Qb = oracle.operator("Pbar", N, h), oracle.operator("Qbar", N, h)
    assert Pb.shape == (N - 1, N - 1) and Qb.shape == (N - 1, N + 1)
    for k in range(5):
        res = Pb @ _dpoly(k, x[1:-1]) - Qb @ _poly(k, x)
        assert np.max(np.abs(res)) < 1e-9 * max(1.0, k * N), (k, res)
    res5 = Pb @ _dpoly(5, x[1:-1]) - Qb @ _poly(5, x)
    assert np.max(np.abs(res5)) > 1e-6


@pytest.mark.parametrize("N", [8, 16, 37])
def test_mimetic_divergence_exact_to_degree_4(N):
    h = 1.0 / N
    xn = np.arange(N + 1) * h
    xc = (np.arange(N) + 0.5) * h
    D = oracle.operator("D", N, h)
    for k in range(5):
        err = D @ _poly(k, xn) - _dpoly(k, xc)
        assert np.max(np.abs(err)) < 1e-9 * max(1.0, k * N), (k, err)
    err5 = D @ _poly(5, xn) - _dpoly(5, xc)
    assert np.max(np.abs(err5)) > 1e-8


@pytest.mark.parametrize("N", [8, 16, 37])
def test_mimetic_gradient_exact_to_degree_4(N):
    h = 1.0 / N
    xn = np.arange(N + 1) * h
    xcb = np.concatenate([[0.0], (np.arange(N) + 0.5) * h, [1.0]])
    G = oracle.operator("G", N, h)
    for k in range(5):
        err = G @ _poly(k, xcb) - _dpoly(k, xn)
        assert np.max(np.abs(err)) < 1e-9 * max(1.0, k * N), (k, err)
    err5 = G @ _poly(5, xcb) - _dpoly(5, xn)
    assert np.max(np.abs(err5)) > 1e-8


def test_operators_shift_invariant_interior_and_scale_with_h():
    # the same grid on [0, 2] (h doubled) must give exactly half the derivative weights
    N = 20
    for name in ("Q", "Qbar", "D", "G"):
        a = oracle.operator(name, N, 1.0 / N)
        b = oracle.operator(name, N, 2.0 / N)
        np.testing.assert_allclose(b, 0.5 * a, rtol=0, atol=1e-12)


def _random_line(method, N, rng):
    np_ = N - 1 if method == CFD else N
    alpha = rng.uniform(0.05, 0.6, np_) / N * 4
    beta = 0.4 / N
    a = rng.standard_normal(np_)
    vm = rng.standard_normal(N + 1)
    return alpha, beta, a, vm


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("N", [8, 13, 32])
def test_line_solve_banded_matches_dense_pivoted(method, N):
    rng = np.random.default_rng(10 + N + 100 * method)
    h = 1.0 / N
    alpha, beta, a, vm = _random_line(method, N, rng)
    ub0, ub1 = rng.standard_normal(2)
    u1, v1 = oracle.line_solve(method, N, h, alpha, beta, a, vm, ub0, ub1, dense=False)
    u2, v2 = oracle.line_solve(method, N, h, alpha, beta, a, vm, ub0, ub1, dense=True)
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v1, v2, rtol=0, atol=1e-12)


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("N", [8, 21, 64])
def test_line_solve_satisfies_definition(method, N):
    """The solution satisfies Eq. 8 written with dense operator inverses (numpy LAPACK):
    ubar + alpha .* (Dv v) = a  and  v + beta .* (Du [ub0, ubar, ub1]) = v^m."""
    rng = np.random.default_rng(7 * N + method)
    h = 1.0 / N
    alpha, beta, a, vm = _random_line(method, N, rng)
    ub0, ub1 = rng.standard_normal(2)
    ubar, v = oracle.line_solve(method, N, h, alpha, beta, a, vm, ub0, ub1)
    if method == CFD:
        Dv = np.linalg.solve(oracle.operator("Pbar", N, h), oracle.operator("Qbar", N, h))
        Du = np.linalg.solve(oracle.operator("P", N, h), oracle.operator("Q", N, h))
    else:
        Dv = oracle.operator("D", N, h)
        Du = oracle.operator("G", N, h)
    u_full = np.concatenate([[ub0], ubar, [ub1]])
    r1 = ubar + alpha * (Dv @ v) - a
    r2 = v + beta * (Du @ u_full) - vm
    assert np.max(np.abs(r1)) < 1e-11
    assert np.max(np.abs(r2)) < 1e-11
