"""Pins of the oracle's fixed-point mode (Eq. 9 and Eq. 10's iterations; App. C, Algorithms 3-4).

The k -> infinity limit (tests/test_oracle_step.py) fixes only the fixed point.  These tests fix
what that limit cannot: the order of the updates inside a sweep and the stopping rule.

The restatement below is written from App. C with NumPy matrix algebra on the whole grid, from
the 1-D operator matrices that tests/test_oracle_operators.py pins on their own (exactness on
polynomials, App. A/B coefficients):

* stage 1 (ADI-rows): U_{k+1} = A - dt/2 K .* (V_k Dv_x^T) on the interior, then
  V_{k+1} = V^m - dt/2 (U_{k+1} Du_x^T) on the interior rows, using the U just computed
  (Gauss-Seidel order); V_0 = V^m;
* stage 2 (ADI-columns): U_{k+1} = C - dt/2 K .* (Dv_y W_k), then W_{k+1} = W* - dt/2 Du_y U_{k+1};
  W_0 = W^m (Eq. 10);
* each stage stops after the first sweep whose ||U_{k+1} - U_k||_F + ||V_{k+1} - V_k||_F (W for
  stage 2) is <= eps, or after kmax sweeps.

Dv = Pbar^{-1} Qbar, Du = P^{-1} Q (CFD) and Dv = D4, Du = G4 (MFD).  Du acts on the whole line
including its Dirichlet values.
"""
import numpy as np
import pytest

import oracle
from oracle import CFD, MFD
from paper_2006_07583_gb300 import workloads as wl


def _ops(method, N, h):
    if method == CFD:
        Dv = np.linalg.solve(oracle.operator("Pbar", N, h), oracle.operator("Qbar", N, h))
        Du = np.linalg.solve(oracle.operator("P", N, h), oracle.operator("Q", N, h))
    else:
        Dv = oracle.operator("D", N, h)
        Du = oracle.operator("G", N, h)
    return Dv, Du


def _paper_step(method, nx, ny, h, dt, kappa, U, V, W, kmax, eps):
    """One PR step with App. C's fixed-point sweeps.  Returns the new fields, and per stage
    the list of test values (one per sweep taken)."""
    Dvx, Dux = _ops(method, nx, h)
    Dvy, Duy = _ops(method, ny, h)
    pix, piy = Dvx.shape[0], Dvy.shape[0]
    I, J = slice(1, piy + 1), slice(1, pix + 1)  # interior rows / columns of U
    beta = 0.5 * dt
    al = 0.5 * dt * kappa[I, J]

    # stage 1 right-hand sides (explicit in y): W* on the interior columns, A on the interior
    Ws = W.copy()
    Ws[:, J] = W[:, J] - beta * (Duy @ U[:, J])
    A = U[I, J] - al * (Dvy @ W[:, J])

    def sweeps(update, start, kmax, eps):
        cur = start
        tests = []
        while True:
            new = update(cur)
            tests.append(sum(np.linalg.norm(n - c) for n, c in zip(new, cur)))
            cur = new
            if tests[-1] <= eps or len(tests) >= kmax:
                return cur, tests

    # stage 1: ADI-rows, Gauss-Seidel order
    def rows(state):
        Uk, Vk = state
        Un = Uk.copy()
        Un[I, J] = A - al * (Vk[I, :] @ Dvx.T)
        Vn = Vk.copy()
        Vn[I, :] = V[I, :] - beta * (Un[I, :] @ Dux.T)
        return Un, Vn

    (Us, Vs), t1 = sweeps(rows, (U.copy(), V.copy()), kmax, eps)

    # stage 2 right-hand sides (explicit in x)
    Vn = Vs.copy()
    Vn[I, :] = Vs[I, :] - beta * (Us[I, :] @ Dux.T)
    C = Us[I, J] - al * (Vs[I, :] @ Dvx.T)

    # stage 2: ADI-columns, starting from W^m
    def cols(state):
        Uk, Wk = state
        Un = Uk.copy()
        Un[I, J] = C - al * (Dvy @ Wk[:, J])
        Wn = Wk.copy()
        Wn[:, J] = Ws[:, J] - beta * (Duy @ Un[:, J])
        return Un, Wn

    (Un, Wn), t2 = sweeps(cols, (Us.copy(), W.copy()), kmax, eps)
    return (Un, Vn, Wn), (t1, t2)


def _state(method, nx, ny, seed):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    kappa = rng.uniform(0.5, 1.5, su)
    U = rng.standard_normal(su)
    # nonzero Dirichlet edges, so that the whole-line derivatives see them
    V = rng.standard_normal(sv)
    W = rng.standard_normal(sw)
    return kappa, U, V, W


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("kmax", [1, 2, 3])
def test_sweeps_follow_gauss_seidel_order(method, kmax):
    """kmax sweeps per stage equal App. C's sweeps element by element.  A Jacobi-order sweep
    (V_{k+1} from U_k) or a stage 2 started from W* instead of W^m differs after one sweep."""
    nx, ny = 13, 11
    h = 1.0 / 13
    dt = 0.6 * h
    kappa, U, V, W = _state(method, nx, ny, 40 + method)
    O = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 1, kmax=kmax, eps=0.0)
    P, _ = _paper_step(method, nx, ny, h, dt, kappa, U, V, W, kmax, 0.0)
    for o, p in zip(O, P):
        np.testing.assert_allclose(o, p, rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(p))))


@pytest.mark.parametrize("method", [CFD, MFD])
def test_two_steps_of_two_sweeps(method):
    """The sweeps carry over from step to step (the second step starts from the first's
    iterated fields)."""
    nx, ny = 10, 12
    h = 0.1
    dt = 0.5 * h
    kappa, U, V, W = _state(method, nx, ny, 50 + method)
    O = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 2, kmax=2, eps=0.0)
    P = (U, V, W)
    for _ in range(2):
        P, _ = _paper_step(method, nx, ny, h, dt, kappa, *P, 2, 0.0)
    for o, p in zip(O, P):
        np.testing.assert_allclose(o, p, rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(p))))


@pytest.mark.parametrize("method", [CFD, MFD])
def test_stopping_rule_counts_sweeps(method):
    """eps placed between the second and third sweeps' test values stops each stage after the
    sweep App. C's rule names; the reported sweep counts and the fields agree with it."""
    nx, ny = 12, 12
    h = 1.0 / 12
    dt = 0.5 * h
    kappa, U, V, W = _state(method, nx, ny, 60 + method)
    _, (t1, t2) = _paper_step(method, nx, ny, h, dt, kappa, U, V, W, 12, 0.0)
    assert t1[2] < t1[1] and t2[2] < t2[1]  # the iteration contracts on this state
    eps = np.sqrt(t1[1] * t1[2])             # strictly between stage 1's 2nd and 3rd values

    def first_below(tests, e):
        for k, t in enumerate(tests):
            if t <= e:
                return k + 1
        return len(tests)

    want = (first_below(t1, eps), first_below(t2, eps))
    assert want[0] == 3
    O = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 1, kmax=12, eps=eps, return_sweeps=True)
    assert tuple(int(x) for x in O[3][0]) == want
    P, _ = _paper_step(method, nx, ny, h, dt, kappa, U, V, W, 12, eps)
    for o, p in zip(O[:3], P):
        np.testing.assert_allclose(o, p, rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(p))))


@pytest.mark.parametrize("method", [CFD, MFD])
def test_stopping_rule_uses_both_norms(method):
    """An eps between the pressure update's norm alone and the full test value (pressure plus
    velocity) keeps iterating: the velocity norm is part of the test."""
    nx, ny = 12, 12
    h = 1.0 / 12
    dt = 0.5 * h
    kappa, U, V, W = _state(method, nx, ny, 70 + method)
    # split stage 1's second-sweep test value into its two terms
    _, (t1, _) = _paper_step(method, nx, ny, h, dt, kappa, U, V, W, 12, 0.0)
    (U1, V1, _), _ = _paper_step_stage1_only(method, nx, ny, h, dt, kappa, U, V, W, 1)
    (U2, V2, _), _ = _paper_step_stage1_only(method, nx, ny, h, dt, kappa, U, V, W, 2)
    du, dv = np.linalg.norm(U2 - U1), np.linalg.norm(V2 - V1)
    assert abs(du + dv - t1[1]) <= 1e-9 * t1[1]
    assert dv > 0.05 * du  # the velocity term is not negligible here
    eps = du + 0.5 * dv     # pressure alone would stop after sweep 2, the full test does not
    O = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 1, kmax=12, eps=eps, return_sweeps=True)
    assert int(O[3][0][0]) > 2


def _paper_step_stage1_only(method, nx, ny, h, dt, kappa, U, V, W, k):
    """Stage 1's fields after exactly k sweeps (read back from the step with kmax = k)."""
    Dvx, Dux = _ops(method, nx, h)
    Dvy, Duy = _ops(method, ny, h)
    pix, piy = Dvx.shape[0], Dvy.shape[0]
    I, J = slice(1, piy + 1), slice(1, pix + 1)
    beta = 0.5 * dt
    al = 0.5 * dt * kappa[I, J]
    A = U[I, J] - al * (Dvy @ W[:, J])
    Uk, Vk = U.copy(), V.copy()
    for _ in range(k):
        Un = Uk.copy()
        Un[I, J] = A - al * (Vk[I, :] @ Dvx.T)
        Vn = Vk.copy()
        Vn[I, :] = V[I, :] - beta * (Un[I, :] @ Dux.T)
        Uk, Vk = Un, Vn
    return (Uk, Vk, None), None


def test_exact_mode_reports_no_sweeps():
    kappa, U, V, W = _state(CFD, 10, 10, 80)
    O = oracle.run(CFD, 10, 10, 0.1, 0.05, kappa, U, V, W, 2, return_sweeps=True)
    assert O[3].shape == (2, 2) and not O[3].any()
