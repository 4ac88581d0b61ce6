"""Pins of the oracle's whole Peaceman-Rachford step.

* Kronecker: on tiny grids the step equals the dense 2-D PR step built from Kronecker
  products of the (separately pinned) 1-D operators -- Eqs. 4/12 and 6-7 written as dense
  matrices and solved with LAPACK.  This pins the line decomposition, index sets, material
  scaling, source time levels and boundary handling.
* Time reversal: J S J = S^{-1} with J = diag(1, -1, -1) on (u, v, w).
* Mirror symmetry under x -> L - x.
* The exact standing wave: small error and a convergence rate near 4 with dt ~ h^2.
* The paper's fixed-point iteration (Eq. 9) converges to the exact line solve.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import CFD, MFD
from paper_2006_07583_gb300 import workloads as wl


def _dv_du(method, N, h):
    if method == CFD:
        Dv = np.linalg.solve(oracle.operator("Pbar", N, h), oracle.operator("Qbar", N, h))
        Du = np.linalg.solve(oracle.operator("P", N, h), oracle.operator("Q", N, h))
    else:
        Dv = oracle.operator("D", N, h)
        Du = oracle.operator("G", N, h)
    return Dv, Du[:, 1:-1]  # Du restricted to interior pressure (homogeneous Dirichlet)


def _kron_step(method, nx, ny, h, dt, kappa, U, V, W, t, src=None):
    """Dense 2-D PR step on the state (ubar, Vbar, Wbar) with u = 0 on the boundary."""
    Dvx, Dux = _dv_du(method, nx, h)
    Dvy, Duy = _dv_du(method, ny, h)
    pix, piy = Dvx.shape[0], Dvy.shape[0]   # interior pressure counts
    nvx, nvy = Dvx.shape[1], Dvy.shape[1]   # velocity points per line
    Ix, Iy = np.eye(pix), np.eye(piy)
    K = np.diag(kappa[1:piy + 1, 1:pix + 1].ravel())
    # state blocks: ubar (piy, pix), Vbar (piy, nvx) = V rows 1..piy, Wbar (nvy, pix)
    nu, nvv, nww = piy * pix, piy * nvx, nvy * pix
    n = nu + nvv + nww
    A1 = np.zeros((n, n)); A2 = np.zeros((n, n))
    su, sv, sw = slice(0, nu), slice(nu, nu + nvv), slice(nu + nvv, n)
    A1[su, sv] = -K @ np.kron(Iy, Dvx)
    A1[sv, su] = -np.kron(Iy, Dux)          # rho = 1
    A2[su, sw] = -K @ np.kron(Dvy, Ix)
    A2[sw, su] = -np.kron(Duy, Ix)
    x = np.concatenate([U[1:piy + 1, 1:pix + 1].ravel(), V[1:piy + 1, :].ravel(),
                        W[:, 1:pix + 1].ravel()])
    F0 = np.zeros(n); F1 = np.zeros(n)
    if src is not None:
        is_, js, amp, f0, td = src
        def ricker(tt):
            q = (math.pi * f0 * (tt - td)) ** 2
            return amp * (1 - 2 * q) * math.exp(-q)
        k = (is_ - 1) * pix + (js - 1)
        F0[k] = ricker(t) / h ** 2
        F1[k] = ricker(t + dt) / h ** 2
    I = np.eye(n)
    tau = 0.5 * dt
    xs = np.linalg.solve(I - tau * A1, (I + tau * A2) @ x + tau * F0)
    x1 = np.linalg.solve(I - tau * A2, (I + tau * A1) @ xs + tau * F1)
    U1, V1, W1 = U.copy(), V.copy(), W.copy()
    U1[1:piy + 1, 1:pix + 1] = x1[su].reshape(piy, pix)
    V1[1:piy + 1, :] = x1[sv].reshape(piy, nvx)
    W1[:, 1:pix + 1] = x1[sw].reshape(nvy, pix)
    return U1, V1, W1


def _random_state(method, nx, ny, rng, scale_k=1.0):
    su, sv, sw = wl.shapes(method, nx, ny)
    kappa = rng.uniform(0.5, 1.5, su) * scale_k
    U = rng.standard_normal(su)
    U[0, :] = U[-1, :] = 0.0; U[:, 0] = U[:, -1] = 0.0
    V = rng.standard_normal(sv)
    W = rng.standard_normal(sw)
    return kappa, U, V, W


@pytest.mark.parametrize("method", [CFD, MFD])
@pytest.mark.parametrize("use_src", [False, True])
def test_step_matches_dense_kronecker(method, use_src):
    rng = np.random.default_rng(3 + method + 10 * use_src)
    nx, ny = 9, 8
    h = 1.0 / 9
    dt = 0.7 * h
    kappa, U, V, W = _random_state(method, nx, ny, rng)
    src = (4, 5, 1.3, 2.0, 0.1) if use_src else None
    t0 = 0.05
    Uo, Vo, Wo = U, V, W
    Uk, Vk, Wk = U, V, W
    for m in range(2):
        Uo, Vo, Wo = oracle.run(method, nx, ny, h, dt, kappa, Uo, Vo, Wo, 1, t0=t0 + m * dt,
                                source=src)
        Uk, Vk, Wk = _kron_step(method, nx, ny, h, dt, kappa, Uk, Vk, Wk, t0 + m * dt, src)
    np.testing.assert_allclose(Uo, Uk, rtol=0, atol=1e-11)
    np.testing.assert_allclose(Vo, Vk, rtol=0, atol=1e-11)
    np.testing.assert_allclose(Wo, Wk, rtol=0, atol=1e-11)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_time_reversal(method):
    rng = np.random.default_rng(21 + method)
    nx, ny = 12, 10
    h = 0.1
    dt = 1.3 * h
    kappa, U, V, W = _random_state(method, nx, ny, rng)
    n = 5
    U1, V1, W1 = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, n)
    U2, V2, W2 = oracle.run(method, nx, ny, h, dt, kappa, U1, -V1, -W1, n)
    np.testing.assert_allclose(U2, U, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-V2, V, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-W2, W, rtol=0, atol=1e-11)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_mirror_symmetry(method):
    """x -> L - x maps a solution to a solution with v -> -v (the operators' mirrored rows)."""
    rng = np.random.default_rng(5 + method)
    nx, ny = 14, 11
    h = 1.0 / 14
    dt = 0.8 * h
    kappa, U, V, W = _random_state(method, nx, ny, rng)
    Um, Vm, Wm, km = U[:, ::-1].copy(), -V[:, ::-1].copy(), W[:, ::-1].copy(), kappa[:, ::-1].copy()
    A = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 3)
    B = oracle.run(method, nx, ny, h, dt, km, Um, Vm, Wm, 3)
    np.testing.assert_allclose(B[0], A[0][:, ::-1], rtol=0, atol=1e-11)
    np.testing.assert_allclose(B[1], -A[1][:, ::-1], rtol=0, atol=1e-11)
    np.testing.assert_allclose(B[2], A[2][:, ::-1], rtol=0, atol=1e-11)


def _standing_wave_error(method, N, dt, T):
    steps = int(round(T / dt))
    U0, V0, W0 = wl.standing_wave(method, N, 0.0)
    kappa = wl.unit_kappa(method, N, N)
    U, V, W = oracle.run(method, N, N, 1.0 / N, dt, kappa, U0, V0, W0, steps)
    Ue, _, _ = wl.standing_wave(method, N, steps * dt)
    return (1.0 / N) * np.linalg.norm(U - Ue), np.max(np.abs(U - Ue))


@pytest.mark.parametrize("method", [CFD, MFD])
def test_standing_wave_convergence_rate_near_4(method):
    """dt = 32 h^2 (so dt ~ h^2) on N = 16, 32, 64 to T = 0.25: both the spatial error and
    the second-order time error scale as h^4."""
    Ns = [16, 32, 64]
    errs = [_standing_wave_error(method, N, 32.0 / N ** 2, 0.25)[0] for N in Ns]
    r = oracle.rates(errs, Ns)
    assert all(3.6 < x < 4.6 for x in r), (errs, r)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_standing_wave_accuracy_config_grid(method):
    """101x101 nodal grid / 100x100 cells, c = 1, dt = 0.5 h, 200 steps (t = 1).

    The trapezoidal (Crank-Nicolson) phase error of the mode omega = sqrt(2) pi is
    (omega dt)^3 / 12 per step, 1.8e-4 after 200 steps; the fourth-order spatial error is
    two orders smaller.  Both schemes must stay inside that bound (and well above roundoff).
    """
    N = 100
    dt = 0.5 / N
    e_fro, e_max = _standing_wave_error(method, N, dt, 200 * dt)
    bound = (math.sqrt(2) * math.pi * dt) ** 3 / 12 * 200
    assert 1e-6 < e_max < 1.2 * bound, (e_max, bound)


@pytest.mark.parametrize("method", [CFD, MFD])
def test_paper_iteration_converges_to_exact_solve(method):
    rng = np.random.default_rng(9 + method)
    nx, ny = 12, 12
    h = 1.0 / 12
    dt = 0.3 * h
    kappa, U, V, W = _random_state(method, nx, ny, rng)
    Ex = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 2)
    It = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 2, kmax=400, eps=1e-14)
    Ik = oracle.run(method, nx, ny, h, dt, kappa, U, V, W, 2, kmax=2, eps=0.0)
    for a, b in zip(Ex, It):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-11)
    d2 = max(np.max(np.abs(a - b)) for a, b in zip(Ex, Ik))
    assert d2 > 1e-8  # two sweeps are visibly short of the fixed point
