"""Stability of the two schemes' exact PR step, measured on the oracle.

Finding (documented in the design notes): with the compact operators of App. A in the
first-order system of Eq. 4, the 1-D semi-discrete operator has eigenvalues with positive
real part (about 0.096/h), and the exact PR step's spectral radius exceeds 1 (about 1.07-1.11
on these grids), so rounding differences grow geometrically.  The mimetic pair of App. B
gives a purely imaginary spectrum and a PR step of spectral radius 1 (to roundoff).  These
pins fix both facts so that a change to either scheme's operators shows up here.
"""
import numpy as np
import pytest

import oracle
from oracle import CFD, MFD
from paper_2006_07583_gb300 import workloads as wl


def _semi_discrete(method, N):
    h = 1.0 / N
    if method == CFD:
        Dv = np.linalg.solve(oracle.operator("Pbar", N, h), oracle.operator("Qbar", N, h))
        Du = np.linalg.solve(oracle.operator("P", N, h), oracle.operator("Q", N, h))[:, 1:-1]
    else:
        Dv = oracle.operator("D", N, h)
        Du = oracle.operator("G", N, h)[:, 1:-1]
    n1, n2 = Dv.shape
    return np.block([[np.zeros((n1, n1)), -Dv], [-Du, np.zeros((n2, n2))]])


@pytest.mark.parametrize("N", [16, 64])
def test_semi_discrete_spectra(N):
    re_cfd = np.linalg.eigvals(_semi_discrete(CFD, N)).real.max() / N
    re_mfd = np.linalg.eigvals(_semi_discrete(MFD, N)).real.max() / N
    assert 0.09 < re_cfd < 0.14
    assert abs(re_mfd) < 1e-12


def _step_matrix(method, N, cfl):
    h = 1.0 / N
    dt = cfl * h
    su, sv, sw = wl.shapes(method, N, N)
    kap = np.ones(su)
    pi = N - 1 if method == CFD else N
    idx = [("U", i, j) for i in range(1, pi + 1) for j in range(1, pi + 1)]
    idx += [("V", i, j) for i in range(1, pi + 1) for j in range(sv[1])]
    idx += [("W", i, j) for i in range(sw[0]) for j in range(1, pi + 1)]
    M = np.zeros((len(idx), len(idx)))
    for k, (f, i, j) in enumerate(idx):
        F = {"U": np.zeros(su), "V": np.zeros(sv), "W": np.zeros(sw)}
        F[f][i, j] = 1.0
        U1, V1, W1 = oracle.run(method, N, N, h, dt, kap, F["U"], F["V"], F["W"], 1)
        R = {"U": U1, "V": V1, "W": W1}
        M[:, k] = [R[g][a, b] for (g, a, b) in idx]
    return M


def test_pr_step_spectral_radius():
    rho_cfd = np.abs(np.linalg.eigvals(_step_matrix(CFD, 16, 0.5))).max()
    rho_mfd = np.abs(np.linalg.eigvals(_step_matrix(MFD, 16, 0.81))).max()
    assert rho_cfd > 1.05
    assert abs(rho_mfd - 1.0) < 1e-10
