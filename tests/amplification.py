"""How far two correct implementations of the PR step may drift apart, measured on the oracle.

Two implementations that solve the same line systems in different elimination orders differ
by rounding at every step, and the scheme carries each step's difference forward like any
other perturbation.  The MFD step has spectral radius 1, so differences add up.  The CFD step
(App. A's boundary closure) has growing modes, about 6 % a step at dt = 0.5 h, so a difference
made at step k has grown by G(n - k) at step n.  The bound used by the long parity tests is

    bar(n) = e * sum_{j < n} G(j),

with G(j) the growth of a random perturbation over j steps of the oracle (max-abs norm for the
FP64 bar, L2 for the FP32 bar) and e the difference one step may add: 5e-15 of max |field| in
FP64 and 5e-7 relative L2 in FP32.  For the neutral MFD step over 200 steps this gives back the
short-run bars of the parity tests (1e-12 and 1e-4); for CFD it grows with the measured
amplification.
"""
from __future__ import annotations

import numpy as np

import oracle

E_FP64 = 5e-15   # per-step difference, relative to max |field|
E_FP32 = 5e-7    # per-step difference, relative L2


def growth(method, nx, ny, h, dt, kappa, U, V, W, nsteps, source=None, seed=1, rel=1e-9,
           threads=None):
    """(G_max, G_l2): arrays of nsteps + 1 growth factors of a random perturbation of relative
    size ``rel`` (interior values only; the Dirichlet edges stay as they are)."""
    threads = threads or max(1, oracle.num_threads())
    rng = np.random.default_rng(seed)
    A = [np.array(f, dtype=np.float64) for f in (U, V, W)]
    B = []
    for f in A:
        p = f + rel * max(np.max(np.abs(f)), 1e-30) * rng.standard_normal(f.shape)
        B.append(p)
    B[0][0, :] = A[0][0, :]; B[0][-1, :] = A[0][-1, :]
    B[0][:, 0] = A[0][:, 0]; B[0][:, -1] = A[0][:, -1]

    def dist(X, Y):
        return (max(np.max(np.abs(x - y)) for x, y in zip(X, Y)),
                np.sqrt(sum(np.linalg.norm(x - y) ** 2 for x, y in zip(X, Y))))

    m0, l0 = dist(A, B)
    gm, gl = [1.0], [1.0]
    for j in range(nsteps):
        A = list(oracle.run(method, nx, ny, h, dt, kappa, *A, 1, t0=j * dt, source=source,
                            threads=threads))
        B = list(oracle.run(method, nx, ny, h, dt, kappa, *B, 1, t0=j * dt, source=source,
                            threads=threads))
        m, l = dist(A, B)
        gm.append(m / m0)
        gl.append(l / l0)
    return np.array(gm), np.array(gl)


def bars(gm, gl, nsteps):
    """(FP64 max-relative bar, FP32 relative-L2 bar) after nsteps."""
    return E_FP64 * float(np.sum(gm[:nsteps])), E_FP32 * float(np.sum(gl[:nsteps]))
