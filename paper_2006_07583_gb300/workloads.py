"""Seeded synthetic inputs for the ADI engine and its oracle.

This module holds none of the scheme's arithmetic: it only builds grids' coordinates,
material fields, initial fields, source parameters and request streams.  Both the CUDA
path's tests/bench and the CPU oracle's tests draw their inputs from here, so that the two
sides see identical data while sharing no computation.

Workloads (all synthetic; the paper uses no dataset):
  * standing wave -- the exact solution of Eq. 11 with Gamma = 0, c = 1 and spatial period
    lambda = 2:  p = cos(sqrt(2) pi t) sin(pi x) sin(pi y), and the matching velocities
    v = -sin(sqrt(2) pi t) cos(pi x) sin(pi y)/sqrt(2), w likewise with x and y swapped.
  * layered medium -- horizontal layers of increasing wave speed times a smooth seeded
    Gaussian perturbation, a Ricker point source at the centre (the 15 Hz seismic case).
  * batch / serving mixes -- seeded lists of grid sizes, methods and step counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CFD = 0
MFD = 1
METHOD_NAMES = {CFD: "cfd", MFD: "mfd"}


def shapes(method: int, nx: int, ny: int):
    """(U, V, W) array shapes; kappa has U's shape.

    CFD (nodal mesh): all (ny+1) x (nx+1).
    MFD (staggered mesh): U (ny+2)x(nx+2) at cell centres plus edges, V (ny+2)x(nx+1) at
    x-nodes, W (ny+1)x(nx+2) at y-nodes.
    """
    if method == CFD:
        s = (ny + 1, nx + 1)
        return s, s, s
    return (ny + 2, nx + 2), (ny + 2, nx + 1), (ny + 1, nx + 2)


def nodes(n: int, h: float) -> np.ndarray:
    return np.arange(n + 1, dtype=np.float64) * h


def centres_and_edges(n: int, h: float) -> np.ndarray:
    """0, h/2, 3h/2, ..., (n-1/2)h, n h  (n+2 points)."""
    x = np.empty(n + 2, dtype=np.float64)
    x[0] = 0.0
    x[1:-1] = (np.arange(n, dtype=np.float64) + 0.5) * h
    x[-1] = n * h
    return x


def point_coords(method: int, nx: int, ny: int, h: float):
    """Coordinates (x, y) 1-D arrays for the U, V and W points."""
    if method == CFD:
        x, y = nodes(nx, h), nodes(ny, h)
        return (x, y), (x, y), (x, y)
    xc, yc = centres_and_edges(nx, h), centres_and_edges(ny, h)
    xn, yn = nodes(nx, h), nodes(ny, h)
    return (xc, yc), (xn, yc), (xc, yn)


def standing_wave(method: int, n: int, t: float):
    """Exact (U, V, W) of the unit-square standing wave at time t on an n x n grid."""
    h = 1.0 / n
    (ux, uy), (vx, vy), (wx, wy) = point_coords(method, n, n, h)
    om = math.sqrt(2.0) * math.pi
    U = math.cos(om * t) * np.outer(np.sin(math.pi * uy), np.sin(math.pi * ux))
    V = -math.sin(om * t) / math.sqrt(2.0) * np.outer(np.sin(math.pi * vy), np.cos(math.pi * vx))
    W = -math.sin(om * t) / math.sqrt(2.0) * np.outer(np.cos(math.pi * wy), np.sin(math.pi * wx))
    # Dirichlet data on the boundary: p = 0 exactly (sin(0) = sin(pi) = 0); clean roundoff.
    U[0, :] = 0.0; U[-1, :] = 0.0; U[:, 0] = 0.0; U[:, -1] = 0.0
    if method == MFD:
        pass  # corners of U are unused by the scheme; they are already 0 here.
    return U, V, W


@dataclass
class HarmonicProblem:
    """The exact solution of Sec. 4, Eq. 11 on the unit square (c = 1, rho = 1):

        u = Psi(x, y) cos(omega t),  Psi = Gamma (x^k - (1-x)^k + y^k - (1-y)^k)
                                          + sin(2 pi x / lam) sin(2 pi y / lam),

    omega = 2 pi / T, with the velocities that the momentum equation of Eq. 1 gives from
    v = w = 0 at t = 0, (v, w) = -(1/omega) grad Psi sin(omega t), and the forcing that makes
    the pressure equation exact, f = -sin(omega t) (omega Psi + (kappa/omega) Laplacian Psi).
    In the time-harmonic form of the ADI engine: walls u = B cos(omega t + phase_b) with
    B = Psi, forcing f = F cos(omega t + phase_f) with F = omega Psi + Laplacian Psi / omega
    and phase_f = pi/2."""
    method: int
    n: int
    gamma: float
    k: int
    lam: float
    period: float

    @property
    def omega(self) -> float:
        return 2.0 * math.pi / self.period

    def _psi(self, x, y):
        g, k, a = self.gamma, self.k, 2.0 * math.pi / self.lam
        X, Y = np.meshgrid(x, y)
        psi = g * (X ** k - (1 - X) ** k + Y ** k - (1 - Y) ** k) + np.sin(a * X) * np.sin(a * Y)
        px = g * k * (X ** (k - 1) + (1 - X) ** (k - 1)) + a * np.cos(a * X) * np.sin(a * Y)
        py = g * k * (Y ** (k - 1) + (1 - Y) ** (k - 1)) + a * np.sin(a * X) * np.cos(a * Y)
        lap = (g * k * (k - 1) * (X ** (k - 2) - (1 - X) ** (k - 2) + Y ** (k - 2) - (1 - Y) ** (k - 2))
               - 2.0 * a * a * np.sin(a * X) * np.sin(a * Y))
        return psi, px, py, lap

    def fields(self, t: float):
        """Exact (U, V, W) at time t."""
        h = 1.0 / self.n
        (ux, uy), (vx, vy), (wx, wy) = point_coords(self.method, self.n, self.n, h)
        om = self.omega
        U = self._psi(ux, uy)[0] * math.cos(om * t)
        V = -self._psi(vx, vy)[1] * math.sin(om * t) / om
        W = -self._psi(wx, wy)[2] * math.sin(om * t) / om
        return U, V, W

    def amplitudes(self):
        """(B, F, omega, phase_b, phase_f) for the engine's and the oracle's harmonic mode."""
        h = 1.0 / self.n
        (ux, uy), _, _ = point_coords(self.method, self.n, self.n, h)
        psi, _, _, lap = self._psi(ux, uy)
        om = self.omega
        return psi, om * psi + lap / om, om, 0.0, 0.5 * math.pi


def unit_kappa(method: int, nx: int, ny: int) -> np.ndarray:
    return np.ones(shapes(method, nx, ny)[0], dtype=np.float64)


def layered_c(method: int, nx: int, ny: int, h: float, speeds=(1500.0, 2500.0, 3500.0, 4500.0),
              pert: float = 0.1, sigma_frac: float = 0.1, seed: int = 1) -> np.ndarray:
    """Wave speed at the U points: equal horizontal layers with the given speeds from top
    (y = 0) to bottom, times (1 + pert * exp(-r^2 / (2 sigma^2))) around a centre drawn
    uniformly in the middle half of the domain; sigma = sigma_frac * min(Lx, Ly)."""
    rng = np.random.default_rng(seed)
    (ux, uy), _, _ = point_coords(method, nx, ny, h)
    Lx, Ly = nx * h, ny * h
    cx = rng.uniform(0.25 * Lx, 0.75 * Lx)
    cy = rng.uniform(0.25 * Ly, 0.75 * Ly)
    sigma = sigma_frac * min(Lx, Ly)
    nl = len(speeds)
    layer = np.minimum((uy / Ly * nl).astype(np.int64), nl - 1)
    c0 = np.asarray(speeds, dtype=np.float64)[layer][:, None] * np.ones((1, ux.size))
    r2 = (ux[None, :] - cx) ** 2 + (uy[:, None] - cy) ** 2
    return c0 * (1.0 + pert * np.exp(-r2 / (2.0 * sigma * sigma)))


def random_layer_speeds(rng: np.random.Generator, lo=1500.0, hi=4500.0):
    nl = int(rng.integers(3, 7))
    return tuple(np.sort(rng.uniform(lo, hi, size=nl)).tolist())


@dataclass
class Ricker:
    """Ricker wavelet s(t) = amp (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
    tau = t - tdelay, applied as a point source f = s/h^2 at U[is, js]."""
    is_: int
    js: int
    f0: float = 15.0
    amp: float = 1.0
    tdelay: float = 0.0

    def __post_init__(self):
        if self.tdelay == 0.0:
            self.tdelay = 1.2 / self.f0

    def as_tuple(self):
        return (self.is_, self.js, self.amp, self.f0, self.tdelay)


def centre_source(method: int, nx: int, ny: int, f0: float = 15.0, amp: float = 1.0) -> Ricker:
    if method == CFD:
        return Ricker(ny // 2, nx // 2, f0=f0, amp=amp)
    return Ricker(ny // 2 + 1, nx // 2 + 1, f0=f0, amp=amp)


def cfl_dt(method: int, h: float, cmax: float) -> float:
    """dt = cfl_max * h / c_max with cfl_max 0.91 (CFD) and 0.81 (MFD) (Sec. 4)."""
    return (0.91 if method == CFD else 0.81) * h / cmax


@dataclass
class SimSpec:
    method: int
    nx: int
    ny: int
    h: float
    dt: float
    steps: int
    c: np.ndarray = field(repr=False)
    source: Ricker | None = None
    U0: np.ndarray | None = field(default=None, repr=False)
    V0: np.ndarray | None = field(default=None, repr=False)
    W0: np.ndarray | None = field(default=None, repr=False)

    @property
    def points(self) -> int:
        return self.nx * self.ny


def seismic_spec(method: int, nx: int, ny: int, steps: int, h: float = 5.0, seed: int = 1,
                 speeds=(1500.0, 2500.0, 3500.0, 4500.0)) -> SimSpec:
    """Layered medium with a seeded Gaussian perturbation and a 15 Hz centre Ricker."""
    c = layered_c(method, nx, ny, h, speeds=speeds, seed=seed)
    dt = cfl_dt(method, h, float(c.max()))
    return SimSpec(method, nx, ny, h, dt, steps, c, centre_source(method, nx, ny))


def batch_specs(n_sims: int = 256, lo: int = 128, hi: int = 1024, steps: int = 500,
                seed: int = 2, h: float = 5.0):
    """Half CFD, half MFD; nx, ny i.i.d. uniform integers in [lo, hi]; seeded layered c."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_sims):
        method = CFD if k < n_sims // 2 else MFD
        nx = int(rng.integers(lo, hi + 1))
        ny = int(rng.integers(lo, hi + 1))
        speeds = random_layer_speeds(rng)
        out.append(seismic_spec(method, nx, ny, steps, h=h, seed=int(rng.integers(1 << 30)),
                                speeds=speeds))
    return out


@dataclass
class Request:
    arrival: float
    spec: SimSpec


def serving_stream(n_requests: int, rate: float, seed: int = 3, lo: int = 64, hi: int = 4096,
                   steps_lo: int = 100, steps_hi: int = 5000, h: float = 5.0,
                   lazy_c: bool = True):
    """Poisson arrivals with rate ``rate`` (requests/s); square grids with side log-uniform in
    [lo, hi]; steps uniform in [steps_lo, steps_hi]; method CFD/MFD with probability 1/2."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        method = int(rng.integers(0, 2))
        speeds = random_layer_speeds(rng)
        sub_seed = int(rng.integers(1 << 30))
        out.append(Request(t, seismic_spec(method, n, n, steps, h=h, seed=sub_seed,
                                           speeds=speeds)))
    return out
