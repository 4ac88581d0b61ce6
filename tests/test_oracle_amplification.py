"""The amplification behind the long-run parity bars (tests/amplification.py), on the
standing-wave configuration (100 x 100 cells, c = 1, dt = 0.5 h, 200 steps).

* MFD: a perturbation neither grows nor decays (spectral radius 1), so the 200-step bars are
  the short-run parity bars, 1e-12 (FP64) and 1e-4 (FP32).
* CFD: a random perturbation grows by 1e4 - 1e6 over 200 steps (about 6 % a step in L2,
  the growing modes of App. A's closure), so the bars at 200 steps are that many times wider.
"""
import numpy as np
import pytest

from amplification import bars, growth
from oracle import CFD, MFD
from paper_2006_07583_gb300 import workloads as wl


@pytest.fixture(scope="module")
def curves():
    out = {}
    N = 100
    for m in (CFD, MFD):
        U, V, W = wl.standing_wave(m, N, 0.0)
        out[m] = growth(m, N, N, 1.0 / N, 0.5 / N, wl.unit_kappa(m, N, N), U, V, W, 200)
    return out


def test_mfd_is_neutral(curves):
    gm, gl = curves[MFD]
    assert np.all(gl < 1.2) and np.all(gl > 0.8)
    b64, b32 = bars(gm, gl, 200)
    assert 0.8e-12 < b64 < 1.5e-12
    assert 0.8e-4 < b32 < 1.2e-4


def test_cfd_grows_about_six_percent_a_step(curves):
    gm, gl = curves[CFD]
    rate = (gl[200] / gl[100]) ** (1.0 / 100)
    assert 1.04 < rate < 1.08, rate
    b64, b32 = bars(gm, gl, 200)
    assert 1e-9 < b64 < 1e-7, b64
    b64_50, b32_50 = bars(gm, gl, 50)
    assert b64_50 < 2e-11 and b32_50 < 2e-3
