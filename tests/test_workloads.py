"""The seeded input generators (CPU): shapes, determinism, the time-step rule, the source and
the batch / serving mixes follow the stated recipes."""
import math

import numpy as np

from paper_2006_07583_gb300 import workloads as wl


def test_shapes():
    assert wl.shapes(wl.CFD, 10, 7) == ((8, 11), (8, 11), (8, 11))
    assert wl.shapes(wl.MFD, 10, 7) == ((9, 12), (9, 11), (8, 12))


def test_seismic_spec_is_seeded_and_follows_the_cfl_rule():
    a = wl.seismic_spec(wl.MFD, 64, 48, 10, h=5.0, seed=3)
    b = wl.seismic_spec(wl.MFD, 64, 48, 10, h=5.0, seed=3)
    c = wl.seismic_spec(wl.MFD, 64, 48, 10, h=5.0, seed=4)
    assert np.array_equal(a.c, b.c) and not np.array_equal(a.c, c.c)
    assert a.c.shape == wl.shapes(wl.MFD, 64, 48)[0] and np.all(a.c > 0)
    assert math.isclose(a.dt, 0.81 * 5.0 / a.c.max())
    cf = wl.seismic_spec(wl.CFD, 64, 48, 10, h=5.0, seed=3)
    assert math.isclose(cf.dt, 0.91 * 5.0 / cf.c.max())
    # speeds stay within the layers' range times the 10 % perturbation
    assert 1500.0 * 0.999 <= a.c.min() and a.c.max() <= 4500.0 * 1.1 + 1e-9


def test_centre_ricker():
    s = wl.centre_source(wl.CFD, 40, 30)
    assert (s.is_, s.js) == (15, 20) and math.isclose(s.tdelay, 1.2 / 15.0) and s.f0 == 15.0
    m = wl.centre_source(wl.MFD, 40, 30)
    assert (m.is_, m.js) == (16, 21)


def test_batch_mix():
    specs = wl.batch_specs(20, 128, 1024, 500, seed=2)
    assert [s.method for s in specs] == [wl.CFD] * 10 + [wl.MFD] * 10
    assert all(128 <= s.nx <= 1024 and 128 <= s.ny <= 1024 and s.steps == 500 for s in specs)
    again = wl.batch_specs(20, 128, 1024, 500, seed=2)
    assert [(s.nx, s.ny) for s in specs] == [(s.nx, s.ny) for s in again]


def test_serving_stream():
    reqs = wl.serving_stream(30, rate=50.0, seed=3, lo=64, hi=1024, steps_lo=100, steps_hi=1000)
    t = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert all(64 <= r.spec.nx <= 1024 and r.spec.nx == r.spec.ny for r in reqs)
    assert all(100 <= r.spec.steps <= 1000 for r in reqs)
    assert {r.spec.method for r in reqs} == {wl.CFD, wl.MFD}


def test_standing_wave_matches_its_formula():
    U, V, W = wl.standing_wave(wl.CFD, 16, 0.3)
    x = np.arange(17) / 16.0
    want = math.cos(math.sqrt(2) * math.pi * 0.3) * np.outer(np.sin(math.pi * x), np.sin(math.pi * x))
    assert np.allclose(U, want, atol=1e-14)
