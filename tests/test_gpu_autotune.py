"""The solver autotuner (adi_autotune): it times every solver a configuration supports on the
simulation's own state, keeps the fastest, and leaves the fields exactly as they were; the
choice is cached per configuration."""
import numpy as np
import pytest

from paper_2006_07583_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adi():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_07583_gb300 import adi as _adi

    _adi.lib()
    return _adi


def _sim(adi, sp, prec):
    s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=prec)
    s.set_source(*sp.source.as_tuple())
    return s


@pytest.mark.parametrize("method,prec", [(wl.CFD, 0), (wl.MFD, 0), (wl.MFD, 1)])
def test_autotune_picks_fastest_and_restores_state(adi, method, prec):
    sp = wl.seismic_spec(method, 300, 220, 40, h=5.0, seed=11 + method)
    s = _sim(adi, sp, prec)
    s.step(7)  # odd: the tuner must restore the parity too
    before = s.read()
    chosen, ms = s.autotune(trials=2, force=True)
    after = s.read()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert chosen in ms and ms[chosen] == min(ms.values())
    assert adi.ADI_SOLVER_LINE in ms and len(ms) >= 2  # thread-per-line plus a chunked solver
    assert s.solver == chosen
    # stepping on is the same as an untuned simulation switched to the chosen solver
    s.step(9)
    got = s.read()
    ref = _sim(adi, sp, prec)
    ref.step(7)
    ref.set_solver(chosen)
    ref.step(9)
    want = ref.read()
    for g, r in zip(got, want):
        assert np.max(np.abs(g - r)) <= 1e-6 * max(np.max(np.abs(r)), 1e-30)
    # cached: the same configuration takes the stored choice without timing again
    s2 = _sim(adi, sp, prec)
    chosen2, ms2 = s2.autotune(trials=2, force=False)
    assert chosen2 == chosen and ms2 == ms and s2.solver == chosen
    for x in (s, ref, s2):
        x.close()


def test_autotune_rejects_bad_arguments(adi):
    sp = wl.seismic_spec(wl.CFD, 64, 64, 5, h=5.0, seed=3)
    s = _sim(adi, sp, 0)
    with pytest.raises(adi.AdiError):
        s.autotune(trials=0)
    with pytest.raises(adi.AdiError):
        s.set_launch(0, 4)  # at most three groups in flight
    s.close()


# (CFD, 4096, 48) in FP32: its 4096-cell x-lines are the ones whose stage fits three times
@pytest.mark.parametrize("method,nx,ny,prec", [(wl.CFD, 300, 220, 0), (wl.MFD, 260, 197, 0),
                                               (wl.CFD, 130, 700, 1), (wl.MFD, 1024, 128, 0),
                                               (wl.CFD, 4096, 48, 0)])
def test_launch_parameters_leave_results_unchanged(adi, method, nx, ny, prec):
    """Every lines-per-CTA cap and ring depth of the factored solver gives the same numbers as
    the automatic launch: each line is solved by the same arithmetic whatever its group."""
    sp = wl.seismic_spec(method, nx, ny, 6, h=5.0, seed=31 + nx)
    ref = _sim(adi, sp, prec)
    assert ref.solver == adi.ADI_SOLVER_FACTORED
    ref.step(6)
    want = ref.read()
    ref.close()
    for cap in (1, 2, 3, 7):
        for ring in (1, 2, 3):
            s = _sim(adi, sp, prec)
            s.set_launch(cap, ring)
            assert s.launch() == (cap, ring)
            s.step(6)
            for g, w in zip(s.read(), want):
                assert np.array_equal(g, w)
            s.close()


def test_autotune_chooses_launch_parameters(adi):
    """On short lines (many per CTA) the tuner times the factored solver's launch parameters too;
    the chosen ones are reported and the fields stay exactly as they were."""
    sp = wl.seismic_spec(wl.MFD, 256, 256, 10, h=5.0, seed=77)
    s = _sim(adi, sp, 0)
    s.step(3)
    before = s.read()
    chosen, ms = s.autotune(trials=4, force=True)
    for a, b in zip(before, s.read()):
        assert np.array_equal(a, b)
    cap, ring = s.launch()
    if chosen == adi.ADI_SOLVER_FACTORED:
        assert cap >= 0 and ring in (0, 1, 2)
    else:
        assert (cap, ring) == (0, 0)
    s.close()
