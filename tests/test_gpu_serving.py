"""The serving loop (adi_server_*): requests of different methods, sizes and step counts
arriving while others run are admitted by the HBM budget, advance together as one batch, and
each gives the same result as the same simulation run alone.

FP32 results equal the alone run bit for bit: every line takes the same arithmetic whatever
else shares its launch, and writing the natural fields at the end of a scheduling quantum does
not change the carried values.
"""
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


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        method = wl.CFD if k % 2 == 0 else wl.MFD
        nx, ny = int(rng.integers(48, 200)), int(rng.integers(48, 200))
        steps = int(rng.integers(5, 60))
        spec = wl.seismic_spec(method, nx, ny, steps, h=5.0, seed=int(rng.integers(1 << 30)),
                               speeds=wl.random_layer_speeds(rng))
        out.append(spec)
    return out


def _alone(adi, sp):
    s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP32)
    s.set_source(*sp.source.as_tuple())
    s.step(sp.steps)
    r = s.read()
    s.close()
    return r


def test_each_result_same_alone_and_in_the_mix(adi):
    specs = _requests(10, seed=31)
    sizes = [adi.server_bytes(sp.method, sp.nx, sp.ny) for sp in specs]
    budget = int(2.5 * max(sizes))  # at most two or three resident at once: requests queue
    srv = adi.Server(budget, quantum=7, max_active=8)
    tickets, submitted = [], 0
    max_running, max_used = 0, 0
    # arrivals: three now, then one more after every scheduling round
    for sp in specs[:3]:
        tickets.append(srv.submit(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, sp.steps,
                                  source=sp.source.as_tuple()))
    submitted = 3
    for _ in range(10000):
        running, pending = srv.tick()
        max_running = max(max_running, running)
        max_used = max(max_used, srv.used_bytes())
        assert srv.used_bytes() <= budget
        if submitted < len(specs):
            sp = specs[submitted]
            tickets.append(srv.submit(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, sp.steps,
                                      source=sp.source.as_tuple()))
            submitted += 1
        elif running == 0 and pending == 0:
            break
    assert max_running >= 2  # work of several requests overlapped on the device
    for t, sp in zip(tickets, specs):
        state, ts, t0, t1 = srv.status(t)
        assert state == adi.ADI_REQ_DONE and 0 <= ts <= t0 <= t1
        got = srv.result(t)
        ref = _alone(adi, sp)
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
        assert np.max(np.abs(ref[0])) > 0  # the source has reached the field
    srv.close()


def test_requests_that_can_never_fit_or_are_invalid_are_rejected(adi):
    sp = wl.seismic_spec(wl.MFD, 64, 64, 5, h=5.0, seed=3)
    srv = adi.Server(adi.server_bytes(sp.method, 64, 64) - 1, quantum=5, max_active=2)
    with pytest.raises(adi.AdiError) as e:
        srv.submit(sp.method, 64, 64, sp.h, sp.dt, sp.c, 5)
    assert e.value.code == 2  # ADI_ENOMEM
    with pytest.raises(adi.AdiError) as e:
        srv.submit(sp.method, 64, 64, sp.h, sp.dt, sp.c, -1)
    assert e.value.code == 1  # ADI_EINVAL
    srv.close()


def test_zero_step_request_returns_its_initial_fields(adi):
    sp = wl.seismic_spec(wl.CFD, 40, 33, 0, h=5.0, seed=4)
    rng = np.random.default_rng(5)
    su, sv, sw = wl.shapes(sp.method, sp.nx, sp.ny)
    U, V, W = rng.standard_normal(su), rng.standard_normal(sv), rng.standard_normal(sw)
    srv = adi.Server(1 << 30, quantum=3, max_active=2)
    t = srv.submit(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, 0, U, V, W)
    srv.tick()
    assert srv.status(t)[0] == adi.ADI_REQ_DONE
    got = srv.result(t)
    for g, r in zip(got, (U, V, W)):
        assert np.max(np.abs(g - r.astype(np.float32))) <= 1e-6 * np.max(np.abs(r))
    srv.close()
