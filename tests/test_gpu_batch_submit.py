"""Asynchronous batches with per-simulation step counts (adi_batch_submit / adi_batch_poll):
each member advances by its own count, the result equals the same simulation stepped alone
bit for bit (the same arithmetic on the same lines, whatever the phases and the other members),
members are busy until the ticket is retired, and a retired or unknown ticket is rejected."""
import time

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


def _specs(seed):
    rng = np.random.default_rng(seed)
    out = []
    for k, steps in enumerate((0, 3, 7, 7, 12, 1)):
        method = wl.CFD if k % 2 == 0 else wl.MFD
        nx, ny = int(rng.integers(40, 300)), int(rng.integers(40, 300))
        out.append(wl.seismic_spec(method, nx, ny, steps, h=5.0, seed=int(rng.integers(1 << 30)),
                                   speeds=wl.random_layer_speeds(rng)))
    return out


def _make(adi, sp):
    s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP32)
    s.set_source(*sp.source.as_tuple())
    return s


def test_submit_poll_each_member_its_own_steps(adi):
    specs = _specs(5)
    sims = [_make(adi, sp) for sp in specs]
    sims[2].step(1)  # members may start at different parities
    t = adi.batch_submit(sims, [sp.steps for sp in specs])
    with pytest.raises(adi.AdiError) as e:
        sims[3].step(1)
    assert e.value.code == 6  # ADI_EBUSY while the ticket runs
    deadline = time.time() + 60
    while not adi.batch_poll(t):
        assert time.time() < deadline
        time.sleep(0.001)
    with pytest.raises(adi.AdiError):
        adi.batch_poll(t)  # retired
    for k, (sp, s) in enumerate(zip(specs, sims)):
        got = s.read()
        r = _make(adi, sp)
        r.step(sp.steps + (1 if k == 2 else 0))
        want = r.read()
        r.close()
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
    sims[3].step(1)  # released
    for s in sims:
        s.close()


def test_submit_rejects_busy_and_bad_arguments(adi):
    specs = _specs(6)[:3]
    sims = [_make(adi, sp) for sp in specs]
    b = adi.Batch(sims[:1])
    with pytest.raises(adi.AdiError) as e:
        adi.batch_submit(sims, [1, 1, 1])
    assert e.value.code == 6  # a member is in a batch
    b.close()
    with pytest.raises(adi.AdiError) as e:
        adi.batch_submit(sims, [1, -1, 1])
    assert e.value.code == 1
    with pytest.raises(adi.AdiError) as e:
        adi.batch_submit([sims[0], sims[0]], [1, 1])
    assert e.value.code == 1
    with pytest.raises(adi.AdiError):
        adi.batch_poll(123456)
    for s in sims:
        s.close()


def test_submit_with_harmonic_and_layer_members(adi):
    """Members with time-harmonic walls and forcing, with absorbing layers, and plain ones, each
    with its own step count in one asynchronous batch: every member ends exactly where it ends
    stepped alone (the phases rebuild the plan as members leave)."""
    specs = _specs(9)
    steps = [sp.steps for sp in specs]

    def make(k):
        sp = specs[k]
        s = _make(adi, sp)
        su = wl.shapes(sp.method, sp.nx, sp.ny)[0]
        rng = np.random.default_rng(100 + k)
        if k % 3 == 1:
            s.set_harmonic(rng.standard_normal(su), rng.standard_normal(su), 40.0, 0.3, 1.1)
        elif k % 3 == 2:
            s.set_sponge(12.0, 0.05)
        return s

    sims = [make(k) for k in range(len(specs))]
    t = adi.batch_submit(sims, steps)
    deadline = time.time() + 60
    while not adi.batch_poll(t):
        assert time.time() < deadline
        time.sleep(0.001)
    for k, s in enumerate(sims):
        r = make(k)
        r.step(steps[k])
        for x, y in zip(s.read(), r.read()):
            assert np.array_equal(x, y), k
        r.close()
        s.close()
