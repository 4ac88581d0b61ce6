"""adi_step_static (one step into caller-owned device buffers, temporaries in a fixed-size
device array of the library) against the handle path (adi_create + adi_step + adi_read_fields
with the thread-per-line solver) on the same seeded inputs, over two calls in a row.

Both paths launch the same kernels in the same order on the same values, so they agree to
rounding; the tolerance is the path's FP64 / FP32 parity bound.
"""
import numpy as np
import pytest

from paper_2006_07583_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CFD, MFD = wl.CFD, wl.MFD


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_07583_gb300 import adi

    adi.lib()
    return adi, torch


def _case(method, nx, ny, seed, dtype):
    rng = np.random.default_rng(seed)
    su, sv, sw = wl.shapes(method, nx, ny)
    h = 1.0 / max(nx, ny)
    # values exactly representable in the path's precision, so both paths see the same data
    c = rng.uniform(0.6, 1.4, su).astype(dtype).astype(np.float64)
    U = rng.standard_normal(su).astype(dtype).astype(np.float64)
    V = rng.standard_normal(sv).astype(dtype).astype(np.float64)
    W = rng.standard_normal(sw).astype(dtype).astype(np.float64)
    dt = 0.8 * h / c.max()
    return h, dt, c, U, V, W


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("method,nx,ny", [(CFD, 40, 29), (MFD, 33, 47), (MFD, 128, 128)])
def test_static_step_matches_handle_path_twice(env, method, nx, ny, prec):
    adi, torch = env
    precision = adi.ADI_FP64 if prec == "fp64" else adi.ADI_FP32
    np_t = np.float64 if prec == "fp64" else np.float32
    t_t = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    h, dt, c, U, V, W = _case(method, nx, ny, 11 + nx, np_t)

    sim = adi.Sim(method, nx, ny, h, dt, c, U, V, W, precision=precision, solver=adi.ADI_SOLVER_LINE)
    dev = [torch.tensor(a.astype(np_t), dtype=t_t, device="cuda") for a in (c, U, V, W)]
    out = [torch.empty_like(x) for x in dev[1:]]
    torch.cuda.synchronize()
    for call in range(2):
        adi.step_static(method, nx, ny, h, dt, precision, *[x.data_ptr() for x in dev],
                        *[x.data_ptr() for x in out])
        sim.step(1)
        Uh, Vh, Wh = sim.read()
        for got, ref, name in zip(out, (Uh, Vh, Wh), "uvw"):
            g = got.cpu().numpy().astype(np.float64)
            err = np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300)
            assert err <= tol, (call, name, err)
        # the outputs become the next call's inputs
        dev = [dev[0]] + [x.clone() for x in out]
    sim.close()


def test_static_step_rejects_sizes_beyond_capacity(env):
    adi, torch = env
    nx = ny = 129  # one more than the array's maximum
    su, sv, sw = wl.shapes(CFD, nx, ny)
    bufs = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in (su, su, sv, sw, su, sv, sw)]
    with pytest.raises(adi.AdiError) as ex:
        adi.step_static(CFD, nx, ny, 1.0 / nx, 0.5 / nx, adi.ADI_FP64, *[b.data_ptr() for b in bufs])
    assert ex.value.code == 2  # ADI_ENOMEM
    # aliased output and input
    b = bufs
    with pytest.raises(adi.AdiError) as ex:
        adi.step_static(CFD, 32, 32, 1.0 / 32, 0.5 / 32, adi.ADI_FP64, *[x.data_ptr() for x in b[:4]],
                        b[1].data_ptr(), b[5].data_ptr(), b[6].data_ptr())
    assert ex.value.code == 1  # ADI_EINVAL
