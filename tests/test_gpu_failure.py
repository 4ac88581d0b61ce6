"""Failure detection on the GPU without a fault: the kernels' bounded waits give up when what
they wait for never comes (here an mbarrier that nothing arrives at), and the status reaches
the host; the context stays usable afterwards."""
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


def test_bounded_wait_gives_up_and_reports(adi):
    gave_up, cycles = adi.selftest_wait_timeout(1024)
    assert gave_up and cycles > 0
    # the context is still usable: a simulation steps normally afterwards
    su, sv, sw = wl.shapes(wl.MFD, 32, 32)
    s = adi.Sim(wl.MFD, 32, 32, 1.0 / 32, 0.01, np.ones(su), precision=adi.ADI_FP32)
    s.step(2)
    assert s.check_finite() == 0
    s.close()


def test_bounded_wait_rejects_bad_limits(adi):
    for polls in (0, -1, (1 << 22) + 1):
        with pytest.raises(adi.AdiError) as e:
            adi.selftest_wait_timeout(polls)
        assert e.value.code == 1
