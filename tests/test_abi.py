"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

CPU-only: no compute call is made (host-only helpers such as adi_strerror and
adi_state_bytes are exercised because they touch no device).
"""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(adi_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2006_07583_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("adi_create", "adi_step", "adi_read_fields", "adi_batch_create", "adi_batch_step",
              "adi_destroy", "adi_strerror", "adi_set_source"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = sorted(n for n in _declared() if n not in exported)
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2006_07583_gb300 import adi

    declared = _declared()
    bound = set(adi.exported_symbols())
    assert declared <= bound, declared - bound


def test_host_only_helpers(libpath):
    from paper_2006_07583_gb300 import adi

    L = adi.lib()
    assert L.adi_abi_version() >= 1
    assert L.adi_strerror(0) == b"ok"
    assert L.adi_strerror(1) == b"invalid argument"
    # invalid configurations report 0 bytes; valid ones a positive count
    assert L.adi_state_bytes(0, 8, 64, 0) == 0
    assert L.adi_state_bytes(2, 64, 64, 0) == 0
    b32 = L.adi_state_bytes(0, 64, 64, 0)
    b64 = L.adi_state_bytes(0, 64, 64, 1)
    assert 0 < b32 < b64


def test_without_a_device_the_path_fails_loudly(libpath):
    """No CPU fallback: with no CUDA device every compute entry point returns ADI_ENOTSUP."""
    import numpy as np
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2006_07583_gb300 import adi, workloads as wl

    su, sv, sw = wl.shapes(0, 32, 32)
    with pytest.raises(adi.AdiError) as e:
        adi.Sim(0, 32, 32, 1.0 / 32, 0.01, np.ones(su))
    assert e.value.code == 7
    with pytest.raises(adi.AdiError) as e:
        adi.fixed_point(0, 32, 32, 1.0 / 32, 0.01, np.ones(su), np.zeros(su), np.zeros(sv), np.zeros(sw), 1)
    assert e.value.code == 7
