"""The C-ABI library loads without a GPU and exports every function include/recoil.h declares."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _declared():
    text = open(os.path.join(ROOT, "include", "recoil.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(recoil_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["recoil_encode_with_splits", "recoil_combine_splits", "recoil_decode", "recoil_decode_batch",
                 "recoil_stream_info", "recoil_workspace_size", "recoil_free", "recoil_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(recoil_lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", recoil_lib.LIB_PATH], text=True)
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(recoil_lib.LIB_PATH)
    for n in _declared():
        getattr(lib, n)


def test_python_binding_names_match(recoil_lib):
    for n in _declared():
        assert hasattr(recoil_lib, n), n


def test_errors_without_gpu(recoil_lib):
    R = recoil_lib
    with pytest.raises(R.RecoilError) as e:
        R.encode_with_splits(np.zeros(10, np.uint8), 0, 4)
    assert e.value.code == R.EINVAL
    with pytest.raises(R.RecoilError) as e:
        R.encode_with_splits(np.arange(10, dtype=np.uint8), 2, 4)      # 10 symbols > 2^2 slots
    assert e.value.code == R.EINVAL
    s = R.encode_with_splits(np.arange(100, dtype=np.uint8) % 7, 8, 4)
    p = R.Plan([s])
    assert p.workspace_size % 256 == 0
    with pytest.raises(R.RecoilError):
        p.decode([0])                                                  # not uploaded
