"""The C-ABI library builds for sm_103a, loads, and exports every entry point the
public header declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(hpc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("hpc_create", "hpc_solve", "hpc_get_omega", "hpc_destroy", "hpc_gram"):
        assert name in d


def test_library_loads_and_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.library_path())
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    assert sorted(set(_declared()) - set(lib.EXPORTED)) == []


def test_status_strings_without_gpu(lib):
    so = lib.load()
    assert so.hpc_status_string(0) == b"ok"
    assert b"capacity" in so.hpc_status_string(-3)
    o = lib.default_options()
    assert o.eps == 1e-6 and o.max_halvings == 60 and o.ls_window == 8


def test_build_is_sm103a_only():
    from paper_1710_10769_gb300 import _build

    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layouts_match_the_header(lib):
    """ctypes mirrors of the header's structs: sizes from the header's field list."""
    assert ctypes.sizeof(lib.Options) == 64
    assert ctypes.sizeof(lib.Stats) == 13 * 8 + 2 * 4 + 8
    assert ctypes.sizeof(lib.Tuning) == 40
    assert ctypes.sizeof(lib.TuneReport) == 8 + lib.TUNE_MAX_TRIALS * 16


def test_binding_checks_matrix_arguments_before_the_abi(lib):
    """The C ABI takes bare pointers and sizes, so the binding checks every matrix it
    passes: shape against the handle's (n, p), row-major contiguity, dtype, and device.
    A mismatch raises before any pointer crosses the boundary."""
    import numpy as np
    import torch

    m = lib._matrix
    X = torch.zeros(3, 4)
    assert m(X, 3, 4, "X") is X
    assert m(X, None, 4, "X") is X
    with pytest.raises(ValueError, match="shape"):
        m(X, 3, 5, "X")
    with pytest.raises(ValueError, match="shape"):
        m(X, 2, None, "X")
    with pytest.raises(ValueError, match="contiguous"):
        m(torch.zeros(4, 3).t(), 3, 4, "X")
    with pytest.raises(ValueError, match="2-D"):
        m(torch.zeros(12), None, None, "X")
    with pytest.raises(TypeError, match="dtype"):
        m(torch.zeros(3, 4, dtype=torch.int32), 3, 4, "X")
    with pytest.raises(ValueError, match="GPU"):
        m(X, 3, 4, "X", cuda=True)
    with pytest.raises(ValueError, match="CUDA"):
        m(np.zeros((3, 4)), 3, 4, "X", cuda=True)
    with pytest.raises(TypeError, match="dtype"):
        m(np.zeros((3, 4), np.int64), 3, 4, "X")
    with pytest.raises(TypeError):
        m([[0.0]], 1, 1, "X")
    assert m(torch.zeros(3, 4, dtype=torch.bfloat16), 3, 4, "X").dtype == torch.bfloat16
    # S for the stateless Gram: (p, lds >= p) rows of unit stride, on the device
    with pytest.raises(ValueError):
        lib._check_s(torch.zeros(4, 4), 4, (torch.float32,))
