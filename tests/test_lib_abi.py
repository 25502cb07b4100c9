"""The C-ABI library builds for sm_103a and exports every entry point that
include/gve.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gve.h")).read()
    return sorted(set(re.findall(r"GVE_API\s+[\w\s\*]+?\b(gve_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2608_14112_b300 import build
    return str(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gve_allocate", "gve_evaluate", "gve_refine", "gve_loss_grad", "gve_backward", "gve_bin",
                 "gve_count_pairs", "gve_ctx_create", "gve_ctx_destroy", "gve_status_str", "gve_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings(libpath):
    L = ctypes.CDLL(libpath)
    L.gve_status_str.restype = ctypes.c_char_p
    L.gve_status_str.argtypes = [ctypes.c_int]
    assert L.gve_status_str(0) == b"ok"
    assert L.gve_status_str(2) == b"infeasible budget"
    assert L.gve_status_str(99) == b"unknown status"


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the sizes the C compiler gives."""
    from paper_2608_14112_b300 import gve
    assert ctypes.sizeof(gve.Dims) == 12
    assert ctypes.sizeof(gve.EvalOpts) == 20
    assert ctypes.sizeof(gve.AllocOpts) == 32
    assert ctypes.sizeof(gve.Schedule) == 48
    assert ctypes.sizeof(gve.Stats) == 72
    assert ctypes.sizeof(gve.AllocInfo) == 56


def test_product_path_has_no_cpu_fallback(monkeypatch):
    """Without a CUDA device the binding raises instead of computing on the CPU."""
    import torch
    from paper_2608_14112_b300 import gve
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        gve.context()
