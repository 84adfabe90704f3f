"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/csvd.h.  CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

from paper_2601_11626_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csvd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(csvd_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def so():
    path = _build.build()
    assert os.path.exists(path)
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("csvd_incr_init", "csvd_incr_append", "csvd_tail_error", "csvd_bounds",
                     "csvd_cluster", "csvd_score", "csvd_tail_grad", "csvd_incr_free"):
        assert required in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_error_string_and_version_without_gpu(so):
    so.csvd_last_error.restype = ctypes.c_char_p
    so.csvd_version.restype = ctypes.c_char_p
    assert so.csvd_last_error() is not None
    assert b"sm_103a" in so.csvd_version()


def test_argument_errors_need_no_gpu(so):
    """Invalid arguments are rejected on the host before any CUDA call."""
    so.csvd_incr_init.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert so.csvd_incr_init(ctypes.byref(h), 8, 16, 0, None) == 1   # r > m
    assert so.csvd_incr_init(ctypes.byref(h), 8, 2, 7, None) == 1    # bad precision
    assert so.csvd_incr_init(None, 8, 2, 0, None) == 1
    # prepared evaluations: missing handles and arguments
    vp = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    so.csvd_score_plan.argtypes = [vp, i32, vp, vp, i32, dbl, i32, vp, i64, vp, vp, vp,
                                   ctypes.POINTER(vp)]
    so.csvd_plan_launch.argtypes = [vp, vp]
    so.csvd_plan_status.argtypes = [vp, vp]
    so.csvd_plan_free.argtypes = [vp]
    assert so.csvd_plan_launch(None, None) == 1
    assert so.csvd_plan_status(None, None) == 1
    assert so.csvd_plan_free(None) == 1
    out = ctypes.c_void_p(1)
    assert so.csvd_score_plan(None, 1, None, None, 1, 0.1, 1, None, 4, None, None, None,
                              ctypes.byref(out)) == 1
    assert out.value is None  # cleared on failure


def test_binding_fails_loudly_without_gpu():
    import torch
    from paper_2601_11626_gb300 import csvd
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        csvd.lib()


def test_product_path_does_not_import_oracle():
    """The CUDA path never routes through the oracle."""
    pkg = os.path.join(ROOT, "paper_2601_11626_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_build_flags_target_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_checks_row_counts_before_any_call():
    """The C ABI reads m rows from a block pointer; the binding refuses a
    block with a different row count before anything reaches the library
    (checked on CPU tensors, where the device test comes first)."""
    from paper_2601_11626_gb300 import csvd
    import torch
    with pytest.raises(ValueError, match="rows, expected m = 8"):
        csvd.block(torch.zeros(7, 2), 8)
    with pytest.raises(ValueError, match="rows, expected m = 8"):
        csvd._blocks([torch.zeros(7, 2), torch.zeros(8, 2)], 8)


def test_launch_planning_selftest_without_gpu(so):
    """The library's host-side planning checks (eigen-core tile placement for
    every launch class and core size, the tile-list walk, launch shared
    memory, one-column row grouping) pass without a GPU."""
    so.csvd_selftest.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    buf = ctypes.create_string_buffer(512)
    rc = so.csvd_selftest(buf, len(buf))
    assert rc == 0, buf.value.decode()
    assert buf.value == b"ok"
