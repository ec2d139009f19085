"""The C ABI library builds, loads and exports every entry point include/nufft.h
declares; argument checks that need no GPU return the documented codes."""

import ctypes
import os
import re

import pytest

from paper_1701_04492_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nufft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nufft\w*)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "nufft2_plan" in names and "nufft2_exec" in names and "nufft1_exec" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding's signature table covers exactly the header
    assert sorted(_lib.SIGNATURES) == names


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    plan = lib.nufft2_plan
    assert plan(ctypes.byref(h), 0, 4, None, 1e-9, 0, 0, 0, None) == -1          # N < 1
    assert plan(ctypes.byref(h), 16, -1, None, 1e-9, 0, 0, 0, None) == -1        # M < 0
    assert plan(ctypes.byref(h), 16, 4, None, 1e-9, 0, 0, 0, None) == -1         # x NULL
    assert plan(ctypes.byref(h), 16, 0, None, 0.0, 0, 0, 0, None) == -1          # eps
    assert plan(ctypes.byref(h), 16, 0, None, 1.0, 0, 0, 0, None) == -1
    assert plan(ctypes.byref(h), 16, 0, None, 1e-9, 2, 0, 0, None) == -1         # precision
    assert plan(ctypes.byref(h), 16, 0, None, 1e-9, 0, 3000, 0, None) == -1      # L not 2^n
    assert plan(ctypes.byref(h), 4096, 0, None, 1e-9, 0, 2048, 0, None) == -1    # L < N
    assert plan(ctypes.byref(h), 16, 0, None, 1e-9, 0, 512, 0, None) == -4       # L < 1024
    assert plan(ctypes.byref(h), 1 << 23, 0, None, 1e-9, 0, 0, 0, None) == -4    # N too large
    assert plan(ctypes.byref(h), 16, 0, None, 1e-9, 0, 0, 8, None) == -1         # unknown flag
    assert plan(None, 16, 0, None, 1e-9, 0, 0, 0, None) == -1
    assert h.value is None
    for fn in ("nufft2_exec", "nufft1_exec", "nufft2_exec_host", "nufft2_exec_unfused"):
        assert getattr(lib, fn)(None, None, None, None) == -1
    assert lib.nufft2_exec_dx(None, None, None, None, 0, None) == -1
    assert lib.nufft2_exec_batch(None, 1, None, 1, None, 1, None) == -1
    assert lib.nufft2_plan_info(None, None, None, None, None) == -1
    assert lib.nufft_destroy(None) == 0
    assert lib.nufft2_plan_reserve(None, 4, 0, None) == -1
    assert lib.nufft2_plan_reserved(None, None, None) == -1
    ms, fl = ctypes.c_float(), ctypes.c_double()
    assert lib.nufft_fp32_fma_peak(0, 1, None, ctypes.byref(ms), ctypes.byref(fl)) == -1      # iters < 1
    assert lib.nufft_fp32_fma_peak(10, 3, None, ctypes.byref(ms), ctypes.byref(fl)) == -1     # blocks per SM
    assert lib.nufft_fp32_fma_peak(10, 1, None, None, ctypes.byref(fl)) == -1
    msgs = [lib.nufft_strerror(code) for code in (0, -1, -2, -3, -4, -5, -6, -7)]
    assert all(msgs) and len(set(msgs)) == len(msgs)       # every status has its own message


def test_argument_errors_of_the_other_entry_families(lib):
    """The 2D plan, the batch plan, the inverse and the no-allocation forward reject bad
    arguments before any device work (so this runs without a GPU)."""
    h = ctypes.c_void_p()
    p2 = lib.nufft2d_plan
    assert p2(None, 64, 64, 0, None, None, 1e-6, 0, 0, None) == -1                    # out NULL
    assert p2(ctypes.byref(h), 0, 64, 0, None, None, 1e-6, 0, 0, None) == -1          # m < 1
    assert p2(ctypes.byref(h), 64, 0, 0, None, None, 1e-6, 0, 0, None) == -1          # n < 1
    assert p2(ctypes.byref(h), 64, 64, -1, None, None, 1e-6, 0, 0, None) == -1        # M < 0
    assert p2(ctypes.byref(h), 64, 64, 0, None, None, 0.0, 0, 0, None) == -1          # eps
    assert p2(ctypes.byref(h), 64, 64, 0, None, None, 1e-6, 2, 0, None) == -1         # precision
    assert p2(ctypes.byref(h), 64, 64, 5, None, None, 1e-6, 0, 0, None) == -1         # x, y NULL
    assert p2(ctypes.byref(h), 64, 64, 0, None, None, 1e-6, 0, 4, None) == -1         # flag
    assert p2(ctypes.byref(h), 4096, 64, 0, None, None, 1e-6, 0, 0, None) == -4       # m > 2048
    assert h.value is None
    b = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(1024, 2048)
    m = (ctypes.c_int64 * 2)(10, 20)
    e = (ctypes.c_double * 2)(1e-6, 1e-9)
    pm = lib.nufft2_plan_many
    assert pm(None, 2, n, m, None, None, e, 0, 0, None) == -1                          # out NULL
    assert pm(ctypes.byref(b), 0, n, m, None, None, e, 0, 0, None) == -1               # count < 1
    assert pm(ctypes.byref(b), 2, None, m, None, None, e, 0, 0, None) == -1            # N NULL
    assert pm(ctypes.byref(b), 2, n, m, None, None, e, 0, 0, None) == -1               # x NULL, M > 0
    assert pm(ctypes.byref(b), 2, n, m, None, None, e, 3, 0, None) == -1               # precision
    assert pm(ctypes.byref(b), 2, n, m, None, None, e, 0, 1, None) == -1               # flag
    assert b.value is None
    it, rr = ctypes.c_int(), ctypes.c_double()
    assert lib.nufft2_inverse(None, None, None, 1e-9, 10, ctypes.byref(it), ctypes.byref(rr), None) == -1
    assert lib.nufft2_exec_noalloc(0, 4, None, 1e-6, None, None, None) == -1          # N < 1
    assert lib.nufft2_exec_noalloc(1 << 20, 4, None, 1e-6, None, None, None) in (-1, -4)
