"""The autotuner's table across processes (nufft_tune_save / _load / _clear): host code
only, so these run without a GPU.  A table round-trips exactly (eps to the last bit),
a malformed table merges nothing, and clearing reports what was held."""

import ctypes

import pytest

from paper_1701_04492_gb300 import _lib, build

HEADER = "nufft-tune-table 1\n"


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _n():
    return ctypes.c_int64(-1)


def _lines(path):
    return open(path).read().splitlines()


def _parse(line):
    """An entry's fields, eps as the double it denotes (its text form may differ)."""
    f = line.split()
    return tuple(float(v) if i == 3 else v for i, v in enumerate(f))


def test_round_trip_and_clear(lib, tmp_path):
    src = tmp_path / "in.txt"
    eps = 1.0 / 3.0 * 1e-9                       # not short in decimal: must survive the text form
    src.write_text(HEADER
                   + "0 1048576 1048576 %.17g 0 12 -> 1048576 0 0\n" % eps
                   + "0 3000 4096 1e-12 1 15 -> 8192 1 1\n")
    n = _n()
    assert lib.nufft_tune_clear(ctypes.byref(n)) == 0
    assert lib.nufft_tune_load(str(src).encode(), ctypes.byref(n)) == 0 and n.value == 2
    out = tmp_path / "out.txt"
    assert lib.nufft_tune_save(str(out).encode(), ctypes.byref(n)) == 0 and n.value == 2
    got = _lines(out)
    assert got[0] == HEADER.strip()
    assert sorted(map(_parse, got[1:])) == sorted(map(_parse, _lines(src)[1:]))
    # a second load of the same table replaces, it does not duplicate
    assert lib.nufft_tune_load(str(out).encode(), ctypes.byref(n)) == 0 and n.value == 2
    assert lib.nufft_tune_clear(ctypes.byref(n)) == 0 and n.value == 2
    assert lib.nufft_tune_clear(ctypes.byref(n)) == 0 and n.value == 0
    empty = tmp_path / "empty.txt"
    assert lib.nufft_tune_save(str(empty).encode(), ctypes.byref(n)) == 0 and n.value == 0
    assert _lines(empty) == [HEADER.strip()]


@pytest.mark.parametrize("body", [
    "0 4096 4096 1e-9 0 12 -> 3000 0 0\n",        # grid not a power of two
    "0 4096 4096 1e-9 0 12 -> 2048 0 0\n",        # grid shorter than N
    "0 4096 4096 1e-9 0 12 -> 512 0 0\n",         # grid below the smallest
    "0 4096 4096 1.5 0 12 -> 4096 0 0\n",         # eps outside (0, 1)
    "0 4096 4096 1e-9 2 12 -> 4096 0 0\n",        # no such precision
    "0 4096 4096 1e-9 0 17 -> 4096 0 0\n",        # rank above Table 2.1's cap
    "0 4096 3000 1e-9 0 12 -> 4096 0 0\n",        # M bound not a power of two
    "0 4096 4096 1e-9 0 12 -> 4096 2 0\n",        # split flag not 0/1
    "0 4096 4096 1e-9 0 12 => 4096 0 0\n",        # not the table's syntax
    "0 4096 4096 1e-9 0 12 -> 4096 0\n",          # a field missing
])
def test_malformed_tables_merge_nothing(lib, tmp_path, body):
    good = "0 8192 8192 1e-6 0 10 -> 8192 0 0\n"
    bad = tmp_path / "bad.txt"
    bad.write_text(HEADER + good + body)
    n = _n()
    lib.nufft_tune_clear(None)
    assert lib.nufft_tune_load(str(bad).encode(), ctypes.byref(n)) == -1
    assert lib.nufft_tune_clear(ctypes.byref(n)) == 0 and n.value == 0   # the good line was not merged either


def test_bad_paths_and_headers(lib, tmp_path):
    assert lib.nufft_tune_load(None, None) == -1
    assert lib.nufft_tune_save(None, None) == -1
    assert lib.nufft_tune_load(str(tmp_path / "missing.txt").encode(), None) == -1
    assert lib.nufft_tune_save(str(tmp_path / "no_dir" / "t.txt").encode(), None) == -1
    wrong = tmp_path / "wrong.txt"
    wrong.write_text("some other file\n0 8192 8192 1e-6 0 10 -> 8192 0 0\n")
    assert lib.nufft_tune_load(str(wrong).encode(), None) == -1
