"""ctypes wrapper of oracle/direct.c: the NUDFT by its definition (eq. (1.2)).

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build()`` compiles the C
file with gcc into ``oracle/_direct.so`` next to it; it is called lazily on first
use and by ``__graft_entry__.build()``.
"""

from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_direct.so")
_lib = None


def build(force=False):
    """Compile direct.c (plain C, OpenMP, no fast-math, no FMA contraction)."""
    stamp = _LIB + ".machine"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        for name in ("nudft2", "nudft2h", "nudft2d"):
            getattr(lib, name).argtypes = [i64, i64, p, p, p]
            getattr(lib, name).restype = None
        lib.nudft2_2d.argtypes = [i64, i64, i64, p, p, p, p]
        lib.nudft2_2d.restype = None
        lib.nudft2h_at.argtypes = [i64, p, i64, p, p, p]
        lib.nudft2h_at.restype = None
        lib.nudft2h_2d_at.argtypes = [i64, p, p, i64, p, p, p, p]
        lib.nudft2h_2d_at.restype = None
        _lib = lib
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nudft2(x, c):
    """f_j = sum_{k<N} c_k exp(-2 pi i x_j k)  (eq. (1.2))."""
    x, c = _f64(x), _c128(c)
    f = np.empty(x.size, dtype=np.complex128)
    _load().nudft2(c.size, x.size, x.ctypes.data, c.ctypes.data, f.ctypes.data)
    return f


def nudft2_adjoint(x, g, N):
    """c_k = sum_j g_j exp(+2 pi i x_j k), k < N: the conjugate transpose of nudft2."""
    x, g = _f64(x), _c128(g)
    c = np.empty(int(N), dtype=np.complex128)
    _load().nudft2h(int(N), x.size, x.ctypes.data, g.ctypes.data, c.ctypes.data)
    return c


def nudft2_adjoint_at(x, g, ks):
    """c_k = sum_j g_j exp(+2 pi i x_j k) at the listed frequencies ks (the adjoint of
    eq. (1.2) at chosen outputs, for sizes where all N outputs would take too long)."""
    x, g = _f64(x), _c128(g)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    c = np.empty(ks.size, dtype=np.complex128)
    _load().nudft2h_at(ks.size, ks.ctypes.data, x.size, x.ctypes.data, g.ctypes.data, c.ctypes.data)
    return c


def nudft2_deriv(x, c):
    """f'_j = sum_k (-2 pi i k) c_k exp(-2 pi i x_j k) = d f_j / d x_j."""
    x, c = _f64(x), _c128(c)
    f = np.empty(x.size, dtype=np.complex128)
    _load().nudft2d(c.size, x.size, x.ctypes.data, c.ctypes.data, f.ctypes.data)
    return f


def nudft2_2d(x, y, C):
    """f_j = sum_{k1<m, k2<n} C[k1, k2] exp(-2 pi i (k1 x_j + k2 y_j))  (eq. (4.1))."""
    x, y, C = _f64(x), _f64(y), _c128(C)
    m, n = C.shape
    f = np.empty(x.size, dtype=np.complex128)
    _load().nudft2_2d(m, n, x.size, x.ctypes.data, y.ctypes.data, C.ctypes.data, f.ctypes.data)
    return f


def nudft2_2d_adjoint(x, y, g, m, n, k1s=None, k2s=None):
    """C[k1, k2] = sum_j g_j exp(+2 pi i (k1 x_j + k2 y_j)): the conjugate transpose of
    nudft2_2d (eq. (4.1)).  With k1s, k2s (equal-length index lists) only those entries
    are formed and returned as a vector; otherwise the whole m x n matrix."""
    x, y, g = _f64(x), _f64(y), _c128(g)
    full = k1s is None
    if full:
        k1s, k2s = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    k1s = np.ascontiguousarray(np.ravel(k1s), dtype=np.int64)
    k2s = np.ascontiguousarray(np.ravel(k2s), dtype=np.int64)
    out = np.empty(k1s.size, dtype=np.complex128)
    _load().nudft2h_2d_at(k1s.size, k1s.ctypes.data, k2s.ctypes.data, x.size, x.ctypes.data, y.ctypes.data,
                          g.ctypes.data, out.ctypes.data)
    return out.reshape(int(m), int(n)) if full else out
