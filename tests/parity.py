"""Comparisons shared by the GPU parity tests: element by element and in the 2-norm.

The rounding of an FFT-based transform at one output is of the order of
u log2(L) times the 2-norm of its input, whatever the size of that output, so the
element-wise bound is taken relative to the root mean square of the reference:

    |got_j - ref_j| <= tol_el * rms(ref)   for every j,
    ||got - ref||_2 <= tol_2 * ||ref||_2.

FP32 (u = 6e-8, log2 L <= 22): tol_2 = 1e-5, the tolerance of the earlier 2-norm
comparisons; tol_el = 3e-5, so that one output off by 3e-5 of a typical one (a
mis-gathered row, a wrong bucket bound, a dropped rank) fails where the 2-norm over a
million outputs would hide it.  FP64 (u = 1.1e-16): tol_2 = 1e-13, tol_el = 1e-12.
"""

import numpy as np

TOL = {"f32": (1e-5, 3e-5), "f64": (1e-13, 1e-12)}


def rel2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rms(a):
    a = np.asarray(a)
    return np.linalg.norm(a) / np.sqrt(max(a.size, 1))


def assert_close(got, ref, prec="f32", scale=1.0, what=""):
    """Both bounds above, each widened by `scale` (the derivative's larger rounding)."""
    got, ref = np.ravel(np.asarray(got)), np.ravel(np.asarray(ref))
    tol2, tolel = TOL[prec]
    err = np.abs(got - ref)
    worst = int(np.argmax(err)) if err.size else 0
    assert rel2(got, ref) <= tol2 * scale, "%s: ||d||_2/||ref||_2 = %.3g" % (what, rel2(got, ref))
    assert (err.size == 0 or err[worst] <= tolel * scale * rms(ref)), \
        "%s: |d|_max = %.3g at %d, rms(ref) = %.3g" % (what, err[worst], worst, rms(ref))
