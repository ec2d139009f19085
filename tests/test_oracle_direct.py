"""Pins for the direct NUDFT oracle (eq. (1.2)) against values fixed by mathematics.

None of these re-type the oracle's formula: they compare it with multiple-precision
brute force (mpmath), closed forms, and a library FFT on the uniform grid.
"""

import math

import mpmath
import numpy as np
import pytest

from oracle import direct
from paper_1701_04492_gb300 import workloads as wl

mpmath.mp.dps = 40


def _mp_nudft(x, c, sign=-1, deriv=False):
    out = []
    for xj in x:
        acc = mpmath.mpc(0)
        for k, ck in enumerate(c):
            term = mpmath.mpc(ck.real, ck.imag) * mpmath.expjpi(sign * 2 * mpmath.mpf(float(xj)) * k)
            if deriv:
                term *= -2j * mpmath.pi * k
            acc += term
        out.append(complex(acc))
    return np.array(out)


def test_single_frequency_is_an_exponential():
    # c = e_k gives f_j = exp(-2 pi i x_j k), including samples far outside [0, 1).
    N = 64
    x = np.concatenate([wl.samples_uniform(20, 3), [-12.3456789, 1000.123456789, 1.0, -0.5, 0.0]])
    for k in (0, 1, 17, 63):
        c = np.zeros(N, complex)
        c[k] = 1.0
        f = direct.nudft2(x, c)
        ref = np.array([complex(mpmath.expjpi(-2 * mpmath.mpf(float(xj)) * k)) for xj in x])
        assert np.max(np.abs(f - ref)) < 1e-15


def test_constant_coefficients_geometric_sum():
    # c = 1: f_j = (1 - e^{-2 pi i N x}) / (1 - e^{-2 pi i x}), = N at integer x.
    N = 300
    x = np.concatenate([wl.samples_uniform(16, 5), [0.0, 2.0, -3.0]])
    f = direct.nudft2(x, np.ones(N, complex))
    for xj, fj in zip(x, f):
        if float(xj).is_integer():
            ref = N
        else:
            X = mpmath.mpf(float(xj))
            ref = complex((1 - mpmath.expjpi(-2 * N * X)) / (1 - mpmath.expjpi(-2 * X)))
        assert abs(fj - ref) < 1e-12


def test_uniform_grid_is_the_fft():
    N = 1024
    c = wl.coeffs_cn(N, 7)
    f = direct.nudft2(wl.samples_equispaced(N), c)
    assert np.max(np.abs(f - np.fft.fft(c))) < 1e-12


def test_shifted_grid_is_a_modulated_fft():
    # x_j = j/N + a: f = FFT(c o exp(-2 pi i a k)).
    N, a = 512, 0.3125 / 512   # dyadic, so every x_j = j/N + a is exact in FP64
    c = wl.coeffs_cn(N, 8)
    x = wl.samples_equispaced(N) + a
    ref = np.fft.fft(c * np.exp(-2j * math.pi * a * np.arange(N)))
    assert np.max(np.abs(direct.nudft2(x, c) - ref)) < 1e-12


def test_bruteforce_multiprecision_tiny():
    N, M = 13, 9
    c = wl.coeffs_cn(N, 9)
    x = np.concatenate([wl.samples_uniform(M - 2, 9), [-7.25, 3.999]])
    f = direct.nudft2(x, c)
    assert np.max(np.abs(f - _mp_nudft(x, c))) < 1e-14


def test_derivative_multiprecision_tiny():
    N, M = 11, 6
    c = wl.coeffs_cn(N, 10)
    x = wl.samples_uniform(M, 10)
    fp = direct.nudft2_deriv(x, c)
    assert np.max(np.abs(fp - _mp_nudft(x, c, deriv=True))) < 1e-12


def test_adjoint_is_conjugate_transpose_multiprecision():
    N, M = 10, 12
    g = wl.cotangent_cn(M, 11)
    x = wl.samples_uniform(M, 11)
    c = direct.nudft2_adjoint(x, g, N)
    # c_k = sum_j g_j exp(+2 pi i x_j k): the k-th entry of the +sign sum over j.
    ref = []
    for k in range(N):
        acc = mpmath.mpc(0)
        for xj, gj in zip(x, g):
            acc += mpmath.mpc(gj.real, gj.imag) * mpmath.expjpi(2 * mpmath.mpf(float(xj)) * k)
        ref.append(complex(acc))
    assert np.max(np.abs(c - np.array(ref))) < 1e-14


def test_2d_separable_is_a_product():
    # C = a b^T gives f_j = nudft(x_j; a) * nudft(y_j; b).
    m, n, M = 12, 9, 30
    a, b = wl.coeffs_cn(m, 12), wl.coeffs_cn(n, 13)
    x, y = wl.samples_2d_uniform(M, 12)
    f = direct.nudft2_2d(x, y, np.outer(a, b))
    ref = direct.nudft2(x, a) * direct.nudft2(y, b)
    assert np.max(np.abs(f - ref)) < 1e-13


def test_2d_multiprecision_tiny():
    m, n, M = 4, 5, 3
    C = wl.coeffs_cn(m * n, 14).reshape(m, n)
    x, y = wl.samples_2d_uniform(M, 14)
    f = direct.nudft2_2d(x, y, C)
    for j in range(M):
        acc = mpmath.mpc(0)
        for k1 in range(m):
            for k2 in range(n):
                e = mpmath.expjpi(-2 * (mpmath.mpf(float(x[j])) * k1 + mpmath.mpf(float(y[j])) * k2))
                acc += mpmath.mpc(C[k1, k2].real, C[k1, k2].imag) * e
        assert abs(f[j] - complex(acc)) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3])
def test_degenerate_sizes(N):
    c = wl.coeffs_cn(N, 15)
    x = wl.samples_uniform(4, 15)
    assert np.max(np.abs(direct.nudft2(x, c) - _mp_nudft(x, c))) < 1e-15
    assert direct.nudft2(np.zeros(0), c).shape == (0,)
