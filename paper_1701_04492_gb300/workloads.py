"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds no arithmetic of the method: it only draws inputs.  Both the
product path (benchmarks, smoke test) and the CPU oracle's tests take their inputs
from here, so the two see identical bits.  Everything is numpy (PCG64), FP64 on the
host; FP32 runs round the same draws to complex64.

Sample sets (section 2.4 and the experiments of section 2):
  uniform      x_j ~ U[0, 1), unsorted
  perturbed    x_j = j/N + gamma * u_j / N, u_j ~ U[-1, 1]   (eq. (2.1) with the bound gamma)
  equispaced   x_j = j / N                                    (gamma = 0: one FFT)
  worst        x_j = (j + gamma)/N for j <= floor(N/2), else (j - gamma)/N  (section 2.4)
Coefficients:
  cn           c_k ~ CN(0, 1): real and imaginary parts i.i.d. N(0, 1/2)
  decay        c_k = randn / (k+1)^2 (the decaying vector of section 2.4), real
  decay_2d     C[k1,k2] ~ CN(0,1) / (1 + k1^2 + k2^2)^(1/2)
"""

from __future__ import annotations

import numpy as np

_TAG_X, _TAG_C, _TAG_Y, _TAG_G, _TAG_P = 11, 22, 33, 44, 55


def _rng(seed, tag):
    return np.random.default_rng([int(seed), int(tag)])


def coeffs_cn(n, seed, tag=_TAG_C):
    r = _rng(seed, tag)
    re = r.standard_normal(n)
    im = r.standard_normal(n)
    return (re + 1j * im) * np.sqrt(0.5)


def coeffs_decay(n, seed):
    r = _rng(seed, _TAG_C)
    return r.standard_normal(n) / (np.arange(1, n + 1, dtype=np.float64) ** 2)


def cotangent_cn(n, seed):
    """A CN(0,1) vector on the sample side (the g of an adjoint or a backward)."""
    return coeffs_cn(n, seed, tag=_TAG_G)


def samples_uniform(m, seed, tag=_TAG_X):
    return _rng(seed, tag).random(m)


def samples_perturbed(n, seed, gamma=0.5):
    u = _rng(seed, _TAG_X).uniform(-1.0, 1.0, n)
    return np.arange(n, dtype=np.float64) / n + gamma * u / n


def samples_equispaced(n):
    return np.arange(n, dtype=np.float64) / n


def samples_worst(n, gamma):
    j = np.arange(n, dtype=np.float64)
    x = (j - gamma) / n
    half = np.arange(n) <= n // 2
    x[half] = (j[half] + gamma) / n
    return x


def coeffs_2d_decay(m, n, seed):
    k1 = np.arange(m, dtype=np.float64)[:, None]
    k2 = np.arange(n, dtype=np.float64)[None, :]
    c = coeffs_cn(m * n, seed).reshape(m, n)
    return c / np.sqrt(1.0 + k1 ** 2 + k2 ** 2)


def samples_2d_uniform(m_samples, seed):
    return samples_uniform(m_samples, seed, _TAG_X), samples_uniform(m_samples, seed, _TAG_Y)


def uneven_batch(count, seed, log2_lo=10, log2_hi=18, eps_set=(1e-4, 1e-7, 1e-12)):
    """Problem sizes and accuracies of a serving-style batch: N log-uniform in
    [2^lo, 2^hi] (rounded to an integer), eps drawn from eps_set."""
    r = _rng(seed, _TAG_P)
    N = np.rint(2.0 ** r.uniform(log2_lo, log2_hi, count)).astype(np.int64)
    eps = np.asarray(eps_set)[r.integers(0, len(eps_set), count)]
    return N, eps
