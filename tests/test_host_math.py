"""The library's host arithmetic of the planning stage (C++), on the CPU, against the
oracle: the rank rule (section 2.1, Table 2.1 cap) and the coefficients of eq. (2.6).
The GPU plans use exactly these functions, so this pins the planner's K and a_pr
without a GPU."""

import ctypes

import numpy as np
import pytest

from oracle import lowrank
from paper_1701_04492_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


GAMMAS = [0.0, 1e-9, 1 / 128, 1 / 64, 1 / 32, 0.04, 1 / 16, 0.1, 1 / 8, 0.2, 1 / 4, 0.3, 0.45, 0.5]
EPSS = [0.5, 1e-2, 1e-4, 1e-6, 1e-7, 1e-9, 1e-12, 1e-14, 1e-15, 2.2e-16]


def test_rank_rule_matches_oracle(lib):
    K = ctypes.c_int()
    for gamma in GAMMAS:
        for eps in EPSS:
            assert lib.nufft_rank(eps, gamma, ctypes.byref(K)) == 0
            assert K.value == lowrank.choose_K(eps, gamma), (eps, gamma, K.value)


def test_rank_rule_table_2_1_single_and_half_rows(lib):
    # Table 2.1 (single precision 1.2e-7, half 9.8e-4) at the band edges gamma = 1/32 .. 1/2
    K = ctypes.c_int()
    for gamma, ks, kh in [(1 / 32, 5, 3), (1 / 16, 6, 3), (1 / 8, 7, 4), (1 / 4, 8, 5), (1 / 2, 10, 7)]:
        assert lib.nufft_rank(1.2e-7, gamma, ctypes.byref(K)) == 0 and K.value == ks
        assert lib.nufft_rank(9.8e-4, gamma, ctypes.byref(K)) == 0 and K.value == kh


def test_rank_rule_rejects(lib):
    K = ctypes.c_int()
    for eps, gamma in [(0.0, 0.1), (1.0, 0.1), (-1e-9, 0.1), (1e-9, -0.1), (1e-9, 0.51), (1e-9, float("nan")),
                       (float("nan"), 0.1)]:
        assert lib.nufft_rank(eps, gamma, ctypes.byref(K)) == -1
    assert lib.nufft_rank(1e-9, 0.1, None) == -1


@pytest.mark.parametrize("K", [1, 4, 12, 16, 24])
@pytest.mark.parametrize("gamma", [0.0, 1 / 32, 1 / 8, 0.5])
def test_coefficients_match_oracle(lib, K, gamma):
    alpha = (ctypes.c_double * (K * K))()
    assert lib.nufft_lowrank_coeffs(K, gamma, alpha) == 0
    al = np.array(alpha[:]).reshape(K, K)
    ref = lowrank.bessel_coefficients(K, gamma) if gamma > 0 else None
    if ref is None:
        # gamma = 0: J_0(0) = 1 and J_n(0) = 0 otherwise, so alpha = 4 on (0, 0) only
        expect = np.zeros((K, K))
        expect[0, 0] = 4.0
        assert np.array_equal(al, expect)
        return
    a = al * (1j ** np.arange(K))[None, :]
    assert np.max(np.abs(a - ref)) <= 1e-15


def test_coefficients_reject(lib):
    alpha = (ctypes.c_double * 4)()
    assert lib.nufft_lowrank_coeffs(0, 0.1, alpha) == -1
    assert lib.nufft_lowrank_coeffs(65, 0.1, alpha) == -1
    assert lib.nufft_lowrank_coeffs(2, 0.6, alpha) == -1
    assert lib.nufft_lowrank_coeffs(2, 0.1, None) == -1
