"""GPU: the inverse NUFFT-II of section 3.3 (CG on the normal equations, the Toeplitz
A^H A applied through its circulant embedding) against the oracle and exact data.

f = A c_true is made by the direct sum of eq. (1.2) (or, at full size, by the FP64
forward transform); the solver must return c_true to the accuracy that the plan's eps,
the CG tolerance and the conditioning allow (perturbed grids with gamma <= 1/8 are well
conditioned: a few dozen iterations), and take about as many iterations as the oracle.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, lowrank  # noqa: E402
from paper_1701_04492_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1701_04492_gb300 import api as a
    return a


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N,gamma", [(4096, 1 / 8), (3000, 1 / 32), (2048, 1 / 4)])
def test_inverse_fp64_recovers_c_and_matches_oracle(api, N, gamma):
    x = wl.samples_perturbed(N, 110, gamma)
    c = wl.coeffs_cn(N, 111)
    f = direct.nudft2(x, c)
    p = api.Plan(N, x, 1e-14, "f64")
    cs, it, rr = p.inverse(torch.tensor(f, device="cuda"), tol=1e-13, maxit=2000)
    cs = cs.cpu().numpy()
    assert rr <= 1e-13
    assert _rel(cs, c) <= 1e-9
    P = lowrank.plan(N, x, 1e-14, p.L)
    co, ito, rro = lowrank.inverse_cg(P, f, 1e-13, 2000)
    assert abs(it - ito) <= 2
    assert _rel(cs, co) <= 1e-10


def test_inverse_on_grid_is_one_step_inverse_fft(api):
    N = 4096
    x = wl.samples_equispaced(N)
    f = wl.coeffs_cn(N, 112)
    p = api.Plan(N, x, 1e-14, "f64")
    cs, it, rr = p.inverse(torch.tensor(f, device="cuda"), tol=1e-13)
    assert it == 1
    assert np.max(np.abs(cs.cpu().numpy() - np.fft.ifft(f))) <= 1e-13 * np.max(np.abs(f))


def test_inverse_fp32(api):
    N = 1 << 14
    x = wl.samples_perturbed(N, 113, 1 / 8)
    c = wl.coeffs_cn(N, 114)
    f = direct.nudft2(x, c).astype(np.complex64)
    p = api.Plan(N, x, 1e-7, "f32")
    cs, it, rr = p.inverse(torch.tensor(f, device="cuda"), tol=1e-5, maxit=500)
    assert rr <= 1e-5
    assert _rel(cs.cpu().numpy(), c) <= 2e-4


def test_inverse_edge_cases_and_determinism(api):
    N = 2048
    x = wl.samples_perturbed(N, 115, 1 / 8)
    p = api.Plan(N, x, 1e-12, "f64")
    zero = torch.zeros(N, dtype=torch.complex128, device="cuda")
    c0, it0, rr0 = p.inverse(zero)
    assert it0 == 0 and rr0 == 0.0 and torch.count_nonzero(c0) == 0
    f = torch.tensor(direct.nudft2(x, wl.coeffs_cn(N, 116)), device="cuda")
    cm, itm, _ = p.inverse(f, maxit=0)
    assert itm == 0 and torch.count_nonzero(cm) == 0
    a, ia, _ = p.inverse(f, tol=1e-12)
    b, ib, _ = p.inverse(f, tol=1e-12)
    assert ia == ib and torch.equal(a, b)


def test_inverse_full_size(api):
    """N = 2^20, gamma = 1/8, FP64: f from the forward transform of a known c."""
    N = 1 << 20
    x = wl.samples_perturbed(N, 117, 1 / 8)
    c = torch.tensor(wl.coeffs_cn(N, 118), device="cuda")
    p = api.Plan(N, x, 1e-14, "f64")
    f = p.forward(c)
    cs, it, rr = p.inverse(f, tol=1e-12, maxit=500)
    assert rr <= 1e-12 and it < 100
    cs, c = cs.cpu().numpy(), c.cpu().numpy()
    assert _rel(cs, c) <= 1e-9
