"""GPU parity of the 2D NUFFT-II (section 4, eq. (4.4)) and its adjoint against the oracle.

FP32 exec vs the 2D low-rank oracle on the same grids: ||df||_2 / ||f||_2 <= 1e-5 and every
|df_j| <= 3e-5 rms(f) (FFT rounding, as in 1D; tests/parity.py).  vs the direct 2D sum of
eq. (4.1): |df|_inf <= max(eps (1 + eps/4), 5e-6) ||C||_1 (the product bound of the two
directions at eps / 2 each, floored at the FP32 target).  The adjoint alike, with ||g||_1.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, lowrank  # noqa: E402
from paper_1701_04492_gb300 import workloads as wl  # noqa: E402
from parity import assert_close  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1701_04492_gb300 import api as a
    return a


def _rel2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _coeffs(m, n, seed):
    r = np.random.default_rng(seed)
    C = (r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))) / np.sqrt(2)
    return C.astype(np.complex64)


@pytest.mark.parametrize("m,n,M", [(64, 64, 5000), (100, 40, 3000), (32, 256, 2000), (256, 32, 4000),
                                   (1024, 48, 6000)])
@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-9])
def test_2d_matches_oracle(api, m, n, M, eps):
    x, y = wl.samples_2d_uniform(M, m + 7 * n)
    C = _coeffs(m, n, m * n)
    p = api.Plan2D(m, n, x, y, eps)
    P = lowrank.plan2d(m, n, x, y, eps, p.Lx, p.Ly)
    assert (p.Kx, p.Ky) == (P.px.K, P.py.K)
    assert p.gamma_x == P.px.gamma and p.gamma_y == P.py.gamma
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    fo = lowrank.nufft2_2d(P, C.astype(np.complex128))
    assert_close(f, fo, "f32", what="2d")
    rows = np.arange(0, M, max(1, M // 50))
    fd = direct.nudft2_2d(x[rows], y[rows], C.astype(np.complex128))
    bound = max(eps * (1 + eps / 4), 5e-6) * np.sum(np.abs(C))
    assert np.max(np.abs(f[rows] - fd)) <= bound


def test_2d_separable_is_product_of_1d_sums(api):
    m, n, M = 128, 64, 4000
    x, y = wl.samples_2d_uniform(M, 90)
    a = wl.coeffs_cn(m, 91).astype(np.complex64)
    b = wl.coeffs_cn(n, 92).astype(np.complex64)
    C = np.outer(a, b).astype(np.complex64)
    p = api.Plan2D(m, n, x, y, 1e-6)
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    ref = direct.nudft2_2d(x, y, C.astype(np.complex128))
    assert np.max(np.abs(f - ref)) <= 5e-6 * np.sum(np.abs(C))


def test_2d_on_grid_is_the_2d_fft(api):
    """Samples on the grid (x = s/m, y = t/n): gamma = 0 in both directions, K = 1, and
    the transform is the plain 2D FFT read at the samples."""
    m, n = 64, 128
    r = np.random.default_rng(93)
    s = r.integers(0, m, 3000)
    t = r.integers(0, n, 3000)
    x, y = s / m, t / n
    C = _coeffs(m, n, 94)
    p = api.Plan2D(m, n, x, y, 1e-9)
    assert (p.Kx, p.Ky) == (1, 1)
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    ref = np.fft.fft2(C.astype(np.complex128))[s, t]
    assert _rel2(f, ref) <= 1e-6
    assert_close(f, ref, "f32", what="on-grid 2D FFT")


def test_2d_deterministic_and_empty(api):
    m, n, M = 256, 256, 20000
    x, y = wl.samples_2d_uniform(M, 95)
    C = torch.tensor(_coeffs(m, n, 96), device="cuda")
    p = api.Plan2D(m, n, x, y, 1e-6)
    f1 = p.forward(C).clone()
    f2 = p.forward(C)
    assert torch.equal(f1, f2)
    e = api.Plan2D(m, n, np.zeros(0), np.zeros(0), 1e-6)
    assert e.forward(C).numel() == 0


def test_2d_full_size_sampled_rows(api):
    """m = n = 1024, M = 2^20, eps = 1e-6, uniform samples, c ~ CN(0,1)/(1 + k1^2 + k2^2)^(1/2):
    every 8192nd sample against the direct 2D sum."""
    m = n = 1024
    M = 1 << 20
    x, y = wl.samples_2d_uniform(M, 2024)
    C = wl.coeffs_2d_decay(m, n, 2024).astype(np.complex64)
    p = api.Plan2D(m, n, x, y, 1e-6)
    assert (p.Kx, p.Ky) == (lowrank.choose_K(5e-7, p.gamma_x), lowrank.choose_K(5e-7, p.gamma_y))
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    rows = np.arange(0, M, 8192)
    fd = direct.nudft2_2d(x[rows], y[rows], C.astype(np.complex128))
    assert np.max(np.abs(f[rows] - fd)) <= 5e-6 * np.sum(np.abs(C))
    assert _rel2(f[rows], fd) <= 1e-5


@pytest.mark.parametrize("m,n,M,eps", [(64, 64, 5000, 1e-9), (100, 40, 3000, 1e-12), (48, 300, 2000, 1e-14),
                                       (256, 1024, 1 << 16, 1e-6)])
def test_2d_fp64_matches_oracle(api, m, n, M, eps):
    """FP64 (the paper's precision): against the FP64 oracle to rounding and against the
    direct 2D sum within eps(1 + eps/4) ||C||_1.  At n = 1024 the ten y-ranks' FP64 slots do
    not all fit in shared memory, so the row pass transforms and gathers them in groups."""
    x, y = wl.samples_2d_uniform(M, m + 3 * n)
    r = np.random.default_rng(m * n + 1)
    C = (r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))) / np.sqrt(2)
    p = api.Plan2D(m, n, x, y, eps, precision="f64")
    P = lowrank.plan2d(m, n, x, y, eps, p.Lx, p.Ly)
    assert (p.Kx, p.Ky) == (P.px.K, P.py.K)
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    assert_close(f, lowrank.nufft2_2d(P, C), "f64", scale=10, what="2d f64")
    rows = np.arange(0, M, max(1, M // 40))
    fd = direct.nudft2_2d(x[rows], y[rows], C)
    assert np.max(np.abs(f[rows] - fd)) <= (eps * (1 + eps / 4) + 1e-13) * np.sum(np.abs(C))


def test_2d_fp32_longest_rows_in_groups(api):
    """n = 2048 in FP32: the ten y-ranks' slots exceed shared memory, so the row pass
    works in groups; the result still matches the oracle."""
    m, n, M = 64, 2048, 20000
    x, y = wl.samples_2d_uniform(M, 98)
    C = _coeffs(m, n, 99)
    p = api.Plan2D(m, n, x, y, 1e-6)
    P = lowrank.plan2d(m, n, x, y, 1e-6, p.Lx, p.Ly)
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    assert_close(f, lowrank.nufft2_2d(P, C.astype(np.complex128)), "f32", what="2d groups")


def test_2d_unsupported_calls(api):
    """The 2D plan has its forward and its adjoint; the x-derivative calls are 1D only."""
    x, y = wl.samples_2d_uniform(100, 97)
    p = api.Plan2D(64, 64, x, y, 1e-6)
    lib = __import__("paper_1701_04492_gb300._lib", fromlist=["load"]).load()
    g = torch.zeros(100, dtype=torch.complex64, device="cuda")
    c = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    gx = torch.zeros(100, dtype=torch.float32, device="cuda")
    import ctypes
    vp = ctypes.c_void_p
    assert lib.nufft2_exec_dx(p._h, vp(c.data_ptr()), vp(g.data_ptr()), vp(gx.data_ptr()), 0, None) == -4
    assert lib.nufft2_exec_deriv(p._h, vp(c.data_ptr()), vp(g.data_ptr()), vp(g.data_ptr()), None) == -4


# ---- the 2D adjoint: C = A^H g (eq. (4.4) conjugated and reversed) --------------------

def _adj_case(m, n, M, eps, prec, seed):
    x, y = wl.samples_2d_uniform(M, seed)
    g = wl.cotangent_cn(M, seed + 1)
    if prec == "f32":
        g = g.astype(np.complex64).astype(np.complex128)
    return x, y, g


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("m,n,M,eps", [(64, 64, 5000, 1e-6), (100, 40, 3000, 1e-9), (32, 256, 2000, 1e-4),
                                       (256, 32, 4000, 1e-12), (1024, 48, 6000, 1e-6), (40, 100, 1, 1e-9),
                                       (1, 1, 10, 1e-6), (33, 2047, 7000, 1e-6)])
def test_2d_adjoint_matches_oracle(api, prec, m, n, M, eps):
    """Every entry against the 2D low-rank oracle (element-wise and in the 2-norm), and
    every entry (small sizes) or a seeded subset against the direct conjugate sum of eq.
    (4.1): |dC|_max <= max(eps (1 + eps/4), 5e-6) ||g||_1 in FP32, (eps (1 + eps/4) + 1e-13)
    ||g||_1 in FP64."""
    x, y, g = _adj_case(m, n, M, eps, prec, m + 5 * n)
    p = api.Plan2D(m, n, x, y, eps, precision=prec)
    P = lowrank.plan2d(m, n, x, y, eps, p.Lx, p.Ly)
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    C = p.adjoint(torch.tensor(g, dtype=cdt, device="cuda")).cpu().numpy()
    assert C.shape == (m, n)
    assert_close(C, lowrank.nufft2_2d_adjoint(P, g), prec, scale=1 if prec == "f32" else 10, what="2d adjoint")
    r = np.random.default_rng(m * n)
    nk = min(m * n, 200)
    k1, k2 = (np.unravel_index(r.choice(m * n, nk, replace=False), (m, n)))
    Cd = direct.nudft2_2d_adjoint(x, y, g, m, n, k1, k2)
    tol = max(eps * (1 + eps / 4), 5e-6) if prec == "f32" else eps * (1 + eps / 4) + 1e-13
    assert np.max(np.abs(C[k1, k2] - Cd)) <= tol * np.sum(np.abs(g))
    p.check()


def test_2d_adjoint_inner_product_fp64(api):
    """<A C, g> = <C, A^H g> for the GPU's own 2D forward and adjoint (FP64, 1e-13 relative)."""
    m, n, M = 96, 80, 7000
    x, y = wl.samples_2d_uniform(M, 300)
    r = np.random.default_rng(301)
    C = (r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))) / np.sqrt(2)
    g = wl.cotangent_cn(M, 302)
    p = api.Plan2D(m, n, x, y, 1e-12, precision="f64")
    f = p.forward(torch.tensor(C, device="cuda")).cpu().numpy()
    ah = p.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    assert abs(np.vdot(g, f) - np.vdot(ah, C)) <= 1e-13 * np.linalg.norm(f) * np.linalg.norm(g)


def test_2d_adjoint_on_grid_is_the_conjugate_2d_fft(api):
    """Samples on the grid: K = 1 in both directions, and A^H g is m n ifft2 of the sums of
    g at each grid point (the conjugate 2D DFT), a closed form."""
    m, n = 64, 128
    r = np.random.default_rng(303)
    s, t = r.integers(0, m, 3000), r.integers(0, n, 3000)
    g = wl.cotangent_cn(3000, 304).astype(np.complex64)
    p = api.Plan2D(m, n, s / m, t / n, 1e-9)
    assert (p.Kx, p.Ky) == (1, 1)
    C = p.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    Z = np.zeros((m, n), dtype=np.complex128)
    np.add.at(Z, (s, t), g.astype(np.complex128))
    assert_close(C, np.fft.ifft2(Z) * m * n, "f32", what="on-grid adjoint")


def test_2d_adjoint_groups_and_deterministic(api):
    """n = 2048 at eps = 1e-12 in FP32: the y-ranks' slots exceed shared memory, so the
    adjoint's row pass scatters and transforms them in groups; repeated calls give the same
    bits (segmented sums, no atomics); an empty sample set gives C = 0."""
    m, n, M = 48, 2048, 20000
    x, y, g = _adj_case(m, n, M, 1e-12, "f32", 305)
    p = api.Plan2D(m, n, x, y, 1e-12)
    assert p.Ky > 10
    gd = torch.tensor(g.astype(np.complex64), device="cuda")
    C1 = p.adjoint(gd).clone()
    C2 = p.adjoint(gd)
    assert torch.equal(C1, C2)
    P = lowrank.plan2d(m, n, x, y, 1e-12, p.Lx, p.Ly)
    assert_close(C1.cpu().numpy(), lowrank.nufft2_2d_adjoint(P, g), "f32", what="grouped adjoint")
    e = api.Plan2D(m, n, np.zeros(0), np.zeros(0), 1e-6)
    Ce = e.adjoint(torch.zeros(0, dtype=torch.complex64, device="cuda"))
    assert torch.count_nonzero(Ce).item() == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_2d_adjoint_full_size(api, prec):
    """The 2D workload's size: m = n = 1024, M = 2^20 uniform samples, eps = 1e-6.  Every
    entry against the 2D oracle; 64 entries against the direct conjugate sum."""
    m = n = 1024
    M = 1 << 20
    x, y, g = _adj_case(m, n, M, 1e-6, prec, 2025)
    p = api.Plan2D(m, n, x, y, 1e-6, precision=prec)
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    C = p.adjoint(torch.tensor(g, dtype=cdt, device="cuda")).cpu().numpy()
    P = lowrank.plan2d(m, n, x, y, 1e-6, p.Lx, p.Ly)
    assert_close(C, lowrank.nufft2_2d_adjoint(P, g), prec, scale=1 if prec == "f32" else 10, what="adjoint")
    r = np.random.default_rng(2026)
    k1, k2 = r.integers(0, m, 64), r.integers(0, n, 64)
    Cd = direct.nudft2_2d_adjoint(x, y, g, m, n, k1, k2)
    tol = 5e-6 if prec == "f32" else 1e-6 * (1 + 1e-6 / 4) + 1e-13
    assert np.max(np.abs(C[k1, k2] - Cd)) <= tol * np.sum(np.abs(g))
