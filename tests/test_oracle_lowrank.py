"""Pins for the low-rank oracle against what the paper and the mathematics fix.

* Table 2.1's ranks (golden fixture) and the bound of eq. (2.7).
* Fig. 2.1's rounding example (golden fixture).
* Theorem A.2: ||A - A_K||_max <= eps, by brute force against the dense A.
* Section 2.4's error bounds against the direct sum (an independent oracle).
* gamma = 0 reduces to the FFT (section 2.1.2); the worst grid of section 2.4 has a
  closed form through a library FFT.
* A^H is the adjoint; the type-I transform of section 3.1 is the transpose.
* The x-derivative against finite differences and torch autograd of a direct sum.
* Planted mistakes (phase sign, primes, the i^r factor) fail the brute-force pin.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import direct, lowrank
from paper_1701_04492_gb300 import workloads as wl


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return json.load(fh)


# --- K -----------------------------------------------------------------------

@pytest.mark.parametrize("row", ["single", "half"])
def test_table_2_1_rows_reproduced(golden_dir, row):
    tab = _load(golden_dir, "table_2_1.json")
    edges = tab["gamma_band_upper_edges"]
    want = tab["rows"][row]["K"]
    got = [lowrank.choose_K(tab["rows"][row]["eps"], g) for g in edges]
    assert got == want


def test_table_2_1_double_row_is_the_cap(golden_dir):
    tab = _load(golden_dir, "table_2_1.json")
    edges = tab["gamma_band_upper_edges"]
    want = tab["rows"]["double"]["K"]
    got = [lowrank.choose_K(tab["rows"]["double"]["eps"], g) for g in edges]
    assert got == want
    # Strictly inside a band the rank never exceeds the band's table entry.
    for lo, hi, K in zip(edges[:-1], edges[1:], want[1:]):
        assert lowrank.choose_K(1e-300 + 2.2e-16, 0.5 * (lo + hi)) <= K


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-7, 1e-9, 1e-12, 1e-14])
@pytest.mark.parametrize("gamma", [1 / 64, 1 / 8, 0.3, 0.5])
def test_rank_within_eq_2_7(eps, gamma):
    # Eq. (2.7) is a sufficient rank; the tail rule picks the smallest rank that
    # satisfies the same triangle-inequality bound, so it can only be smaller.
    assert lowrank.choose_K(eps, gamma) <= lowrank.lambert_w_rank(eps, gamma)


def _eq_2_7_root(eps, gamma):
    """The u > 5 gamma with u log(u / (5 gamma)) = log(140 / eps), by bisection.

    With z = log(140/eps) / (5 gamma) and u = 5 gamma e^{W(z)}: W(z) = log(u / (5 gamma))
    and W e^W = z give u log(u / (5 gamma)) = log(140 / eps), i.e. 140 (5 gamma / u)^u = eps,
    the bound in the proof of Lemma A.1 solved for the rank.  No Lambert W is evaluated,
    so this pins the oracle's use of W (its branch, its argument) from outside."""
    lo, hi = 5.0 * gamma, 1e4
    target = math.log(140.0 / eps)
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if mid * math.log(mid / (5.0 * gamma)) > target:
            hi = mid
        else:
            lo = mid
    return hi


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-9, 1e-12, 1e-14, 2.2e-16])
@pytest.mark.parametrize("gamma", [1 / 64, 1 / 32, 1 / 8, 0.25, 0.3, 0.5])
def test_eq_2_7_against_its_defining_equation(eps, gamma):
    """lambert_w_rank is eq. (2.7): max{3, ceil(u)} for the root u of the bound it inverts."""
    u = _eq_2_7_root(eps, gamma)
    assert lowrank.lambert_w_rank(eps, gamma) == max(3, math.ceil(u))
    # the root does satisfy 140 (5 gamma / u)^u = eps
    assert math.isclose(140.0 * (5.0 * gamma / u) ** u, eps, rel_tol=1e-9)


def test_eq_2_7_hand_values():
    """Eq. (2.7) evaluated by hand at gamma = 1/2: for eps = 1e-9, log(140/eps) = 25.665;
    u = 14.564 solves u log(u / 2.5) = 25.665 (14.564 x 1.7623 = 25.666), so K = 15.  The
    same at eps = 1e-4 (u = 10.12: 10.12 x 1.3983 = 14.152 = log(1.4e6)) gives K = 11, and the
    floor of 3 applies where u < 3 (eps = 1e-2, gamma = 1/64: u = 2.70)."""
    assert lowrank.lambert_w_rank(1e-9, 0.5) == 15
    assert lowrank.lambert_w_rank(1e-4, 0.5) == 11
    assert lowrank.lambert_w_rank(1e-2, 1 / 64) == 3
    # a plausible slip, log in place of W, gives another rank at the metric workload
    z = math.log(140.0 / 1e-9) / 2.5
    assert max(3, math.ceil(2.5 * math.exp(math.log(z)))) != 15


def test_rank_at_the_metric_workload():
    # gamma -> 1/2, eps = 1e-9: K = 12, and 11 does not suffice.
    assert lowrank.choose_K(1e-9, 0.5) == 12
    assert lowrank.tail_bound(11, 0.5) > 1e-9


def test_rank_monotone_in_gamma_and_eps():
    gs = np.linspace(1e-3, 0.5, 40)
    for eps in (1e-4, 1e-9, 1e-14):
        Ks = [lowrank.choose_K(eps, g) for g in gs]
        assert all(a <= b for a, b in zip(Ks, Ks[1:]))
    for g in (0.1, 0.5):
        Ks = [lowrank.choose_K(e, g) for e in (1e-2, 1e-4, 1e-8, 1e-12)]
        assert all(a <= b for a, b in zip(Ks, Ks[1:]))


# --- rounding (eqs. (2.8)-(2.9)) ------------------------------------------------

def test_fig_2_1_example(golden_dir):
    fig = _load(golden_dir, "fig_2_1.json")
    N = fig["N"]
    x = np.array(fig["x_times_N_as_drawn"]) / N
    s, t, delta = lowrank.round_to_grid(x, N)
    assert s.tolist() == fig["s_arrow_targets_as_drawn"]
    assert t.tolist() == fig["t_from_eq_2_9"]
    assert np.all(np.abs(delta) <= 0.5)


def test_rounding_ties_wrap_and_negative():
    L = 16
    x = np.array([0.5 / L, 1.5 / L, 1.0, -0.25 / L, -3.0 - 1.0 / L, 15.5 / L, 7.0 + 3.0 / L])
    s, t, delta = lowrank.round_to_grid(x, L)
    assert s.tolist() == [0, 2, 16, 0, -49, 16, 115]     # ties to even
    assert t.tolist() == [0, 2, 0, 0, 15, 0, 3]          # Euclidean mod
    assert np.all(np.abs(delta) <= 0.5)
    assert np.all(L * x == s + delta)


# --- Theorem A.2 by brute force ------------------------------------------------

SAMPLE_SETS = {
    "uniform": lambda n, L: wl.samples_uniform(n, 21),
    "perturbed": lambda n, L: wl.samples_perturbed(n, 22, 0.5),
    "perturbed_1/8": lambda n, L: wl.samples_perturbed(n, 23, 0.125),
    "worst_1/32": lambda n, L: wl.samples_worst(n, 1 / 32),
    "wide": lambda n, L: 10.0 * wl.samples_uniform(n, 24) - 5.0,
}


@pytest.mark.parametrize("name", sorted(SAMPLE_SETS))
@pytest.mark.parametrize("eps", [1e-4, 1e-9, 1e-12])
@pytest.mark.parametrize("N,L", [(256, 256), (200, 256), (128, 256), (97, 97)])
def test_low_rank_approximation_bound(name, eps, N, L):
    x = SAMPLE_SETS[name](N, L)
    P = lowrank.plan(N, x, eps, L)
    err = np.max(np.abs(lowrank.dense_A(P) - lowrank.dense_AK(P)))
    assert err <= eps
    assert err <= lowrank.tail_bound(P.K, P.gamma) + 1e-14
    assert P.gamma <= N / (2 * L) + 1e-15


def test_oversampling_lowers_the_rank():
    # Section 2.3: on a grid of 2N points gamma <= 1/4, so double precision needs
    # 13 FFTs of length 2N instead of 16 of length N (Table 2.1).
    N = 1024
    x = wl.samples_uniform(N, 25)
    assert lowrank.plan(N, x, 2.2e-16).K == 16
    assert lowrank.plan(N, x, 2.2e-16, 2 * N).K == 13


def _plant(monkeypatch, what):
    if what == "phase_sign":
        monkeypatch.setattr(lowrank, "phase", lambda d: np.exp(1j * math.pi * np.asarray(d)))
    elif what == "no_primes":
        monkeypatch.setattr(lowrank, "prime_weights", lambda K: np.ones(K))
    elif what == "no_i_power":
        orig = lowrank.bessel_coefficients
        monkeypatch.setattr(lowrank, "bessel_coefficients",
                            lambda K, g: np.abs(orig(K, g)) * np.sign(orig(K, g).real + orig(K, g).imag))
    elif what == "bessel_sign":
        orig = lowrank.bessel_coefficients

        def flipped(K, g):
            return orig(K, -g)
        monkeypatch.setattr(lowrank, "bessel_coefficients", flipped)


@pytest.mark.parametrize("what", ["phase_sign", "no_primes", "no_i_power", "bessel_sign"])
def test_planted_mistakes_break_the_bound(monkeypatch, what):
    N = 128
    x = wl.samples_uniform(N, 26)
    _plant(monkeypatch, what)
    P = lowrank.plan(N, x, 1e-9)
    err = np.max(np.abs(lowrank.dense_A(P) - lowrank.dense_AK(P)))
    assert err > 1e-3


# --- the whole method against the direct sum (section 2.4) ---------------------

@pytest.mark.parametrize("eps", [1e-4, 1e-9, 1e-12])
@pytest.mark.parametrize("name", ["uniform", "perturbed", "wide"])
@pytest.mark.parametrize("N,L", [(4096, 4096), (3000, 4096), (1000, 1000)])
def test_error_bound_against_direct(eps, name, N, L):
    x = SAMPLE_SETS[name](N, L)
    c = wl.coeffs_cn(N, 31)
    P = lowrank.plan(N, x, eps, L)
    f = lowrank.nufft2(P, c)
    fd = direct.nudft2(x, c)
    rounding = 1e-15 * N * math.log2(L)
    # infinity norm: |((A - A_K) o F(t,:)) c|_j <= ||A - A_K||_max ||c||_1
    assert np.max(np.abs(f - fd)) <= (eps + rounding) * np.sum(np.abs(c))
    # 2-norm bound of section 2.4: N eps ||c||_2
    assert np.linalg.norm(f - fd) <= N * (eps + rounding) * np.linalg.norm(c)


def test_gamma_zero_is_one_fft():
    N = 2048
    c = wl.coeffs_cn(N, 32)
    P = lowrank.plan(N, wl.samples_equispaced(N), 1e-12)
    assert P.K == 1 and P.gamma == 0.0
    assert np.array_equal(lowrank.nufft2(P, c), np.fft.fft(c)[P.t])


@pytest.mark.parametrize("N,gamma", [(4096, 0.5), (4096, 1 / 8), (1 << 16, 1 / 32), (1 << 16, 0.5)])
def test_worst_grid_closed_form(N, gamma):
    # Section 2.4's worst grid: each half is a shifted uniform grid, so
    # f_j = FFT(c o exp(-+2 pi i gamma k / N))_j exactly.
    x = wl.samples_worst(N, gamma)
    c = wl.coeffs_cn(N, 33)
    k = np.arange(N)
    plus = np.fft.fft(c * np.exp(-2j * math.pi * gamma * k / N))
    minus = np.fft.fft(c * np.exp(2j * math.pi * gamma * k / N))
    ref = np.where(np.arange(N) <= N // 2, plus, minus)
    for eps in (1e-9, 1e-14):
        P = lowrank.plan(N, x, eps)
        f = lowrank.nufft2(P, c)
        assert np.max(np.abs(f - ref)) <= (eps + 1e-15 * N) * np.sum(np.abs(c))


def test_error_growth_decaying_coefficients():
    # Section 2.4: with c ~ randn / k^2 the error is far below the Gaussian case.
    N = 2048
    x = wl.samples_uniform(N, 34)
    P = lowrank.plan(N, x, 1e-7)
    e_gauss = np.linalg.norm(lowrank.nufft2(P, wl.coeffs_cn(N, 34)) - direct.nudft2(x, wl.coeffs_cn(N, 34)))
    cd = wl.coeffs_decay(N, 34)
    e_decay = np.linalg.norm(lowrank.nufft2(P, cd) - direct.nudft2(x, cd))
    assert e_decay < e_gauss


# --- adjoint, transpose and derivative ----------------------------------------

@pytest.mark.parametrize("N,L,M", [(4096, 4096, 4096), (1000, 1024, 1500), (64, 64, 10)])
def test_adjoint_identity(N, L, M):
    x = wl.samples_uniform(M, 41)
    c = wl.coeffs_cn(N, 41)
    g = wl.cotangent_cn(M, 41)
    P = lowrank.plan(N, x, 1e-9, L)
    lhs = np.vdot(g, lowrank.nufft2(P, c))
    rhs = np.vdot(lowrank.nufft2_adjoint(P, g), c)
    scale = np.linalg.norm(lowrank.nufft2(P, c)) * np.linalg.norm(g)
    assert abs(lhs - rhs) <= 1e-13 * scale


@pytest.mark.parametrize("eps", [1e-6, 1e-12])
def test_adjoint_against_direct(eps):
    N, M = 2048, 3000
    x = wl.samples_uniform(M, 42)
    g = wl.cotangent_cn(M, 42)
    P = lowrank.plan(N, x, eps, 2048)
    c = lowrank.nufft2_adjoint(P, g)
    ref = direct.nudft2_adjoint(x, g, N)
    assert np.max(np.abs(c - ref)) <= (eps + 1e-15 * M) * np.sum(np.abs(g))


def test_type1_is_the_transpose():
    # Section 3.1: F~1 c with (F~1)_jk = exp(-2 pi i (j/N) w_k) equals F~2^T c for
    # samples w_k / N.
    N = 512
    w = N * wl.samples_uniform(N, 43)
    g = wl.cotangent_cn(N, 43)
    P = lowrank.plan(N, w / N, 1e-12)
    f1 = lowrank.nufft1(P, g)
    j = np.arange(N)
    ref = np.exp(-2j * math.pi * np.outer(j, w) / N) @ g
    assert np.max(np.abs(f1 - ref)) <= 1e-11 * np.sum(np.abs(g))


def test_x_derivative_against_direct_and_finite_differences():
    N, M = 200, 120
    x = wl.samples_uniform(M, 44)
    c = wl.coeffs_cn(N, 44)
    g = wl.cotangent_cn(M, 44)
    P = lowrank.plan(N, x, 1e-12, 256)
    gx = lowrank.nufft2_dx(P, c, g)
    ref = np.real(np.conj(g) * direct.nudft2_deriv(x, c))
    assert np.max(np.abs(gx - ref)) <= 1e-9 * np.sum(np.abs(c)) * 2 * math.pi * N
    # central differences of Re<f, g> = Re sum_j conj(g_j) f_j, h = 1e-6 (FP64);
    # truncation (2 pi N h)^2 / 6 ~ 3e-7 relative at N = 200.
    h = 1e-6
    fp = direct.nudft2(x + h, c)
    fm = direct.nudft2(x - h, c)
    fd = np.real(np.conj(g) * (fp - fm)) / (2 * h)
    assert np.max(np.abs(gx - fd)) <= 1e-5 * np.max(np.abs(ref))


def test_x_derivative_against_torch_autograd():
    torch = pytest.importorskip("torch")
    N, M = 96, 50
    x = wl.samples_uniform(M, 45)
    c = wl.coeffs_cn(N, 45)
    g = wl.cotangent_cn(M, 45)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    ct = torch.tensor(c, dtype=torch.complex128, requires_grad=True)
    k = torch.arange(N, dtype=torch.float64)
    f = (torch.exp(-2j * math.pi * xt[:, None] * k[None, :]) * ct[None, :]).sum(1)
    loss = (torch.conj(torch.tensor(g)) * f).real.sum()
    loss.backward()
    P = lowrank.plan(N, x, 1e-13, 128)
    assert np.max(np.abs(lowrank.nufft2_dx(P, c, g) - xt.grad.numpy())) <= 1e-8 * N * N
    # d loss / d c in torch's convention (conjugate Wirtinger, x2) is A^H g.
    gc = ct.grad.numpy()
    assert np.max(np.abs(lowrank.nufft2_adjoint(P, g) - gc)) <= 1e-11 * np.sum(np.abs(g))


# ---- two dimensions (section 4, eq. (4.4)) ----------------------------------------

@pytest.mark.parametrize("m,n", [(16, 24), (32, 8), (40, 40)])
@pytest.mark.parametrize("eps", [1e-4, 1e-9, 1e-12])
def test_2d_within_bound_of_direct_sum(m, n, eps):
    """|f_K - f|_inf <= (eps (1 + eps/4) + rounding) ||C||_1 (the product bound of the
    two directions at eps / 2 each), against the direct 2D sum of eq. (4.1)."""
    M = 300
    x, y = wl.samples_2d_uniform(M, 70 + m)
    r = np.random.default_rng(m * n)
    C = (r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))) / np.sqrt(2)
    P = lowrank.plan2d(m, n, x, y, eps)
    f = lowrank.nufft2_2d(P, C)
    fd = direct.nudft2_2d(x, y, C)
    assert np.max(np.abs(f - fd)) <= (eps * (1 + eps / 4) + 1e-13) * np.sum(np.abs(C))


def test_2d_separable_is_product_of_1d_sums():
    """C = a b^T: f_j = (sum_k1 a_k1 e^{-2 pi i k1 x_j}) (sum_k2 b_k2 e^{-2 pi i k2 y_j}),
    which pins the pairing of k1 with x and k2 with y (m != n)."""
    m, n, M = 24, 40, 200
    x, y = wl.samples_2d_uniform(M, 81)
    a = wl.coeffs_cn(m, 82)
    b = wl.coeffs_cn(n, 83)
    P = lowrank.plan2d(m, n, x, y, 1e-12)
    f = lowrank.nufft2_2d(P, np.outer(a, b))
    ref = direct.nudft2(x, a) * direct.nudft2(y, b)
    assert np.max(np.abs(f - ref)) <= 2e-12 * np.sum(np.abs(a)) * np.sum(np.abs(b))


def test_2d_single_column_is_the_1d_method():
    """n = 1: only k2 = 0, so the 2D transform is the 1D transform of C[:, 0] in x."""
    m, M = 64, 150
    x, y = wl.samples_2d_uniform(M, 84)
    c = wl.coeffs_cn(m, 85)
    P = lowrank.plan2d(m, 1, x, y, 1e-10)
    f = lowrank.nufft2_2d(P, c[:, None])
    assert np.max(np.abs(f - direct.nudft2(x, c))) <= 1.1e-10 * np.sum(np.abs(c))


def test_2d_planted_phase_sign_breaks_the_bound(monkeypatch):
    """The e^{+i pi d} misprint of the Lemma's proof, planted in the oracle, fails the pin."""
    m, n, M = 16, 16, 100
    x, y = wl.samples_2d_uniform(M, 86)
    C = np.outer(wl.coeffs_cn(m, 87), wl.coeffs_cn(n, 88))
    monkeypatch.setattr(lowrank, "phase", lambda d: np.exp(1j * np.pi * np.asarray(d)))
    P = lowrank.plan2d(m, n, x, y, 1e-9)
    f = lowrank.nufft2_2d(P, C)
    assert np.max(np.abs(f - direct.nudft2_2d(x, y, C))) > 1e-3 * np.sum(np.abs(C))


@pytest.mark.parametrize("m,n", [(16, 24), (40, 8)])
@pytest.mark.parametrize("eps", [1e-4, 1e-12])
def test_2d_adjoint_within_bound_of_direct_sum(m, n, eps):
    """The 2D adjoint against the direct conjugate sum of eq. (4.1): each entry of A^H - A_K^H
    is the conjugate of an entry of A - A_K, so |dC|_max <= (eps (1 + eps/4) + rounding) ||g||_1."""
    M = 300
    x, y = wl.samples_2d_uniform(M, 170 + m)
    g = wl.cotangent_cn(M, 171 + n)
    P = lowrank.plan2d(m, n, x, y, eps)
    C = lowrank.nufft2_2d_adjoint(P, g)
    Cd = direct.nudft2_2d_adjoint(x, y, g, m, n)
    assert np.max(np.abs(C - Cd)) <= (eps * (1 + eps / 4) + 1e-13) * np.sum(np.abs(g))


@pytest.mark.parametrize("Lx,Ly", [(None, None), (64, 32)])
def test_2d_adjoint_identity(Lx, Ly):
    """<A C, g> = <C, A^H g> for the oracle's own forward and adjoint (the same factors)."""
    m, n, M = 24, 20, 400
    x, y = wl.samples_2d_uniform(M, 172)
    C = wl.coeffs_cn(m * n, 173).reshape(m, n)
    g = wl.cotangent_cn(M, 174)
    P = lowrank.plan2d(m, n, x, y, 1e-9, Lx, Ly)
    f = lowrank.nufft2_2d(P, C)
    ah = lowrank.nufft2_2d_adjoint(P, g)
    assert abs(np.vdot(g, f) - np.vdot(ah, C)) <= 1e-13 * np.linalg.norm(f) * np.linalg.norm(g)


def test_2d_adjoint_single_column_is_the_1d_adjoint():
    """n = 1: C[:, 0] = sum_j g_j exp(+2 pi i k1 x_j), the 1D adjoint sum in x."""
    m, M = 64, 150
    x, y = wl.samples_2d_uniform(M, 175)
    g = wl.cotangent_cn(M, 176)
    P = lowrank.plan2d(m, 1, x, y, 1e-10)
    C = lowrank.nufft2_2d_adjoint(P, g)
    assert C.shape == (m, 1)
    assert np.max(np.abs(C[:, 0] - direct.nudft2_adjoint(x, g, m))) <= 1.1e-10 * np.sum(np.abs(g))


@pytest.mark.parametrize("what", ["phase_sign", "no_conj"])
def test_2d_adjoint_planted_mistakes_break_the_bound(monkeypatch, what):
    """A planted phase sign, or factors used without their conjugate, fail the direct pin."""
    m, n, M = 16, 16, 100
    x, y = wl.samples_2d_uniform(M, 177)
    g = wl.cotangent_cn(M, 178)
    if what == "phase_sign":
        monkeypatch.setattr(lowrank, "phase", lambda d: np.exp(1j * np.pi * np.asarray(d)))
    else:
        monkeypatch.setattr(lowrank.np, "conj", lambda v: np.asarray(v))
    P = lowrank.plan2d(m, n, x, y, 1e-9)
    C = lowrank.nufft2_2d_adjoint(P, g)
    monkeypatch.undo()
    assert np.max(np.abs(C - direct.nudft2_2d_adjoint(x, y, g, m, n))) > 1e-3 * np.sum(np.abs(g))


def test_direct_adjoint_at_chosen_outputs_is_the_full_sum():
    """The subset forms of the direct adjoint sums return the matching entries of the full ones."""
    M, N, m, n = 200, 96, 12, 10
    x, y = wl.samples_2d_uniform(M, 179)
    g = wl.cotangent_cn(M, 180)
    ks = np.array([0, 1, 50, 95])
    assert np.array_equal(direct.nudft2_adjoint_at(x, g, ks), direct.nudft2_adjoint(x, g, N)[ks])
    Cf = direct.nudft2_2d_adjoint(x, y, g, m, n)
    k1, k2 = np.array([0, 11, 3]), np.array([9, 0, 4])
    assert np.array_equal(direct.nudft2_2d_adjoint(x, y, g, m, n, k1, k2), Cf[k1, k2])
    # and the full 2D adjoint is the conjugate transpose of the dense 2D matrix
    A = np.exp(-2j * np.pi * (np.outer(x, np.repeat(np.arange(m), n)) + np.outer(y, np.tile(np.arange(n), m))))
    assert np.max(np.abs(Cf.ravel() - A.conj().T @ g)) <= 1e-12 * np.sum(np.abs(g))


# ---- inverse NUFFT-II (section 3.3) -------------------------------------------------

def test_toeplitz_product_is_the_dense_normal_matrix():
    """The circulant product equals the dense A^H A applied to a vector (A exact)."""
    N = 96
    x = wl.samples_perturbed(N, 100, 0.25)
    P = lowrank.plan(N, x, 1e-14)
    lam = lowrank.circulant_eigenvalues(lowrank.toeplitz_column(P))
    v = wl.coeffs_cn(N, 101)
    A = np.exp(-2j * np.pi * np.outer(x, np.arange(N)))
    ref = A.conj().T @ (A @ v)
    assert np.max(np.abs(lowrank.toeplitz_apply(lam, v) - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("gamma", [1 / 32, 1 / 8, 1 / 4])
def test_inverse_recovers_coefficients(gamma):
    """f = A c exactly (the direct sum); CG on the normal equations returns c."""
    N = 256
    x = wl.samples_perturbed(N, 102, gamma)
    c = wl.coeffs_cn(N, 103)
    f = direct.nudft2(x, c)
    P = lowrank.plan(N, x, 1e-14)
    cs, it, rr = lowrank.inverse_cg(P, f, 1e-13, 500)
    assert rr <= 1e-13
    assert np.linalg.norm(cs - c) / np.linalg.norm(c) <= 1e-10
    assert it < 100


def test_inverse_on_the_grid_is_the_inverse_fft_in_one_step():
    """gamma = 0: A = F, A^H A = N I, and one CG step gives ifft(f)."""
    N = 128
    x = wl.samples_equispaced(N)
    f = wl.coeffs_cn(N, 104)
    P = lowrank.plan(N, x, 1e-14)
    cs, it, rr = lowrank.inverse_cg(P, f, 1e-13, 10)
    assert it == 1
    assert np.max(np.abs(cs - np.fft.ifft(f))) <= 1e-14 * np.max(np.abs(f))


def test_inverse_iterations_grow_with_gamma():
    """Fig. 3.1: more perturbed samples need more CG iterations (fixed N, seed, tol)."""
    N = 512
    its = []
    for gamma in (0.0, 1 / 32, 1 / 8, 7 / 16):
        x = wl.samples_perturbed(N, 105, gamma) if gamma > 0 else wl.samples_equispaced(N)
        c = wl.coeffs_cn(N, 106)
        P = lowrank.plan(N, x, 1e-14)
        its.append(lowrank.inverse_cg(P, direct.nudft2(x, c), 1e-12, 2000)[1])
    assert its[0] == 1 and its[0] < its[1] <= its[2] < its[3]
