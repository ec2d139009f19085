"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (each follows from the rounding of the path it checks):
  FP64 exec  vs the low-rank oracle: ||df||_2 / ||f||_2 <= 1e-13 and every
             |df_j| <= 1e-12 rms(f) (same method, rounding only); vs the direct sum:
             |df|_inf <= (eps + 1e-13) ||c||_1.
  FP32 exec  vs the low-rank oracle: ||df||_2 / ||f||_2 <= 1e-5 and every
             |df_j| <= 3e-5 rms(f) (FP32 FFT rounding, ~u log2 L; tests/parity.py);
             vs the direct sum: |df|_inf <= max(eps, 5e-6) ||c||_1, the forward's and
             the adjoint's (with ||g||_1) alike.
  Integer plan results (t) and the FP64 perturbations d: bit-exact.
"""

import math

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


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _cdt(prec):
    return torch.complex64 if prec == "f32" else torch.complex128


def _cast(c, prec):
    """The coefficients the GPU sees (FP32 runs round them; the oracle uses the same values)."""
    return c.astype(np.complex64).astype(np.complex128) if prec == "f32" else c


TOL_REL = {"f32": 1e-5, "f64": 1e-13}


def _samples(kind, n, seed):
    return {"uniform": lambda: wl.samples_uniform(n, seed),
            "perturbed": lambda: wl.samples_perturbed(n, seed, 0.5),
            "equispaced": lambda: wl.samples_equispaced(n),
            "wide": lambda: 20.0 * wl.samples_uniform(n, seed) - 10.0,
            "worst": lambda: wl.samples_worst(n, 1 / 8)}[kind]()


# ---- plan: eqs. (2.8)-(2.9), gamma, K, a_pr -------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "perturbed", "wide", "equispaced"])
@pytest.mark.parametrize("N,L,M", [(4096, 0, 4096), (3000, 0, 5000), (1000, 2048, 777)])
def test_plan_matches_oracle(api, kind, N, L, M):
    x = _samples(kind, M, 3)
    if kind == "equispaced":
        x = wl.samples_equispaced(N)[: M] if M <= N else np.arange(M) / N
    plan = api.Plan(N, x, 1e-9, "f64", L=L)
    P = lowrank.plan(N, x, 1e-9, plan.L)
    t, d, alpha = plan.export()
    assert np.array_equal(t.cpu().numpy(), P.t.astype(np.int32))
    assert np.array_equal(d.cpu().numpy(), P.d)             # bit-exact FP64
    assert plan.gamma == P.gamma
    assert plan.K == P.K
    if P.gamma > 0:
        ipow = (1j) ** np.arange(P.K)
        assert np.max(np.abs(alpha * ipow[None, :] - P.a)) <= 1e-15


def test_plan_rejects_nonfinite(api):
    x = wl.samples_uniform(100, 4)
    x[17] = np.nan
    with pytest.raises(api.NufftError) as e:
        api.Plan(128, x, 1e-9, "f32")
    assert e.value.code == -1
    x[17] = 1e300
    with pytest.raises(api.NufftError):
        api.Plan(128, x, 1e-9, "f32")


# ---- forward -----------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["uniform", "equispaced"])
def test_c1_against_direct(api, prec, kind):
    # 1D NUFFT-II at N = 4096, eps = 1e-12: full comparison with the direct sum.
    N, eps = 4096, 1e-12
    x = wl.samples_uniform(N, 1) if kind == "uniform" else wl.samples_equispaced(N)
    c = _cast(wl.coeffs_cn(N, 1), prec)
    plan = api.Plan(N, x, eps, prec)
    f = plan.forward(_dev(c, _cdt(prec))).cpu().numpy()
    fd = direct.nudft2(x, c)
    tol = (eps + 1e-13) if prec == "f64" else max(eps, 5e-6)
    assert np.max(np.abs(f - fd)) <= tol * np.sum(np.abs(c))
    if kind == "equispaced":
        assert plan.K == 1
        assert _rel2(f, np.fft.fft(c)) <= TOL_REL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["uniform", "perturbed", "wide", "worst"])
@pytest.mark.parametrize("N,L,M,eps", [(4096, 0, 4096, 1e-9), (3000, 0, 4100, 1e-4),
                                       (1000, 1024, 777, 1e-12), (2048, 4096, 3000, 1e-14),
                                       (50000, 0, 65536, 1e-9), (1, 0, 5, 1e-9), (17, 0, 1, 1e-6)])
def test_forward_against_oracle(api, prec, kind, N, L, M, eps):
    x = _samples(kind, M, 5)
    c = _cast(wl.coeffs_cn(N, 5), prec)
    plan = api.Plan(N, x, eps, prec, L=L)
    f = plan.forward(_dev(c, _cdt(prec))).cpu().numpy()
    P = lowrank.plan(N, x, eps, plan.L)
    assert plan.K == P.K
    fo = lowrank.nufft2(P, c)
    assert_close(f, fo, prec, what="forward")


def test_zero_samples(api):
    plan = api.Plan(64, np.zeros(0), 1e-9, "f32")
    c = _dev(wl.coeffs_cn(64, 6), torch.complex64)
    assert plan.forward(c).numel() == 0
    g = torch.zeros(0, dtype=torch.complex64, device="cuda")
    assert torch.count_nonzero(plan.adjoint(g)).item() == 0


# ---- adjoint (A^H) and the paper's type I (A^T) ----------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("N,L,M,eps", [(4096, 0, 4096, 1e-9), (3000, 0, 5000, 1e-12),
                                       (1000, 2048, 777, 1e-6), (65536, 0, 65536, 1e-9)])
def test_adjoint_against_oracle(api, prec, N, L, M, eps):
    x = wl.samples_uniform(M, 7)
    g = _cast(wl.cotangent_cn(M, 7), prec)
    plan = api.Plan(N, x, eps, prec, L=L)
    c = plan.adjoint(_dev(g, _cdt(prec))).cpu().numpy()
    P = lowrank.plan(N, x, eps, plan.L)
    assert_close(c, lowrank.nufft2_adjoint(P, g), prec, what="adjoint")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["uniform", "perturbed"])
def test_c1_adjoint_against_direct(api, prec, kind):
    """The adjoint at N = M = 4096, eps = 1e-12, every output against the direct adjoint
    sum: |dc|_inf <= (eps + 1e-13) ||g||_1 in FP64, max(eps, 5e-6) ||g||_1 in FP32 (each
    entry of A^H - A_K^H is bounded by eps, as for the forward)."""
    N, eps = 4096, 1e-12
    x = _samples(kind, N, 31)
    g = _cast(wl.cotangent_cn(N, 31), prec)
    plan = api.Plan(N, x, eps, prec)
    ah = plan.adjoint(_dev(g, _cdt(prec))).cpu().numpy()
    ref = direct.nudft2_adjoint(x, g, N)
    tol = (eps + 1e-13) if prec == "f64" else max(eps, 5e-6)
    assert np.max(np.abs(ah - ref)) <= tol * np.sum(np.abs(g))
    assert_close(ah, lowrank.nufft2_adjoint(lowrank.plan(N, x, eps, plan.L), g), prec, what="adjoint")


def test_adjoint_against_direct_and_inner_product(api):
    N, M, eps = 2048, 3000, 1e-12
    x = wl.samples_uniform(M, 8)
    c = wl.coeffs_cn(N, 8)
    g = wl.cotangent_cn(M, 8)
    plan = api.Plan(N, x, eps, "f64")
    f = plan.forward(_dev(c, torch.complex128)).cpu().numpy()
    ah = plan.adjoint(_dev(g, torch.complex128)).cpu().numpy()
    assert np.max(np.abs(ah - direct.nudft2_adjoint(x, g, N))) <= (eps + 1e-13) * np.sum(np.abs(g))
    lhs, rhs = np.vdot(g, f), np.vdot(ah, c)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(f) * np.linalg.norm(g)
    # section 3.1: F~1 = F~2^T, conj(A^H conj(g))
    at = plan.transpose(_dev(g, torch.complex128)).cpu().numpy()
    assert _rel2(at, lowrank.nufft1(lowrank.plan(N, x, eps), g)) <= 1e-13


# ---- derivative with respect to x ----------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dx_against_oracle(api, prec):
    N, M, eps = 4096, 3000, 1e-10
    x = wl.samples_uniform(M, 9)
    c = _cast(wl.coeffs_cn(N, 9), prec)
    g = _cast(wl.cotangent_cn(M, 9), prec)
    plan = api.Plan(N, x, eps, prec)
    gx = plan.dx(_dev(c, _cdt(prec)), _dev(g, _cdt(prec))).cpu().numpy().astype(np.float64)
    ref = lowrank.nufft2_dx(lowrank.plan(N, x, eps), c, g)
    assert _rel2(gx, ref) <= TOL_REL[prec] * 10
    exact = np.real(np.conj(g) * direct.nudft2_deriv(x, c))
    assert np.max(np.abs(gx - exact)) <= max(eps, 5e-6 if prec == "f32" else 1e-13) * \
        2 * math.pi * N * np.sum(np.abs(c)) * np.max(np.abs(g))
    # accumulate flag
    gx2 = torch.full((M,), 1.5, dtype=plan.rdtype, device="cuda")
    plan.dx(_dev(c, _cdt(prec)), _dev(g, _cdt(prec)), gx2, accumulate=True)
    assert np.allclose(gx2.cpu().numpy() - 1.5, gx, rtol=1e-5, atol=1e-3 * np.max(np.abs(gx)) * TOL_REL[prec])


# ---- full-size workload: N = M = 2^20, eps = 1e-9 ----------------------------------------

@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["perturbed", "uniform"])
def test_full_size_against_oracle(api, prec, kind):
    N = 1 << 20
    x = _samples(kind, N, 10)
    c = _cast(wl.coeffs_cn(N, 10), prec)
    plan = api.Plan(N, x, 1e-9, prec)
    assert plan.K == 12
    f = plan.forward(_dev(c, _cdt(prec))).cpu().numpy()
    P = lowrank.plan(N, x, 1e-9, plan.L)
    assert_close(f, lowrank.nufft2(P, c), prec, what="forward")
    # a seeded subset of rows against the direct sum: 4096 at the benchmark's own
    # configuration (FP32, perturbed grid), 256 elsewhere
    nrows = 4096 if (prec, kind) == ("f32", "perturbed") else 256
    rows = np.random.default_rng(10).choice(N, nrows, replace=False)
    fd = direct.nudft2(x[rows], c)
    tol = (1e-9 + 1e-13) if prec == "f64" else 5e-6
    assert np.max(np.abs(f[rows] - fd)) <= tol * np.sum(np.abs(c))
    # adjoint at full size: every output against the oracle, and a seeded subset of
    # frequencies (1024 at the benchmark's configuration, 256 elsewhere) against the
    # direct adjoint sum within the same bound with ||g||_1
    g = _cast(wl.cotangent_cn(N, 10), prec)
    ah = plan.adjoint(_dev(g, _cdt(prec))).cpu().numpy()
    assert_close(ah, lowrank.nufft2_adjoint(P, g), prec, what="adjoint")
    ks = np.random.default_rng(11).choice(N, 1024 if nrows == 4096 else 256, replace=False)
    assert np.max(np.abs(ah[ks] - direct.nudft2_adjoint_at(x, g, ks))) <= tol * np.sum(np.abs(g))


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["perturbed", "uniform"])
@pytest.mark.parametrize("eps", [1e-4, 1e-14])
def test_full_size_eps_sweep(api, prec, kind, eps):
    """N = M = 2^20 at the two other accuracies of the 2^20 workload: eps = 1e-4 (K = 8) and
    eps = 1e-14 (K = 16, Table 2.1's cap), both sample distributions, both precisions.
    Forward and adjoint element by element against the low-rank oracle; 256 rows and 256
    frequencies against the direct sums within (eps + 1e-13) ||.||_1 (FP64) or
    max(eps, 5e-6) ||.||_1 (FP32)."""
    N = 1 << 20
    x = _samples(kind, N, 40)
    c = _cast(wl.coeffs_cn(N, 40), prec)
    g = _cast(wl.cotangent_cn(N, 41), prec)
    plan = api.Plan(N, x, eps, prec)
    P = lowrank.plan(N, x, eps, plan.L)
    assert plan.K == P.K == {1e-4: 8, 1e-14: 16}[eps]
    f = plan.forward(_dev(c, _cdt(prec))).cpu().numpy()
    assert_close(f, lowrank.nufft2(P, c), prec, what="forward")
    ah = plan.adjoint(_dev(g, _cdt(prec))).cpu().numpy()
    assert_close(ah, lowrank.nufft2_adjoint(P, g), prec, what="adjoint")
    tol = (eps + 1e-13) if prec == "f64" else max(eps, 5e-6)
    rows = np.random.default_rng(42).choice(N, 256, replace=False)
    assert np.max(np.abs(f[rows] - direct.nudft2(x[rows], c))) <= tol * np.sum(np.abs(c))
    assert np.max(np.abs(ah[rows] - direct.nudft2_adjoint_at(x, g, rows))) <= tol * np.sum(np.abs(g))


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("gamma", [0.5, 1 / 8, 1 / 32, 0.0])
def test_full_size_worst_grid_closed_form(api, prec, gamma):
    """Section 2.4's worst grid at N = 2^20: each half is a shifted uniform grid, so the
    exact transform of the whole vector is one FFT per half (a closed form, no oracle
    involved); the error bound ||A - A_K||_max <= eps gives |df|_inf <= eps ||c||_1
    (section 2.4's bounds, plus the FP32 rounding of the FFT in single precision)."""
    N = 1 << 20
    x = wl.samples_worst(N, gamma)
    c = _cast(wl.coeffs_cn(N, 12), prec)
    plan = api.Plan(N, x, 1e-9, prec)
    assert plan.gamma == pytest.approx(gamma, abs=1e-12)
    assert plan.K == lowrank.choose_K(1e-9, plan.gamma)
    f = plan.forward(_dev(c, _cdt(prec))).cpu().numpy()
    k = np.arange(N)
    cc = c.astype(np.complex128)
    plus = np.fft.fft(cc * np.exp(-2j * math.pi * gamma * k / N))
    minus = np.fft.fft(cc * np.exp(2j * math.pi * gamma * k / N))
    ref = np.where(k <= N // 2, plus, minus)
    tol = (1e-9 + 1e-13) if prec == "f64" else 5e-6
    assert np.max(np.abs(f - ref)) <= tol * np.sum(np.abs(cc))
    # the 2-norm form of the same bound: ||df||_2 <= N eps ||c||_2, plus FP32 FFT rounding
    rnd = 1e-13 if prec == "f64" else TOL_REL[prec]
    assert np.linalg.norm(f - ref) <= N * 1e-9 * np.linalg.norm(cc) + rnd * np.linalg.norm(ref)


# ---- unfused comparator, host path, batch, determinism -------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unfused_equals_fused(api, prec):
    N, M = 8192, 10000
    x = wl.samples_uniform(M, 11)
    c = _cast(wl.coeffs_cn(N, 11), prec)
    plan = api.Plan(N, x, 1e-9, prec, unfused=True)
    cd = _dev(c, _cdt(prec))
    fu = plan.forward_unfused(cd).cpu().numpy()
    ff = plan.forward(cd).cpu().numpy()
    assert _rel2(fu, ff) <= TOL_REL[prec] * 2
    plan2 = api.Plan(N, x, 1e-9, prec)
    with pytest.raises(api.NufftError) as e:
        plan2.forward_unfused(cd)
    assert e.value.code == -5


def test_host_path_and_batch(api):
    N, M, B = 4096, 5000, 5
    x = wl.samples_uniform(M, 12)
    plan = api.Plan(N, x, 1e-9, "f32")
    cs = np.stack([wl.coeffs_cn(N, 100 + b) for b in range(B)]).astype(np.complex64)
    cd = _dev(cs, torch.complex64)
    fb = plan.forward_batch(cd).cpu().numpy()
    for b in range(B):
        assert np.array_equal(fb[b], plan.forward(cd[b].contiguous()).cpu().numpy())
    ch = torch.tensor(cs[0]).pin_memory()
    fh = torch.empty(M, dtype=torch.complex64).pin_memory()
    plan.forward_host(ch, fh)
    assert np.array_equal(fh.numpy(), fb[0])


def test_deterministic(api):
    N, M = 65536, 70000
    x = wl.samples_uniform(M, 13)
    plan = api.Plan(N, x, 1e-9, "f32")
    c = _dev(wl.coeffs_cn(N, 13), torch.complex64)
    g = _dev(wl.cotangent_cn(M, 13), torch.complex64)
    assert torch.equal(plan.forward(c), plan.forward(c))
    assert torch.equal(plan.adjoint(g), plan.adjoint(g))
    # a second plan on the same samples gives the same bits
    plan2 = api.Plan(N, x, 1e-9, "f32")
    assert torch.equal(plan.forward(c), plan2.forward(c))


# ---- the forward with its x-derivative in one exec, and autograd ---------------------------

@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("N,L,M,kind", [(4096, 0, 4096, "uniform"), (3000, 0, 5000, "perturbed"),
                                        (1000, 2048, 777, "uniform"), (1 << 20, 0, 1 << 20, "perturbed"),
                                        (5, 0, 9, "equispaced")])
def test_forward_deriv_against_oracle(api, prec, N, L, M, kind):
    x = _samples(kind, M, 21) if kind != "equispaced" else np.arange(M) / N
    c = _cast(wl.coeffs_cn(N, 21), prec)
    plan = api.Plan(N, x, 1e-9, prec, L=L)
    f, fp = plan.forward_deriv(_dev(c, _cdt(prec)))
    P = lowrank.plan(N, x, 1e-9, plan.L)
    assert_close(f.cpu().numpy(), lowrank.nufft2(P, c), prec, what="f")
    ref = lowrank.nufft2(P, -2j * math.pi * np.arange(N) * c)
    assert_close(fp.cpu().numpy(), ref, prec, scale=10, what="f'")
    # the plain forward gives the same f
    assert _rel2(f.cpu().numpy(), plan.forward(_dev(c, _cdt(prec))).cpu().numpy()) <= TOL_REL[prec]


def test_grad_x_matches_dx(api):
    N, M = 4096, 5000
    x = wl.samples_uniform(M, 22)
    c = _dev(wl.coeffs_cn(N, 22).astype(np.complex64), torch.complex64)
    g = _dev(wl.cotangent_cn(M, 22).astype(np.complex64), torch.complex64)
    plan = api.Plan(N, x, 1e-9, "f32")
    f, fp = plan.forward_deriv(c)
    gx = plan.grad_x(g, fp).cpu().numpy()
    ref = np.real(np.conj(g.cpu().numpy()) * fp.cpu().numpy())
    assert np.max(np.abs(gx - ref)) <= 1e-6 * np.max(np.abs(ref))
    gx2 = plan.dx(c, g).cpu().numpy()
    assert np.linalg.norm(gx - gx2) <= 1e-5 * np.linalg.norm(gx2)
    acc = torch.full((M,), 2.0, dtype=torch.float32, device="cuda")
    plan.grad_x(g, fp, acc, accumulate=True)
    assert np.allclose(acc.cpu().numpy() - 2.0, gx, rtol=1e-5, atol=1e-5 * np.max(np.abs(gx)))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_autograd_against_oracle(api, prec):
    # loss = sum |f - f_target|^2 for a batch of coefficient vectors sharing x
    N, M, B = 4096, 4096, 4
    x = wl.samples_uniform(M, 23)
    cs = np.stack([_cast(wl.coeffs_cn(N, 300 + b), prec) for b in range(B)])
    ct = _cast(wl.coeffs_cn(N, 399), prec)
    cdt = _cdt(prec)
    plan = api.Plan(N, x, 1e-10, prec)
    ftarget = plan.forward(_dev(ct, cdt))
    xt = torch.tensor(x, dtype=torch.float64, device="cuda", requires_grad=True)
    c = _dev(cs, cdt).requires_grad_(True)
    f = api.nufft2(c, xt, plan=plan)
    loss = ((f - ftarget[None, :]).abs() ** 2).sum()
    loss.backward()
    P = lowrank.plan(N, x, 1e-10, plan.L)
    ftn = lowrank.nufft2(P, ct)
    gc_ref, gx_ref = [], np.zeros(M)
    for b in range(B):
        fb = lowrank.nufft2(P, cs[b])
        gb = 2.0 * (fb - ftn)                      # torch's gradient of |f - f*|^2 w.r.t. f
        gc_ref.append(lowrank.nufft2_adjoint(P, gb))
        gx_ref += lowrank.nufft2_dx(P, cs[b], gb)
    tol = 1e-4 if prec == "f32" else 1e-10
    assert _rel2(c.grad.cpu().numpy(), np.stack(gc_ref)) <= tol
    assert _rel2(xt.grad.cpu().numpy(), gx_ref) <= tol


def test_autograd_finite_differences_fp64(api):
    # central differences of the loss in x (h = 1e-6) and in c, on the FP64 path at N = 200
    N, M = 200, 150
    x = wl.samples_uniform(M, 24)
    c0 = wl.coeffs_cn(N, 24)
    g0 = wl.cotangent_cn(M, 24)

    def loss_of(xv, cv):
        plan = api.Plan(N, xv, 1e-13, "f64")
        f = plan.forward(_dev(cv, torch.complex128)).cpu().numpy()
        return float(np.real(np.vdot(g0, f)))

    plan = api.Plan(N, x, 1e-13, "f64")
    xt = torch.tensor(x, dtype=torch.float64, device="cuda", requires_grad=True)
    c = _dev(c0, torch.complex128).requires_grad_(True)
    f = api.nufft2(c, xt, plan=plan)
    (torch.conj(_dev(g0, torch.complex128)) * f).real.sum().backward()
    h = 1e-6
    for j in (0, 37, 149):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (loss_of(xp, c0) - loss_of(xm, c0)) / (2 * h)
        assert abs(xt.grad[j].item() - fd) <= 1e-5 * max(1.0, abs(fd))
    for k in (0, 99):
        e = np.zeros(N, complex)
        e[k] = 1.0
        fd_re = (loss_of(x, c0 + h * e) - loss_of(x, c0 - h * e)) / (2 * h)
        # torch's complex gradient: d loss / d Re c_k = Re(grad_k)
        assert abs(c.grad[k].real.item() - fd_re) <= 1e-6 * max(1.0, abs(fd_re))


def test_autograd_training_batch_n2e18(api):
    """The differentiable workload at its full size: N = M = 2^18, a batch of 64 complex64
    coefficient vectors sharing uniform x, loss = sum |f - f*|^2 with f* = A c* for a
    seeded c*.  dL/dc of every batch member, element by element, against the FP64 oracle
    gradient 2 A^H (A c - A c*); dL/dx at every sample against the oracle's
    sum_b Re(conj(g_b) f'_b), and on 32 sampled rows against the direct derivative sum of
    eq. (1.2) summed over the whole batch."""
    N = M = 1 << 18
    B = 64
    x = wl.samples_uniform(M, 2024)
    cs = np.stack([wl.coeffs_cn(N, 500 + b).astype(np.complex64) for b in range(B)])
    ct = wl.coeffs_cn(N, 599).astype(np.complex64)
    plan = api.Plan(N, x, 1e-9, "f32")
    ftarget = plan.forward(_dev(ct, torch.complex64))
    xt = torch.tensor(x, dtype=torch.float64, device="cuda", requires_grad=True)
    c = _dev(cs, torch.complex64).requires_grad_(True)
    f = api.nufft2(c, xt, plan=plan)
    loss = ((f - ftarget[None, :]).abs() ** 2).sum()
    loss.backward()
    gc = c.grad.cpu().numpy()
    gxg = xt.grad.cpu().numpy()
    fg = f.detach().cpu().numpy()
    ftg = ftarget.cpu().numpy()
    # dL/dc against the FP64 oracle for every member, and dL/dx summed over them (the
    # cotangent g_b = 2 (f_b - f*) is taken from the GPU's own f, as autograd does)
    P = lowrank.plan(N, x, 1e-9, plan.L)
    ft64 = lowrank.nufft2(P, ct.astype(np.complex128))
    gx_or = np.zeros(M)
    for b in range(B):
        gb = 2.0 * (lowrank.nufft2(P, cs[b].astype(np.complex128)) - ft64)
        assert_close(gc[b], lowrank.nufft2_adjoint(P, gb), "f32", scale=10, what="dL/dc %d" % b)
        gx_or += lowrank.nufft2_dx(P, cs[b].astype(np.complex128),
                                   2.0 * (fg[b].astype(np.complex128) - ftg.astype(np.complex128)))
    assert_close(gxg, gx_or, "f32", scale=10, what="dL/dx")
    # dL/dx on sampled rows: sum_b Re(conj(g_bj) f'_bj), f' by the direct derivative sum
    rows = np.arange(0, M, M // 32)
    ref = np.zeros(rows.size)
    for b in range(B):
        gb = 2.0 * (fg[b, rows].astype(np.complex128) - ftg[rows])
        fpb = direct.nudft2_deriv(x[rows], cs[b].astype(np.complex128))
        ref += np.real(np.conj(gb) * fpb)
    assert _rel2(gxg[rows], ref) <= 1e-4


@pytest.mark.parametrize("prec,N", [("f32", 4096), ("f32", 3000), ("f64", 4096), ("f32", 1 << 19)])
def test_batch_calls_match_single_calls(api, prec, N):
    """nufft2_exec_batch / nufft1_exec_batch / nufft2_exec_deriv_batch: one launch per
    pass for a batch sharing x (FP32 grids up to 2^18), else member by member; both
    must equal the single-vector calls bit for bit; grad_x_batch sums the members."""
    B, M = 6, N + 123
    x = wl.samples_uniform(M, 70)
    cdt = _cdt(prec)
    plan = api.Plan(N, x, 1e-9, prec)
    c = _dev(np.stack([_cast(wl.coeffs_cn(N, 700 + b), prec) for b in range(B)]), cdt)
    g = _dev(np.stack([wl.cotangent_cn(M, 800 + b) for b in range(B)]).astype(np.complex64 if prec == "f32"
                                                                                else np.complex128), cdt)
    f = plan.forward_batch(c)
    gc = plan.adjoint_batch(g)
    fd, fpd = plan.forward_deriv_batch(c)
    for b in (0, B - 1):
        assert torch.equal(f[b], plan.forward(c[b].contiguous())), b
        assert torch.equal(gc[b], plan.adjoint(g[b].contiguous())), b
        f1, fp1 = plan.forward_deriv(c[b].contiguous())
        assert torch.equal(fd[b], f1) and torch.equal(fpd[b], fp1), b
    gx = plan.grad_x_batch(g, fpd)
    ref = sum(plan.grad_x(g[b].contiguous(), fpd[b].contiguous()).double() for b in range(B))
    tol = 1e-5 if prec == "f32" else 1e-12
    assert float((gx.double() - ref).abs().max() / ref.abs().max()) <= tol
    # a larger batch reallocates the workspace; results stay the same
    c2 = torch.cat([c, c])
    assert torch.equal(plan.forward_batch(c2)[B:], f)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_step_host_matches_device_calls(api, prec):
    """nufft2_step_host (host buffers, overlapped copies) returns what the device calls do."""
    N, M = 5000, 6000
    x = wl.samples_perturbed(M, 71, 0.5) * (N / M)
    plan = api.Plan(N, x, 1e-9, prec)
    cdt, rdt = _cdt(prec), (torch.float32 if prec == "f32" else torch.float64)
    c = torch.tensor(_cast(wl.coeffs_cn(N, 72), prec).astype(np.complex64 if prec == "f32" else np.complex128))
    g = torch.tensor(wl.cotangent_cn(M, 73).astype(np.complex64 if prec == "f32" else np.complex128))
    ch, gh = c.pin_memory(), g.pin_memory()
    fh = torch.empty(M, dtype=cdt).pin_memory()
    gch = torch.empty(N, dtype=cdt).pin_memory()
    gxh = torch.empty(M, dtype=rdt).pin_memory()
    cd, gd = c.cuda(), g.cuda()
    f_ref, fp_ref = plan.forward_deriv(cd)
    gc_ref = plan.adjoint(gd)
    gx_ref = plan.grad_x(gd, fp_ref)
    for _ in range(2):
        plan.step_host(ch, gh, fh, gch, gxh)
        torch.cuda.synchronize()
        assert torch.equal(fh, f_ref.cpu())
        assert torch.equal(gch, gc_ref.cpu())
        assert torch.equal(gxh, gx_ref.cpu())
