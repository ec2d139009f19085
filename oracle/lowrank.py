"""The paper's low-rank NUFFT, written out step by step on the CPU in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product library never
imports this module.

Notation follows the paper.  N frequencies k = 0..N-1, M samples x_j, coefficients
c in C^N, values f in C^M, working accuracy eps, rank K.

The grid the samples are rounded to has L >= N points.  L = N is the method of
section 2.2; L > N is the oversampling variant of section 2.3 ("Oversampling"),
where the FFTs have length L and the zero-padded coefficients occupy k < N.  With
d_j = (L x_j - s_j) * N / L the perturbation matrix is exactly the section 2.1 form

    A_jk = exp(-2 pi i d_j k / N),       |d_j| <= gamma = max_j |d_j| <= N / (2L),

so every formula below uses d_j and gamma exactly as the paper uses N(x - s/N) and
gamma.  For L = N, d_j is the paper's N x_j - s_j.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import jv

# Table 2.1: the ranks the paper uses in double precision (eps ~ 2.2e-16), by the
# band of gamma.  Its bands are 0, (0,1/32], (1/32,1/16], (1/16,1/8], (1/8,1/4],
# (1/4,1/2].
TABLE_2_1_DOUBLE = ((0.0, 1), (1 / 32, 8), (1 / 16, 9), (1 / 8, 11), (1 / 4, 13), (1 / 2, 16))

# Terms with p or r beyond this are below 1e-60 for gamma <= 1/2; the tail sum of
# choose_K stops here.
TAIL_TERMS = 64


# ---------------------------------------------------------------------------
# Planning stage (section 2.3 "Planning the transform")
# ---------------------------------------------------------------------------

def round_to_grid(x, L):
    """Eqs. (2.8)-(2.9): s = round(L x), t = mod(s, L), delta = L x - s.

    Ties go to the even integer (numpy's rint); the paper allows any tie-break.
    x may be any finite real: the periodicity of exp(-2 pi i x k) lets s leave
    [0, L], and the Euclidean modulus puts t in [0, L) (section 2.2 notes that its
    implementation does not need x in [0, 1)).
    """
    x = np.asarray(x, dtype=np.float64)
    Lx = float(L) * x
    s = np.rint(Lx)
    t = np.mod(s, L).astype(np.int64)
    delta = Lx - s
    return s, t, delta


def bessel_coefficients(K, gamma):
    """The coefficients a_pr of eq. (2.6) (and eq. (A.1)), 0 <= p, r < K.

    a_pr = 4 i^r J_{(p+r)/2}(-gamma pi / 2) J_{(r-p)/2}(-gamma pi / 2) when p - r is
    even, else 0.  scipy's jv handles the negative order (r - p)/2 and the negative
    argument for integer orders.
    """
    z = -gamma * math.pi / 2.0
    a = np.zeros((K, K), dtype=np.complex128)
    for p in range(K):
        for r in range(K):
            if (p - r) % 2 == 0:
                a[p, r] = 4.0 * (1j ** r) * jv((p + r) // 2, z) * jv((r - p) // 2, z)
    return a


def prime_weights(K):
    """The primes on the sums of eq. (2.6): the first term is halved."""
    w = np.ones(K)
    w[0] = 0.5
    return w


def tail_bound(K, gamma):
    """sum of w_p w_r |a_pr| over the terms that a rank-K truncation drops.

    By the triangle inequality with |T_p| <= 1 and |exp(i theta)| = 1 (the argument
    of the proof of Lemma A.1) this bounds ||A - A_K||_max.  The dropped terms are
    those with p >= K OR r >= K.  They are summed directly, smallest first, so that
    no cancellation limits the bound near 1e-16.
    """
    a = np.abs(bessel_coefficients(TAIL_TERMS, gamma))
    w = prime_weights(TAIL_TERMS)
    W = np.outer(w, w) * a
    idx = np.arange(TAIL_TERMS)
    dropped = np.maximum.outer(idx, idx) >= K
    return float(np.sort(W[dropped]).sum())


def table_double_rank(gamma):
    """Table 2.1, double-precision row: the rank for the band holding gamma."""
    for edge, K in TABLE_2_1_DOUBLE:
        if gamma <= edge:
            return K
    raise ValueError("gamma must be <= 1/2")


def choose_K(eps, gamma):
    """The rank for working accuracy eps and perturbation gamma.

    gamma = 0: K = 1 (section 2.1.2: A is the matrix of all ones).
    Otherwise the smallest K whose dropped-term bound (tail_bound) is <= eps,
    capped by Table 2.1's double-precision row, below which FP64 rounding rules.
    """
    if not (0.0 < eps < 1.0):
        raise ValueError("eps must be in (0, 1)")
    if gamma == 0.0:
        return 1
    cap = table_double_rank(gamma)
    for K in range(1, cap + 1):
        if tail_bound(K, gamma) <= eps:
            return K
    return cap


def lambert_w_rank(eps, gamma):
    """Eq. (2.7): K = max{3, ceil(5 gamma exp(W(log(140/eps) / (5 gamma))))}."""
    from scipy.special import lambertw
    w = lambertw(math.log(140.0 / eps) / (5.0 * gamma)).real
    return max(3, int(math.ceil(5.0 * gamma * math.exp(w))))


def chebyshev_T(K, y):
    """T_0..T_{K-1} at the points y by the three-term recurrence (NIST 18.9.1)."""
    y = np.asarray(y, dtype=np.float64)
    T = np.empty(y.shape + (K,), dtype=np.float64)
    T[..., 0] = 1.0
    if K > 1:
        T[..., 1] = y
    for p in range(1, K - 1):
        T[..., p + 1] = 2.0 * y * T[..., p] - T[..., p - 1]
    return T


def phase(d):
    """The factor exp(-i pi d) of eq. (2.6)."""
    return np.exp(-1j * math.pi * np.asarray(d, dtype=np.float64))


@dataclass
class Plan:
    N: int
    M: int
    L: int
    eps: float
    s: np.ndarray
    t: np.ndarray
    delta: np.ndarray
    d: np.ndarray
    gamma: float
    K: int
    a: np.ndarray      # K x K coefficients (empty when gamma == 0)
    U: np.ndarray      # M x K, complex
    V: np.ndarray      # N x K, real


def plan(N, x, eps, L=None):
    """Planning stage: gamma, t, K and the factors U, V (sections 2.2 and 2.3).

    u_r = sum'_p a_pr exp(-i pi d) T_p(d / gamma)      (M-vector, r = 0..K-1)
    v_r = T_r(2k/N - 1) for r >= 1, v_0 = 1/2           (the r-prime of eq. (2.6))
    """
    N = int(N)
    L = N if L is None else int(L)
    if L < N:
        raise ValueError("grid size L must be >= N")
    x = np.asarray(x, dtype=np.float64)
    s, t, delta = round_to_grid(x, L)
    d = delta * (float(N) / float(L))
    gamma = float(np.max(np.abs(d))) if d.size else 0.0
    K = choose_K(eps, gamma)
    k = np.arange(N, dtype=np.float64)
    if gamma == 0.0:
        a = np.zeros((0, 0), dtype=np.complex128)
        U = np.ones((x.size, 1), dtype=np.complex128)
        V = np.ones((N, 1), dtype=np.float64)
    else:
        a = bessel_coefficients(K, gamma)
        w = prime_weights(K)
        Tx = chebyshev_T(K, d / gamma)                   # M x K : T_p(d_j / gamma)
        U = phase(d)[:, None] * ((Tx * w) @ a)           # u_r = sum'_p a_pr e^{-i pi d} T_p
        V = chebyshev_T(K, 2.0 * k / N - 1.0)            # N x K : T_r(2k/N - 1)
        V[:, 0] *= 0.5                                   # v_0 = T_0 / 2
    return Plan(N=N, M=x.size, L=L, eps=eps, s=s, t=t, delta=delta, d=d,
                gamma=gamma, K=K, a=a, U=U, V=V)


# ---------------------------------------------------------------------------
# Online stage (section 2.3 "Vectorization")
# ---------------------------------------------------------------------------

def nufft2(P, c):
    """f = sum_r D_{u_r} I_L(t,:) F_L D_{v_r} c, eq. (2.11), as the two-step form.

    Step 1: X = I_L(t,:) F_L [D_{v_0} c | ... | D_{v_{K-1}} c]  (c zero-padded to L)
    Step 2: f = [D_{u_0} X_0 | ... | D_{u_{K-1}} X_{K-1}] 1
    """
    c = np.asarray(c, dtype=np.complex128)
    W = np.zeros((P.L, P.K), dtype=np.complex128)
    W[:P.N, :] = P.V * c[:, None]
    X = np.fft.fft(W, axis=0)[P.t, :]
    return (P.U * X).sum(axis=1)


def nufft2_adjoint(P, g):
    """c = A^H g for the A of nufft2: the conjugate transpose of every step.

    Z_r[tau] = sum_{j: t_j = tau} conj(u_r(j)) g_j, then c = sum_r D_{v_r} (L ifft(Z_r))[:N],
    using F^H z = conj(F) z = L * ifft(z) (section 3.1 uses F^T = N conj(F)^{-1}).
    """
    g = np.asarray(g, dtype=np.complex128)
    Z = np.zeros((P.L, P.K), dtype=np.complex128)
    np.add.at(Z, P.t, np.conj(P.U) * g[:, None])
    Y = np.fft.ifft(Z, axis=0) * P.L
    return (P.V * Y[:P.N, :]).sum(axis=1)


def nufft1(P, g):
    """The paper's NUFFT-I of section 3.1: the TRANSPOSE F~2^T g, = conj(A^H conj(g))."""
    return np.conj(nufft2_adjoint(P, np.conj(np.asarray(g, dtype=np.complex128))))


def nufft2_dx(P, c, g):
    """d/dx_j of Re <f, g>: Re(conj(g_j) f'_j) with f' = A((-2 pi i k) o c).

    f_j = sum_k c_k exp(-2 pi i x_j k) gives df_j/dx_j = sum_k (-2 pi i k) c_k
    exp(-2 pi i x_j k), which is the NUFFT-II of (-2 pi i k) o c on the same plan.
    """
    k = np.arange(P.N, dtype=np.float64)
    fp = nufft2(P, -2j * math.pi * k * np.asarray(c, dtype=np.complex128))
    return np.real(np.conj(np.asarray(g, dtype=np.complex128)) * fp)


def dense_A(P):
    """The exact perturbation matrix A_jk = exp(-2 pi i d_j k / N) (section 2.2)."""
    k = np.arange(P.N, dtype=np.float64)
    return np.exp(-2j * math.pi * np.outer(P.d, k) / P.N)


def dense_AK(P):
    """The rank-K approximation A_K = U V^T of eq. (2.6)."""
    return P.U @ P.V.T


# ---------------------------------------------------------------------------
# Two dimensions (section 4, eq. (4.4))
# ---------------------------------------------------------------------------
#
# Reading of section 4's indices (garbled between m and n in the text): C is m x n,
# k1 < m pairs with x and k2 < n with y; x is rounded on an m-point grid and y on an
# n-point grid.  Each direction is the 1D method of section 2 with accuracy eps / 2:
# with |A^x - A^x_K| <= e_x and |A^y - A^y_K| <= e_y entrywise, the product of the two
# approximations is off by at most e_x + e_y + e_x e_y = eps (1 + eps / 4).


@dataclass
class Plan2D:
    m: int
    n: int
    px: Plan        # the x direction: N = m frequencies, samples x
    py: Plan        # the y direction: N = n frequencies, samples y


def plan2d(m, n, x, y, eps, Lx=None, Ly=None):
    """Planning stage of the 2D NUFFT-II: one 1D plan per direction at eps / 2."""
    return Plan2D(m=int(m), n=int(n), px=plan(m, x, eps / 2.0, Lx), py=plan(n, y, eps / 2.0, Ly))


def nufft2_2d(P, C):
    """f_j = sum_{r1, r2} u^x_r1(j) u^y_r2(j) [F2(D_{v^x_r1} C D_{v^y_r2})][t^x_j, t^y_j]  (eq. (4.4)).

    Each term is a full 2D FFT of the scaled (zero-padded) coefficient matrix, read at
    the rounded grid point of every sample.
    """
    C = np.asarray(C, dtype=np.complex128)
    px, py = P.px, P.py
    f = np.zeros(px.M, dtype=np.complex128)
    for r1 in range(px.K):
        for r2 in range(py.K):
            W = np.zeros((px.L, py.L), dtype=np.complex128)
            W[:P.m, :P.n] = px.V[:, r1][:, None] * C * py.V[:, r2][None, :]
            X = np.fft.fft2(W)
            f += px.U[:, r1] * py.U[:, r2] * X[px.t, py.t]
    return f


def nufft2_2d_adjoint(P, g):
    """C = A^H g for the A of nufft2_2d: every step of eq. (4.4) conjugated and reversed.

    For each (r1, r2): Z[tau_x, tau_y] = sum_{j: (t^x_j, t^y_j) = (tau_x, tau_y)}
    conj(u^x_r1(j) u^y_r2(j)) g_j, then the conjugate 2D DFT (F2^H z = Lx Ly ifft2(z)),
    cut to the m x n frequencies and scaled by v^x_r1(k1) v^y_r2(k2) (real); the terms
    are summed.  Section 3.1 gives the 1D transpose; this is its 2D, conjugated form.
    """
    g = np.asarray(g, dtype=np.complex128)
    px, py = P.px, P.py
    C = np.zeros((P.m, P.n), dtype=np.complex128)
    for r1 in range(px.K):
        for r2 in range(py.K):
            Z = np.zeros((px.L, py.L), dtype=np.complex128)
            np.add.at(Z, (px.t, py.t), np.conj(px.U[:, r1] * py.U[:, r2]) * g)
            Y = np.fft.ifft2(Z) * (px.L * py.L)
            C += px.V[:, r1][:, None] * Y[:P.m, :P.n] * py.V[:, r2][None, :]
    return C


# ---------------------------------------------------------------------------
# Inverse NUFFT-II (section 3.3): CG on the normal equations
# ---------------------------------------------------------------------------
#
# A c = f with A the N x N NUDFT-II matrix of perturbed equispaced samples
# (0 <= gamma < 1/2).  A^H A is Toeplitz, (A^H A)_jk = sum_p exp(2 pi i x_p (j - k)),
# Hermitian positive definite; its first column is A^H applied to the all-ones vector
# (A e_0 = 1), and a product with it is one FFT and one inverse FFT of size 2N through
# the circulant matrix whose first column is [t_0, ..., t_{N-1}, 0, conj(t_{N-1}), ...,
# conj(t_1)].


def toeplitz_column(P):
    """t_d = sum_p exp(2 pi i x_p d), d = 0..N-1: the first column of A^H A, as A^H 1."""
    return nufft2_adjoint(P, np.ones(P.M, dtype=np.complex128))


def circulant_eigenvalues(t):
    """FFT of the 2N-circulant that embeds the Hermitian Toeplitz matrix with column t."""
    N = t.size
    col = np.zeros(2 * N, dtype=np.complex128)
    col[:N] = t
    col[N + 1:] = np.conj(t[1:][::-1])
    return np.fft.fft(col)


def toeplitz_apply(lam, x):
    """(A^H A) x: the first N entries of the circulant product of the zero-padded x."""
    N = x.size
    y = np.fft.ifft(lam * np.fft.fft(np.concatenate([x, np.zeros(N, dtype=np.complex128)])))
    return y[:N]


def inverse_cg(P, f, tol, maxit):
    """Solve A c = f by CG on A^H A c = A^H f (section 3.3).  Stops when the residual of
    the normal equations has fallen by tol relative to A^H f, or after maxit iterations.
    Returns (c, iterations, final relative residual)."""
    lam = circulant_eigenvalues(toeplitz_column(P))
    b = nufft2_adjoint(P, np.asarray(f, dtype=np.complex128))
    c = np.zeros(P.N, dtype=np.complex128)
    r = b.copy()
    p = r.copy()
    rs = float(np.vdot(r, r).real)
    bnorm = math.sqrt(rs)
    it = 0
    while it < maxit and math.sqrt(rs) > tol * bnorm:
        Ap = toeplitz_apply(lam, p)
        alpha = rs / float(np.vdot(p, Ap).real)
        c += alpha * p
        r -= alpha * Ap
        rs_new = float(np.vdot(r, r).real)
        p = r + (rs_new / rs) * p
        rs = rs_new
        it += 1
    return c, it, (math.sqrt(rs) / bnorm if bnorm > 0 else 0.0)
