// passes.cuh -- the exec kernels of the low-rank NUFFT (section 2.3, two-step form).
//
// Forward, f = sum_r D_{u_r} I_L(t,:) F_L D_{v_r} c (eq. (2.11)), with the L-point
// FFT split four-step as L = L1 * L2, input index k = k1 + L1 k2, output index
// n = L2 n1 + n2:
//   pass 1  (one CTA per block of C columns k1 and one rank r):
//           x_k = i^r T_r(2k/N - 1) c_k          V-scale, fused into the load
//           Y_r[n2][k1] = w_L^{n2 k1} sum_{k2} x_{k1 + L1 k2} w_{L2}^{n2 k2}
//   pass 2  (one CTA per bucket of B2 rows n2, all ranks):
//           X_r[L2 n1 + n2] = sum_{k1} Y_r[n2][k1] w_{L1}^{n1 k1}   into shared memory
//           f_j = exp(-i pi d_j) sum_r mu_r(xi_j) X_r[t_j]          gather, U-scale, rank-sum
//           for the samples j whose grid point t_j lies in the bucket.
// With the primes of eq. (2.6) folded into beta, u_r(j) v_r(k) =
// exp(-i pi d_j) mu_r(j) i^r T_r(2k/N - 1), mu_r = sum_p beta_rp T_p(d_j / gamma).
//
// Adjoint, c = A^H g, the same steps conjugated and reversed:
//   pass A  Z_r[t] = sum_{j: t_j = t} mu_r(j) exp(+i pi d_j) g_j    (segmented over
//           the sorted samples, no atomics), inverse row DFTs, conj twiddle -> Y_r
//   pass B  inverse column DFTs, c_k = sum_r (-i)^r T_r(2k/N - 1) (...)_k
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "async_copy.cuh"
#include "fft_team.cuh"
#include "nufft_internal.h"

namespace nufft {

enum PassMode : int {
    MODE_PLAIN_IN = 1,    // pass 1 reads a pre-scaled W_r instead of c
    MODE_PLAIN_OUT = 2,   // pass 2 writes X_r in natural order instead of gathering
    MODE_PRESCALE = 4,    // pass 1 scales c by -2 pi i k (pass 2 then gathers f')
    MODE_DERIV = 16,      // K + 1 ranks; pass 2 forms f and f' = df/dx from the same rows
    MODE_GX = 32,         // pass 2 writes gx (+)= Re(conj(g) f') instead of a value
    MODE_FACTORS = 8      // read the plan's materialised U (sorted) and V instead of
                          // recomputing them (the FP64 plans: FP64 arithmetic is scarce)
};

// The fused kernels of FP64 plans (double-word arithmetic, or native FP64) read the
// plan's materialised factors (MODE_FACTORS); those of FP32 plans recompute them.  Fixed
// per element type, so the FP32 kernels carry no code for it.
template <typename T> constexpr bool kFactors = std::is_same<T, double>::value || std::is_same<T, dfloat>::value;

// The arithmetic of a 1D plan's fused exec: FP32 plans compute in FP32; FP64 plans in
// double-word FP32 pairs (dfloat.cuh: about 48 bits, from the FP32 pipes), since GB300's
// FP64 pipe is a small fraction of its FP32 one.  Their arrays stay complex128.
template <typename T> using Arith = typename std::conditional<std::is_same<T, double>::value, dfloat, T>::type;

// The row passes keep each lane's stage twiddles in registers across its row FFTs
// (FP32; in FP64 they would take twice the registers).
template <typename T> constexpr bool kTwReg = std::is_same<T, float>::value;


// The caller's arrays hold io_c<T> / io_r<T> (complex64 / float, or complex128 / double);
// to_cx and from_cx convert an element on load and on store (the identity except for the
// double-word kernels, whose caller's arrays are complex128).
template <typename T> __device__ __forceinline__ cx<T> to_cx(const io_c<T> &v) {
    if constexpr (std::is_same<T, dfloat>::value) {
        cx<T> r;
        r.x = dfloat(v.x);
        r.y = dfloat(v.y);
        return r;
    } else {
        return v;
    }
}
template <typename T> __device__ __forceinline__ io_c<T> from_cx(const cx<T> &v) {
    if constexpr (std::is_same<T, dfloat>::value) {
        return make_double2(v.x.to_double(), v.y.to_double());
    } else {
        return v;
    }
}

template <typename T> struct PassArgs;
// gx_j = re, or gx_j += re
template <typename T>
__device__ __forceinline__ void store_gx(const PassArgs<T> &a, int j, T re) {
    if constexpr (std::is_same<T, dfloat>::value) {
        a.gx[j] = a.accumulate ? a.gx[j] + re.to_double() : re.to_double();
    } else {
        a.gx[j] = a.accumulate ? a.gx[j] + re : re;
    }
}

template <typename T>
struct PassArgs {
    const io_c<T> *in;    // pass 1: c (or W);  pass A: g
    cx<T> *Y;             // intermediate, K x L2 x L1
    io_c<T> *out;         // pass 2: f (or X);  pass B: c
    const io_c<T> *g;     // dx cotangent
    io_r<T> *gx;          // dx output
    cx<T> *fscr;          // partial sums over rank groups (sorted order)
    cx<T> *part;          // pass B: per-split partial sums, SB x L
    int *counters;        // pass B: per-column-block tickets (zero between calls)
    const int32_t *tsorted, *perm, *bstart;
    const T *dsorted;
    const cx<T> *twc, *twr;     // stage twiddle tables: column FFTs (L2), row FFTs (L1)
    const cx<T> *twhi, *twlo;   // four-step twiddle w_L^m = twhi[m >> 12] twlo[m & 4095]
    int64_t N, M, L;
    int L1, L2, lg1, lg2;
    int K, G, B2, C, lgC, S;
    int mode, accumulate;
    int chunk;            // pass A: samples staged per chunk
    int mbar_off;         // pass 2: byte offset of the slot mbarriers in shared memory
    int CQ, lgCQ;         // pass A/B: columns of pass B's tiles (the adjoint intermediate's tiling)
    int nranks;           // ranks transformed: K, or K + 1 for MODE_DERIV
    io_c<T> *out2;        // MODE_DERIV: f' output (may be null)
    T piN;                // pi N
    int *err;             // device error word (bounded waits that timed out)
    const T *vfac;        // MODE_FACTORS: V[r][k] = v_r(k) of eq. (2.6), K x N
    const cx<T> *ufac;    // MODE_FACTORS: U[i][r] = u_r(perm[i]) of eq. (2.6), sorted order, M x K
    T inv_gamma;
    int SB;               // pass B: rank splits (CTAs per column block)
    int64_t in_off, out_off;   // batched launches: this problem's offsets into the packed in / out
    // two dimensions (section 4): N = m is the x extent, the y direction has K2 ranks
    int ncol, ldc;        // pass 1: valid columns (n) and the row stride of C (n)
    int K2;               // rank in y
    const T *dsorted2;    // d^y in sorted order
    const T *vy;          // T_r2(2 k2 / n - 1) for k2 < n (0 beyond), K2 x L1
    T inv_gamma2;         // 1 / gamma_y
};

// T_r(z) by the three-term recurrence (NIST 18.9.1).
template <typename T>
__device__ __forceinline__ T cheb_T(int r, T z) {
    if (r == 0) return T(1);
    T a = T(1), b = z;
    for (int q = 1; q < r; ++q) {
        const T c = fma(T(2) * z, b, -a);
        a = b;
        b = c;
    }
    return b;
}

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T *s, T *c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float *s, float *c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double *s, double *c) { sincospi(x, s, c); }

// w_L^m for 0 <= m < L from the two-level table (two roundings, ~1.5 ulp).
template <typename T>
__device__ __forceinline__ cx<T> twiddle_L(const PassArgs<T> &a, int m) {
    const cx<T> hi = ldg_cx(&a.twhi[m >> 12]);
    const cx<T> lo = ldg_cx(&a.twlo[m & 4095]);
    return cmul<T>(hi, lo);
}

// The four-step twiddle w_L^{n k} of an FFT output with index n = tt + TT q (q < E)
// splits as w_L^{tt k} w_L^{TT q k}: a per-thread base times a per-(team, q)
// table that the team fills in shared memory.  Entries: tab[q * ld].
template <typename T, int E, int TT>
__device__ __forceinline__ void fill_fourstep(const PassArgs<T> &a, int k, int tt, cx<T> *tab, int ld) {
#pragma unroll
    for (int q = tt; q < E; q += TT) tab[q * ld] = twiddle_L<T>(a, TT * q * k);
}

// beta_rp as the kernels read it: from the kernel's parameter space (one plan per
// launch), or from a shared-memory copy (batched launches) read through a volatile
// pointer, one broadcast load per use, so that the compiler does not hold the KM^2
// values in registers.
template <typename T, int KM>
__device__ __forceinline__ T beta_at(const Beta<T, KM> &b, int r, int q) { return b.b[r][q]; }
template <typename T, int KM>
struct BetaShared {
    const volatile T *p;
};
template <typename T, int KM>
__device__ __forceinline__ T beta_at(const BetaShared<T, KM> &b, int r, int q) { return b.p[r * KM + q]; }

// acc + a b, compensated: the exact error of the product (an FMA) and of the sum
// (two-sum) are added into comp, which the caller adds to acc at the end.  The forward's
// rank-sum of eq. (2.11) is accumulated so: at 2^20 (FP32, K = 12) the error against the
// FP64 oracle falls from 2.05e-7 to 1.94e-7 in the 2-norm and from 1.26e-9 to 1.00e-9
// ||c||_1 in the infinity norm, for 5 us of pass 2's 67.
template <typename T>
__device__ __forceinline__ void mac_comp(T &acc, T &comp, T a, T b) {
    const T p = a * b;
    const T pe = fma(a, b, -p);
    const T s = acc + p;
    const T z = s - acc;
    comp += ((acc - (s - z)) + (p - z)) + pe;
    acc = s;
}

template <typename T>
__device__ __forceinline__ cx<T> *smem_base() {
    extern __shared__ __align__(16) unsigned char nufft_smem_raw[];
    return reinterpret_cast<cx<T> *>(nufft_smem_raw);
}

// ---- pass 1: V-scale + column FFTs (length L2) + four-step twiddle ----------------
// Shared memory: C exchange slots of S elements, then the four-step table [q][cc].
// TWO_D: the column pass of section 4's transform.  C is row-major m x n (row stride
// ldc), the column element e is the x-frequency k1 < m (z = (2 e - m) / m), a column is
// the y-frequency k2 < n, and there is no four-step twiddle (the 2D DFT separates).
template <typename T, int P2, bool TWO_D = false>
__device__ __forceinline__ void pass1_body(const PassArgs<T> &a, const int bx, const int by) {
    constexpr int E = e_of<T, P2, PK_COL_FWD>();
    using TF = TeamFft<T, P2, E, false>;
    constexpr int TT = TF::TT;
    cx<T> *smem = smem_base<T>();
    // the thread's role among the C TT threads the pass needs; in a larger CTA (the
    // persistent batch kernel) the extra threads shadow a role exactly, writing the same
    // values to the same places (the leader-only steps stay with thread 0)
    const int lt = threadIdx.x & (a.C * TT - 1);
    const int cc = lt & (a.C - 1);
    const int tt = lt >> a.lgC;
    const int k1 = bx * a.C + cc;
    const int r = by;
    cx<T> *ftab = smem + a.C * a.S;
    if constexpr (!TWO_D) fill_fourstep<T, E, TT>(a, k1, tt, ftab + cc, a.C);
    cx<T> v[E];
    const int k0 = k1 + a.L1 * tt, kstride = a.L1 * TT;   // 1D: element m is c[k0 + m kstride]
    if constexpr (TWO_D) {
        // element e = tt + TT m of column k1: C[e][k1]
        const bool col_ok = k1 < a.ncol;
        const io_c<T> *cb = a.in + (int64_t)tt * a.ldc + k1;
        const int64_t estride = (int64_t)TT * a.ldc;
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = (col_ok && tt + TT * m < a.N) ? to_cx<T>(cb[m * estride]) : mk<T>(0, 0);
    } else if (a.mode & MODE_PLAIN_IN) {
        const io_c<T> *W = a.in + (int64_t)r * a.L + k1 + a.L1 * tt;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = to_cx<T>(W[m * (a.L1 * TT)]);
    } else {
        const io_c<T> *cb = a.in + k0;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = k0 + m * kstride < a.N ? to_cx<T>(cb[m * kstride]) : mk<T>(0, 0);
    }
    if (!(a.mode & MODE_PLAIN_IN)) {
        if constexpr (kFactors<T> && !TWO_D) {
            // x_k = v_r(k) c_k with the plan's V
            const T *vr = a.vfac + (int64_t)r * a.N;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = k0 + m * kstride;
                const T w = k < a.N ? vr[k] : T(0);
                cx<T> cv = v[m];
                if (a.mode & MODE_PRESCALE) {
                    const T wk = T(6.283185307179586476925286766559) * T(k);
                    cv = mk<T>(wk * cv.y, -wk * cv.x);
                }
                v[m] = mk<T>(w * cv.x, w * cv.y);
            }
        } else {
        // v_r(k) = T_r(z_k), z_k = (2k - N)/N, by the three-term recurrence run
        // across the elements (element-innermost for independent FMAs)
        const int Ni = (int)a.N;   // N < 2^23: 32-bit conversions (64-bit ones run on the FP64 pipe)
        const T invN = T(1) / T(Ni);
        constexpr int H = E < 8 ? E : 8;
#pragma unroll
        for (int h0 = 0; h0 < E; h0 += H) {
            T z2[H], ta[H], tb[H];
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const int k = TWO_D ? tt + TT * (h0 + m) : k1 + a.L1 * (tt + TT * (h0 + m));
                const T z = T(2 * k - Ni) * invN;
                z2[m] = T(2) * z;
                ta[m] = T(1);
                tb[m] = z;
            }
            int q = 1;
            for (; q + 1 < r; q += 2) {
#pragma unroll
                for (int m = 0; m < H; ++m) {
                    ta[m] = fma(z2[m], tb[m], -ta[m]);
                    tb[m] = fma(z2[m], ta[m], -tb[m]);
                }
            }
            const bool odd = q < r;
#pragma unroll
            for (int m = 0; m < H; ++m) {
                T tr = r == 0 ? T(1) : tb[m];
                if (odd) tr = fma(z2[m], tb[m], -ta[m]);
                cx<T> cv = v[h0 + m];
                if (a.mode & MODE_PRESCALE) {   // (-2 pi i k) c_k
                    const int k = k1 + a.L1 * (tt + TT * (h0 + m));
                    const T w = T(6.283185307179586476925286766559) * T(k);
                    cv = mk<T>(w * cv.y, -w * cv.x);
                }
                v[h0 + m] = mul_ipow<T>(mk<T>(tr * cv.x, tr * cv.y), r);
            }
        }
        }
    }
    TF::run(v, tt, smem + cc * a.S, a.twc);
    // output n2 = tt + TT q(e) goes to Y_r[n2][k1]
    cx<T> *yb = a.Y + (int64_t)r * a.L + tt * a.L1 + k1;
    const int ystride = TT * a.L1;
    const bool y_ok = idx_ok(r < a.nranks && k1 < a.L1 && tt < TT, a.err);   // stores only: barriers follow
    if constexpr (TWO_D) {
        if (y_ok) {
#pragma unroll
            for (int e = 0; e < E; ++e) yb[TF::out_q(e) * ystride] = v[e];
        }
    } else {
        __syncthreads();   // the four-step table is complete
        const cx<T> base = twiddle_L<T>(a, tt * k1);
        const cx<T> *fb = ftab + cc;
        if (y_ok) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int q = TF::out_q(e);
                const cx<T> w = cmul<T>(base, fb[q * a.C]);
                yb[q * ystride] = cmul<T>(v[e], w);
            }
        }
    }
}

// ---- pass 2: row FFTs (length L1) into shared memory, then gather/U-scale/rank-sum --
template <typename T, int P1, int KM, typename BT>
__device__ __forceinline__ void pass2_body(const PassArgs<T> &a, const BT &beta, const int bx) {
    constexpr int E = e_of<T, P1, PK_ROW_FWD>();
    using TF = TeamFft<T, P1, E, false>;
    constexpr int TT = TF::TT;
    constexpr bool WS = TT <= 32;   // each team inside one warp: its FFT syncs the warp only
    cx<T> *smem = smem_base<T>();
    const int nt = blockDim.x / TT;
    const int team = threadIdx.x / TT, tt = threadIdx.x % TT;
    const int b = bx;
    int i0 = a.bstart[b], i1 = a.bstart[b + 1];
    if (!idx_ok(i0 >= 0 && i0 <= i1 && i1 <= a.M, a.err)) i1 = i0 = 0;   // no samples (barriers follow)
    const int L2m = a.L2 - 1;
    const int Gs = a.G > 0 ? a.G : 1;   // never a zero stride
    // one mbarrier per slot: the rows of a rank group arrive by bulk copy (TMA)
    // while earlier rows are transformed
    uint64_t *mbar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(smem) + a.mbar_off);
    __shared__ int cta_failed;
    if (threadIdx.x == 0) {
        cta_failed = 0;
        for (int q = 0; q < Gs * a.B2; ++q) mbar_init(&mbar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t ROW_BYTES = P1 * sizeof(cx<T>);
    int gi = 0;
    for (int g0 = 0; g0 < a.nranks; g0 += Gs, ++gi) {
        const int gc = min(Gs, a.nranks - g0);
        const int njobs = gc * a.B2;
        if (threadIdx.x == 0) {
            for (int q = 0; q < njobs; ++q) {
                const cx<T> *src = a.Y + ((int64_t)(g0 + q / a.B2) * a.L2 + b * a.B2 + q % a.B2) * a.L1;
                mbar_arrive_expect_tx(&mbar[q], ROW_BYTES);
                bulk_copy_g2s(smem + q * a.S, src, ROW_BYTES, &mbar[q]);
            }
        }
        // this lane's stage twiddles, loaded once for all its row FFTs of this group
        typename TF::Tw twreg;
        if constexpr (kTwReg<T>) TF::load_tw(twreg, tt, a.twr);
        // one round of row FFTs, one job per team; PRED: a round with idle teams
        auto round = [&](const int j0, auto pred) {
            constexpr bool PRED = decltype(pred)::value;
            const int job = j0 + team;
            const bool act = !PRED || job < njobs;   // idle teams only meet the barriers
            cx<T> *sm = smem + (act ? job : 0) * a.S;
            cx<T> v[E];
            if (act) mbar_wait_bounded(&mbar[job], gi & 1, a.err, &cta_failed);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = act ? sm[tt + TT * m] : mk<T>(0, 0);   // row as copied
            team_sync<WS>();   // the row is read before the transform reuses its slot
            if constexpr (kTwReg<T>) TF::template run_reg<PRED, WS>(v, tt, sm, twreg, act);
            else TF::template run<PRED, WS>(v, tt, sm, a.twr, act);
            if (act) {
#pragma unroll
                for (int e = 0; e < E; ++e) sm[TF::out_padded(tt, e)] = v[e];
            }
        };
        for (int j0 = 0; j0 < njobs; j0 += nt) {
            if (j0 + nt <= njobs) round(j0, std::false_type{});
            else round(j0, std::true_type{});
        }
        __syncthreads();
        if (a.mode & MODE_PLAIN_OUT) {
            // X_r[L2 n1 + n2] in natural order, rows fastest for coalescing
            const int tot = njobs * a.L1;
            for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
                const int row = idx % a.B2;
                const int rest = idx / a.B2;
                const int n1 = rest % a.L1;
                const int rl = rest / a.L1;
                a.out[(int64_t)(g0 + rl) * a.L + (int64_t)a.L2 * n1 + b * a.B2 + row] =
                    from_cx<T>(smem[(rl * a.B2 + row) * a.S + padi<E>(n1)]);
            }
        } else if ((a.mode & MODE_DERIV) && !kFactors<T>) {
          if constexpr (!kFactors<T>) {
            // f and f' = df/dx from the K + 1 staged ranks (one group).  With
            // k = N (z + 1)/2 and z T_r = (T_{r+1} + T_{r-1})/2, the rank-r term of
            // A_K((-2 pi i k) o c) is -pi i N (X_r - i X_{r+1}/2 + i X_{r-1}/2) (r >= 1;
            // X_0 - i X_1 for r = 0), so f'_j = -pi i N e^{-i pi d} sum_{s<=K} rho_s X_s[t_j]
            // with rho_s = mu_s + i (mu_{s+1}/2 - mu_{s-1}/2 [s >= 2] - mu_0 [s = 1]).
            // software-pipelined: the next sample's t, d and j are loaded while this
            // one is formed
            int tn = 0, jn = 0;
            T dn = T(0);
            if (i0 + (int)threadIdx.x < i1) {
                tn = a.tsorted[i0 + threadIdx.x];
                dn = a.dsorted[i0 + threadIdx.x];
                jn = a.perm[i0 + threadIdx.x];
            }
#pragma unroll 1
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int t = tn, j = jn;
                const T d = dn;
                if (i + (int)blockDim.x < i1) {
                    tn = a.tsorted[i + blockDim.x];
                    dn = a.dsorted[i + blockDim.x];
                    jn = a.perm[i + blockDim.x];
                }
                const int row = (t & L2m) - b * a.B2;
                const int n1 = t >> a.lg2;
                if (!idx_ok(row >= 0 && row < a.B2 && n1 >= 0 && n1 < a.L1, a.err)) continue;
                const T xi = d * a.inv_gamma;
                T Tp[KM];
                Tp[0] = T(1);
                if (KM > 1) Tp[1] = xi;
#pragma unroll
                for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * xi, Tp[q - 1], -Tp[q - 2]);
                T mu[KM];
#pragma unroll
                for (int r = 0; r < KM; ++r) {
                    T m = T(0);
#pragma unroll
                    for (int q = (r & 1); q < KM; q += 2) m = fma(beta_at(beta, r, q), Tp[q], m);
                    mu[r] = m;   // zero for r >= K (beta is zero-padded)
                }
                // plain sums here: compensating these four products per rank cost 20 % of
                // the derivative pass (70 -> 84 us at 2^20)
                cx<T> S = mk<T>(0, 0), Sp = mk<T>(0, 0);
#pragma unroll
                for (int sidx = 0; sidx <= KM; ++sidx) {
                    if (sidx < a.nranks) {
                        const cx<T> x = smem[(sidx * a.B2 + row) * a.S + padi<E>(n1)];
                        const T ms = sidx < KM ? mu[sidx] : T(0);
                        T ri = sidx + 1 < KM ? T(0.5) * mu[sidx + 1] : T(0);
                        if (sidx == 1) ri -= mu[0];
                        if (sidx >= 2 && sidx - 1 < KM) ri -= T(0.5) * mu[sidx - 1];
                        S.x = fma(ms, x.x, S.x);
                        S.y = fma(ms, x.y, S.y);
                        Sp.x = fma(ms, x.x, fma(-ri, x.y, Sp.x));
                        Sp.y = fma(ms, x.y, fma(ri, x.x, Sp.y));
                    }
                }
                T sn, cs;
                sincospi_t<T>(d, &sn, &cs);
                const cx<T> f = mk<T>(fma(S.x, cs, S.y * sn), fma(S.y, cs, -S.x * sn));
                const cx<T> ph = mk<T>(fma(Sp.x, cs, Sp.y * sn), fma(Sp.y, cs, -Sp.x * sn));
                const cx<T> fp = mk<T>(a.piN * ph.y, -a.piN * ph.x);   // -i pi N (phase Sp)
                if (!idx_ok(j >= 0 && j < a.M, a.err)) continue;
                if (a.out) a.out[j] = from_cx<T>(f);
                if (a.out2) a.out2[j] = from_cx<T>(fp);
                if (a.mode & MODE_GX) {
                    const cx<T> gg = to_cx<T>(a.g[j]);
                    const T re = fma(gg.x, fp.x, gg.y * fp.y);
                    store_gx<T>(a, j, re);
                }
            }
          }
        } else {
            // software-pipelined as the derivative mode's loop (d only where the factors
            // are recomputed)
            int tn = 0, jn = 0;
            T dn = T(0);
            if (i0 + (int)threadIdx.x < i1) {
                tn = a.tsorted[i0 + threadIdx.x];
                if constexpr (!kFactors<T>) dn = a.dsorted[i0 + threadIdx.x];
                jn = a.perm[i0 + threadIdx.x];
            }
#pragma unroll 1
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int t = tn, j = jn;
                const T d = dn;
                if (i + (int)blockDim.x < i1) {
                    tn = a.tsorted[i + blockDim.x];
                    if constexpr (!kFactors<T>) dn = a.dsorted[i + blockDim.x];
                    jn = a.perm[i + blockDim.x];
                }
                const int row = (t & L2m) - b * a.B2;
                const int n1 = t >> a.lg2;
                if (!idx_ok(row >= 0 && row < a.B2 && n1 >= 0 && n1 < a.L1, a.err)) continue;
                cx<T> acc = g0 == 0 ? mk<T>(0, 0) : a.fscr[i];
                cx<T> comp = mk<T>(0, 0);   // the rank-sum's compensation
                constexpr bool fac = kFactors<T>;
                if constexpr (fac) {
                    // f_j = sum_r u_r(j) X_r[t_j] with the plan's U (phase included)
                    const cx<T> *ui = a.ufac + (int64_t)i * a.K;
                    for (int r = g0; r < g0 + gc; ++r) {
                        const cx<T> x = smem[((r - g0) * a.B2 + row) * a.S + padi<E>(n1)];
                        const cx<T> u = ui[r];
                        acc.x = fma(u.x, x.x, fma(-u.y, x.y, acc.x));
                        acc.y = fma(u.x, x.y, fma(u.y, x.x, acc.y));
                    }
                } else {
                    const T xi = d * a.inv_gamma;
                    T Tp[KM];
                    Tp[0] = T(1);
                    if (KM > 1) Tp[1] = xi;
#pragma unroll
                    for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * xi, Tp[q - 1], -Tp[q - 2]);
#pragma unroll
                    for (int r = 0; r < KM; ++r) {
                        if (r >= g0 && r < g0 + gc) {
                            T mu = T(0);
#pragma unroll
                            for (int q = (r & 1); q < KM; q += 2) mu = fma(beta_at(beta, r, q), Tp[q], mu);
                            const cx<T> x = smem[((r - g0) * a.B2 + row) * a.S + padi<E>(n1)];
                            mac_comp<T>(acc.x, comp.x, mu, x.x);
                            mac_comp<T>(acc.y, comp.y, mu, x.y);
                        }
                    }
                }
                if constexpr (!fac) {
                    acc.x += comp.x;
                    acc.y += comp.y;
                }
                if (g0 + gc < a.nranks) {
                    a.fscr[i] = acc;
                } else {
                    cx<T> val = acc;
                    if constexpr (!fac) {
                        T sn, cs;
                        sincospi_t<T>(d, &sn, &cs);
                        val = mk<T>(fma(acc.x, cs, acc.y * sn), fma(acc.y, cs, -acc.x * sn));
                    }
                    if (!idx_ok(j >= 0 && j < a.M, a.err)) continue;
                    if (a.mode & MODE_GX) {
                        const cx<T> gg = to_cx<T>(a.g[j]);
                        const T re = fma(gg.x, val.x, gg.y * val.y);
                        store_gx<T>(a, j, re);
                    } else {
                        a.out[j] = from_cx<T>(val);
                    }
                }
            }
        }
        fence_proxy_async_smem();   // these slot accesses precede the next group's copies
        __syncthreads();
    }
}

// ---- pass A (adjoint): segmented scatter into shared memory, inverse row FFTs -----
template <typename T, int P1, int KM, typename BT>
__device__ __forceinline__ void passA_body(const PassArgs<T> &a, const BT &beta, const int bx) {
    constexpr int E = e_of<T, P1, PK_ROW_ADJ>();
    using TF = TeamFft<T, P1, E, true>;
    constexpr int TT = TF::TT;
    constexpr bool WS = TT <= 32;   // each team inside one warp: its FFT rounds sync the warp only
    cx<T> *smem = smem_base<T>();
    const int nt = blockDim.x / TT;
    const int team = threadIdx.x / TT, tt = threadIdx.x % TT;
    const int b = bx;
    int i0 = a.bstart[b], i1 = a.bstart[b + 1];
    if (!idx_ok(i0 >= 0 && i0 <= i1 && i1 <= a.M, a.err)) i1 = i0 = 0;   // no samples (barriers follow)
    const int L2m = a.L2 - 1;
    const int Gs = a.G > 0 ? a.G : 1;   // never a zero stride
    __shared__ int rounds_max;          // the chunk's longest run of equal grid points, less one
    for (int g0 = 0; g0 < a.K; g0 += Gs) {
        const int gc = min(Gs, a.K - g0);
        const int njobs = gc * a.B2;
        const int nslots = Gs * a.B2;   // fixed offsets for the tables and staging below
        const int chunk = a.chunk > 0 ? a.chunk : 1;   // never a zero stride
        // a chunk's t, d and j are fetched into registers one chunk ahead (up to PF per
        // thread), so that their loads are in flight during the previous chunk's scatter
        // (or, for the first, during the zero fill); the gather of g waits for j only
        constexpr int PF = 2;
        const bool pf = chunk <= PF * (int)blockDim.x;
        int pt[PF], pj[PF];
        T pd[PF];
        auto fetch = [&](const int c0) {
            const int n = min(chunk, i1 - c0);
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int i = threadIdx.x + u * blockDim.x;
                if (i < n) {
                    pt[u] = a.tsorted[c0 + i];
                    if constexpr (!kFactors<T>) pd[u] = a.dsorted[c0 + i];
                    pj[u] = a.perm[c0 + i];
                }
            }
        };
        if (pf && i0 < i1) fetch(i0);
        for (int idx = threadIdx.x; idx < njobs * a.S; idx += blockDim.x) smem[idx] = mk<T>(0, 0);
        __syncthreads();
        // the bucket's samples, staged chunk by chunk: t, d and the gathered g
        int32_t *st_t = reinterpret_cast<int32_t *>(smem + nslots * a.S + nt * E);
        T *st_d = reinterpret_cast<T *>(st_t + a.chunk);
        cx<T> *st_g = reinterpret_cast<cx<T> *>(st_d + a.chunk);
        for (int c0 = i0; c0 < i1; c0 += chunk) {
            const int n = min(chunk, i1 - c0);
            __syncthreads();   // the previous chunk is consumed
            if (pf) {
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int i = threadIdx.x + u * blockDim.x;
                    if (i < n) {
                        st_t[i] = pt[u];
                        if constexpr (!kFactors<T>) st_d[i] = pd[u];
                        const int j = pj[u];
                        st_g[i] = idx_ok(j >= 0 && j < a.M, a.err) ? to_cx<T>(a.in[j]) : mk<T>(0, 0);
                    }
                }
                if (c0 + chunk < i1) fetch(c0 + chunk);
            } else {
#pragma unroll 4
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    st_t[i] = a.tsorted[c0 + i];
                    if constexpr (!kFactors<T>) st_d[i] = a.dsorted[c0 + i];
                    const int j = a.perm[c0 + i];
                    st_g[i] = idx_ok(j >= 0 && j < a.M, a.err) ? to_cx<T>(a.in[j]) : mk<T>(0, 0);
                }
            }
            // The chunk's samples are added into the slots sample-parallel, in rounds: round q
            // adds the q-th sample (within this chunk) of every run of equal grid points, so
            // each slot receives its samples one after another in sorted order -- the same
            // operations in the same order as one thread summing the run, and no two threads
            // of a round touch the same slot.  A run continued from the previous chunk adds to
            // what that chunk left in the slot.  (One round when every grid point holds at most
            // one sample of the chunk, as on a perturbed equispaced grid.)
            auto run_pos = [&](const int i) {
                const int t = st_t[i];
                int q = 0;
                while (q < i && st_t[i - q - 1] == t) ++q;
                return q;
            };
            if (threadIdx.x == 0) rounds_max = 0;
            __syncthreads();
            {
                int qm = 0;
                for (int i = threadIdx.x; i < n; i += blockDim.x) qm = max(qm, run_pos(i));
                if (qm > 0) atomicMax(&rounds_max, qm);
            }
            __syncthreads();
            const int nrounds = rounds_max + 1;
            for (int qr = 0; qr < nrounds; ++qr) {
#pragma unroll 1
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    if (nrounds > 1 && run_pos(i) != qr) continue;
                    const int t = st_t[i];
                    const int row = (t & L2m) - b * a.B2;
                    const int n1 = t >> a.lg2;
                    if (!idx_ok(row >= 0 && row < a.B2 && n1 >= 0 && n1 < a.L1, a.err)) continue;
                    cx<T> *slot = smem + row * a.S + padi<E>(n1);   // rank r at + (r - g0) B2 S
                    const cx<T> gg = st_g[i];
                    if constexpr (kFactors<T>) {
                        // Z_r += conj(u_r(j)) g_j with the plan's U
                        const cx<T> *ui = a.ufac + (int64_t)(c0 + i) * a.K;
#pragma unroll
                        for (int r = 0; r < KM; ++r) {
                            if (r >= g0 && r < g0 + gc) {
                                const cx<T> u = ui[r];
                                cx<T> z = slot[(r - g0) * a.B2 * a.S];
                                z.x = fma(u.x, gg.x, fma(u.y, gg.y, z.x));
                                z.y = fma(u.x, gg.y, fma(-u.y, gg.x, z.y));
                                slot[(r - g0) * a.B2 * a.S] = z;
                            }
                        }
                    } else {
                        const T d = st_d[i];
                        const T xi = d * a.inv_gamma;
                        T Tp[KM];
                        Tp[0] = T(1);
                        if (KM > 1) Tp[1] = xi;
#pragma unroll
                        for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * xi, Tp[q - 1], -Tp[q - 2]);
                        T sn, cs;
                        sincospi_t<T>(d, &sn, &cs);
                        const cx<T> h = mk<T>(fma(gg.x, cs, -gg.y * sn), fma(gg.y, cs, gg.x * sn));  // g e^{+i pi d}
#pragma unroll
                        for (int r = 0; r < KM; ++r) {
                            if (r >= g0 && r < g0 + gc) {
                                T mu = T(0);
#pragma unroll
                                for (int q = (r & 1); q < KM; q += 2) mu = fma(beta_at(beta, r, q), Tp[q], mu);
                                cx<T> z = slot[(r - g0) * a.B2 * a.S];
                                z.x = fma(mu, h.x, z.x);
                                z.y = fma(mu, h.y, z.y);
                                slot[(r - g0) * a.B2 * a.S] = z;
                            }
                        }
                    }
                }
                if (qr + 1 < nrounds) __syncthreads();   // the next round adds to these slots
            }
        }
        __syncthreads();
        // this lane's stage twiddles, loaded once for all its row FFTs of this group
        typename TF::Tw twreg;
        if constexpr (kTwReg<T>) TF::load_tw(twreg, tt, a.twr);
        cx<T> *ftab = smem + nslots * a.S + team * E;   // this team's four-step table
        // with one row per bucket (B2 = 1) every job has the same row n2 = b: its
        // four-step table and base twiddle are made once for all the rounds
        const bool one_row = a.B2 == 1;
        cx<T> base1 = mk<T>(1, 0);
        if (one_row) {
            fill_fourstep<T, E, TT>(a, b, tt, ftab, 1);
            base1 = twiddle_L<T>(a, b * tt);
        }
        auto round = [&](const int j0, auto pred) {   // PRED: a round with idle teams
            constexpr bool PRED = decltype(pred)::value;
            const int job = j0 + team;
            const bool act = !PRED || job < njobs;   // idle teams only meet the barriers
            const int rl = act ? job / a.B2 : 0, row = act ? job % a.B2 : 0;
            const int n2 = b * a.B2 + row;
            cx<T> *sm = smem + (act ? job : 0) * a.S;
            cx<T> v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (!act) v[m] = mk<T>(0, 0);
                else if constexpr (TT % E == 0) v[m] = sm[padi_run<E, TT>(padi<E>(tt), m)];
                else v[m] = sm[padi<E>(tt + TT * m)];
            }
            if (!one_row) fill_fourstep<T, E, TT>(a, n2, tt, ftab, 1);
            // the base twiddle w_L^{n2 tt}, loaded before the transform hides its latency
            const cx<T> base = one_row ? base1 : twiddle_L<T>(a, n2 * tt);
            team_sync<WS>();
            if constexpr (kTwReg<T>) TF::template run_reg<PRED, WS>(v, tt, sm, twreg, act);
            else TF::template run<PRED, WS>(v, tt, sm, a.twr, act);
            if (act) {
                // column-tiled layout for pass B: Y'_r[k1 / CQ][n2][k1 % CQ], so each
                // CQ-column tile of a rank is one contiguous block
                cx<T> *dst = a.Y + (int64_t)(g0 + rl) * a.L + n2 * a.CQ;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k1 = TF::out_index(tt, e);
                    dst[(k1 >> a.lgCQ) * (a.L2 << a.lgCQ) + (k1 & (a.CQ - 1))] =
                        cmulc<T>(v[e], cmul<T>(base, ftab[TF::out_q(e)]));
                }
            }
            team_sync<WS>();   // the next job may refill the team's ftab
        };
        for (int j0 = 0; j0 < njobs; j0 += nt) {
            if (j0 + nt <= njobs) round(j0, std::false_type{});
            else round(j0, std::true_type{});
        }
        __syncthreads();
    }
}

// ---- pass B (adjoint): inverse column FFTs, V-scale and rank-sum -----------------
// Grid (L1 / C, SB): CTA (x, s) sums the ranks r = s, s + SB, s + 2 SB, ... of its C
// columns.  Each rank's C-column tile of the intermediate is one contiguous block
// (pass A writes [k1 / C][n2][k1 % C]); it arrives by bulk asynchronous copy into
// one of two buffers while the other rank is transformed, and the transform then
// works in that buffer.  The sum over ranks is held in registers.  With SB > 1
// each CTA stores its partial sum to part[s], and the last CTA of the column block
// (an atomic ticket, no waiting) adds the SB partials in the fixed order
// s = 0..SB-1, so the result does not depend on which CTA finishes last.
// Pass B's CTA: a 32 KiB tile of CB columns, TT threads each (E = 16): 256 threads in
// FP32 (CB = 4096 / L2 columns of L2 / 16 threads), 128 in FP64.
template <typename T> struct PassBBounds;
template <> struct PassBBounds<float> { static constexpr int threads = 256, blocks = 2; };
template <> struct PassBBounds<double> { static constexpr int threads = 128, blocks = 3; };
template <> struct PassBBounds<dfloat> { static constexpr int threads = 128, blocks = 3; };

// TWO_D: the column pass of the 2D adjoint (section 4).  A column is the y-frequency
// k2 = k1 (this CTA's column index), its elements the x-frequencies k = out_index < m
// with z = (2 k - m) / m, and C[k][k2] goes to out[k * ldc + k2] for k < N = m, k2 < ncol.
template <typename T, int P2, bool TWO_D = false>
__device__ __forceinline__ void passB_body(const PassArgs<T> &a, const int bx, const int by) {
    constexpr int E = e_of<T, P2, PK_COL_ADJ>();
    using TF = TeamFft<T, P2, E, true>;
    constexpr int TT = TF::TT;
    cx<T> *smem = smem_base<T>();
    // the thread's role among the C TT threads the pass needs (extra threads of a larger
    // CTA shadow a role exactly, as in pass 1; the copies and tickets stay with thread 0)
    const int lt = threadIdx.x & (a.C * TT - 1);
    const int cc = lt & (a.C - 1);
    const int tt = lt >> a.lgC;
    const int k1 = bx * a.C + cc;
    const int s = by, SB = a.SB;
    const int Ni = (int)a.N;   // N < 2^23: 32-bit conversions (64-bit ones run on the FP64 pipe)
    const int bufsz = a.C * a.S;                        // elements per buffer
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * bufsz);
    __shared__ int cta_failed;
    const uint32_t tile_bytes = (uint32_t)(a.C * P2 * sizeof(cx<T>));
    const int64_t tile_off = (int64_t)bx * a.C * P2;
    const int nr = s < a.K ? (a.K - s + SB - 1) / SB : 0;   // ranks of this CTA
    if (threadIdx.x == 0) {
        cta_failed = 0;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        for (int i = 0; i < 2 && i < nr; ++i) {
            mbar_arrive_expect_tx(&mbar[i], tile_bytes);
            bulk_copy_g2s(smem + i * bufsz, a.Y + (int64_t)(s + i * SB) * a.L + tile_off, tile_bytes, &mbar[i]);
        }
    }
    __syncthreads();
    cx<T> acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = mk<T>(0, 0);
    for (int i = 0; i < nr; ++i) {
        const int r = s + i * SB;
        cx<T> *buf = smem + (i & 1) * bufsz;
        mbar_wait_bounded(&mbar[i & 1], (i >> 1) & 1, a.err, &cta_failed);
        cx<T> v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = buf[(tt + TT * m) * a.C + cc];   // tile as copied
        __syncthreads();
        TF::run(v, tt, buf + cc * a.S, a.twc);
        if constexpr (kFactors<T> && !TWO_D) {   // the plan's v_r(k) (real), no i^r
            const T *vr = a.vfac + (int64_t)r * a.N;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = k1 + a.L1 * TF::out_index(tt, e);
                const T w = k < a.N ? vr[k] : T(0);
                acc[e].x = fma(w, v[e].x, acc[e].x);
                acc[e].y = fma(w, v[e].y, acc[e].y);
            }
        } else {
        // (-i)^r T_r(z_k) v, the recurrence run element-innermost in chunks of H
        const T invN = T(1) / T(Ni);
        constexpr int H = E < 8 ? E : 8;
#pragma unroll
        for (int h0 = 0; h0 < E; h0 += H) {
            T z2[H], ta[H], tb[H];
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const int k = TWO_D ? TF::out_index(tt, h0 + m) : k1 + a.L1 * TF::out_index(tt, h0 + m);
                const T z = T(2 * k - Ni) * invN;
                z2[m] = T(2) * z;
                ta[m] = T(1);
                tb[m] = z;
            }
            int q = 1;
            for (; q + 1 < r; q += 2) {
#pragma unroll
                for (int m = 0; m < H; ++m) {
                    ta[m] = fma(z2[m], tb[m], -ta[m]);
                    tb[m] = fma(z2[m], ta[m], -tb[m]);
                }
            }
            const bool odd = q < r;
#pragma unroll
            for (int m = 0; m < H; ++m) {
                T tr = r == 0 ? T(1) : tb[m];
                if (odd) tr = fma(z2[m], tb[m], -ta[m]);
                const cx<T> y = mul_ipow<T>(v[h0 + m], -r);
                acc[h0 + m].x = fma(tr, y.x, acc[h0 + m].x);
                acc[h0 + m].y = fma(tr, y.y, acc[h0 + m].y);
            }
        }
        }
        // this buffer is free again: refill it with the rank after next
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && i + 2 < nr) {
            mbar_arrive_expect_tx(&mbar[i & 1], tile_bytes);
            bulk_copy_g2s(buf, a.Y + (int64_t)(r + 2 * SB) * a.L + tile_off, tile_bytes, &mbar[i & 1]);
        }
    }
    // c_k (1D), or C[k][k1] (2D), for the output element e
    auto store = [&](const int e, const cx<T> val) {
        if constexpr (TWO_D) {
            const int k = TF::out_index(tt, e);
            if (k < a.N && k1 < a.ncol) a.out[(int64_t)k * a.ldc + k1] = from_cx<T>(val);
        } else {
            const int k = k1 + a.L1 * TF::out_index(tt, e);
            if (k < a.N) a.out[k] = from_cx<T>(val);
        }
    };
    if (SB == 1) {
#pragma unroll
        for (int e = 0; e < E; ++e) store(e, acc[e]);
        return;
    }
    // partial sums -> part[s]; the last CTA of this column block reduces them
    cx<T> *mine = a.part + (int64_t)s * a.L;
#pragma unroll
    for (int e = 0; e < E; ++e) mine[k1 + a.L1 * TF::out_index(tt, e)] = acc[e];
    __threadfence();
    __syncthreads();
    __shared__ int ticket;
    if (threadIdx.x == 0) ticket = atomicAdd(&a.counters[bx], 1);
    __syncthreads();
    if (ticket != SB - 1) return;
    __threadfence();
    // the sum over s2 = 0..SB-1 in that order, H elements at a time so that their
    // loads are in flight together; this CTA's own partial comes from its registers
    constexpr int H = E < 8 ? E : 8;
#pragma unroll
    for (int h0 = 0; h0 < E; h0 += H) {
        cx<T> t[H];
#pragma unroll
        for (int m = 0; m < H; ++m) t[m] = mk<T>(0, 0);
        for (int s2 = 0; s2 < SB; ++s2) {
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const int k = k1 + a.L1 * TF::out_index(tt, h0 + m);
                const cx<T> pv = s2 == s ? acc[h0 + m] : ldcg_cx(&a.part[(int64_t)s2 * a.L + k]);
                t[m].x += pv.x;
                t[m].y += pv.y;
            }
        }
#pragma unroll
        for (int m = 0; m < H; ++m) store(h0 + m, t[m]);
    }
    if (threadIdx.x == 0) a.counters[bx] = 0;   // ready for the next call
}


// ---- 2D row pass (section 4, eq. (4.4)) ---------------------------------------------
// One CTA per x-grid row s1 = b.  For each r1 the row W_r1[s1][:] of pass 1's output
// arrives by bulk copy (two buffers: the row of r1 + 2 is fetched while r1 + 1 is
// used), and the teams transform it once per r2 under the y-scale,
// X_r1r2[s1][:] = F_L1(i^r2 T_r2(z^y) o W_r1[s1][:]), one slot each.  The samples on
// row s1 then add u^x_r1 sum_r2 u^y_r2 X_r1r2[s1][t^y] to their partial sums (fscr,
// sorted order, the same thread for a sample at every r1); at the last r1 the phase
// exp(-i pi (d^x + d^y)) is applied and f written.  The pass-1 transforms over k1 are
// shared by every r2, which is the saving the paper notes after eq. (4.4).
// Shared memory: two row buffers (L1 each), K2 slots of S, two mbarriers.
template <typename T, int P1, int KM, typename BT>
__device__ __forceinline__ void pass2d_body(const PassArgs<T> &a, const BT &betax, const BT &betay,
                                            const int b) {
    constexpr int E = e_of<T, P1, PK_ROW_FWD>();
    using TF = TeamFft<T, P1, E, false>;
    constexpr int TT = TF::TT;
    cx<T> *smem = smem_base<T>();
    const int team = threadIdx.x / TT, tt = threadIdx.x % TT;
    const int nt = blockDim.x / TT;
    const int K1 = a.K, K2 = a.K2;
    // the K2 y-ranks of a row are transformed and gathered G2 at a time (all at once
    // when their slots fit; the FP64 rows of the longest grids take two groups or more)
    const int G2 = a.G > 0 ? min(a.G, K2) : K2;
    cx<T> *stg = smem;                 // two rows as copied
    cx<T> *slots = smem + 2 * P1;      // G2 transformed rows
    uint64_t *mbar = reinterpret_cast<uint64_t *>(slots + G2 * a.S);
    __shared__ int cta_failed;
    constexpr uint32_t ROW_BYTES = P1 * sizeof(cx<T>);
    const cx<T> *rows = a.Y + (int64_t)b * a.L1;   // W_r1[s1][:] at rows + r1 L
    if (threadIdx.x == 0) {
        cta_failed = 0;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        for (int i = 0; i < 2 && i < K1; ++i) {
            mbar_arrive_expect_tx(&mbar[i], ROW_BYTES);
            bulk_copy_g2s(stg + i * P1, rows + (int64_t)i * a.L, ROW_BYTES, &mbar[i]);
        }
    }
    __syncthreads();
    int i0 = a.bstart[b], i1 = a.bstart[b + 1];
    if (!idx_ok(i0 >= 0 && i0 <= i1 && i1 <= a.M, a.err)) i1 = i0 = 0;   // no samples (barriers follow)
    const T invg = a.inv_gamma, invg2 = a.inv_gamma2;
    for (int r1 = 0; r1 < K1; ++r1) {
        const int buf = r1 & 1;
        mbar_wait_bounded(&mbar[buf], (r1 >> 1) & 1, a.err, &cta_failed);
        const cx<T> *row = stg + buf * P1;
        // this lane's stage twiddles, loaded once for all its row FFTs of this r1
        typename TF::Tw twreg;
        if constexpr (kTwReg<T>) TF::load_tw(twreg, tt, a.twr);
        for (int g2 = 0; g2 < K2; g2 += G2) {
            const int gc2 = min(G2, K2 - g2);
            auto round = [&](const int j0, auto pred) {   // one r2 per team; PRED: idle teams
                constexpr bool PRED = decltype(pred)::value;
                const int jj = j0 + team;
                const bool act = !PRED || jj < gc2;
                const int r2 = g2 + (act ? jj : 0);
                cx<T> *sm = slots + (act ? jj : 0) * a.S;
                const T *vy = a.vy + (int64_t)r2 * P1;
                cx<T> v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int k = tt + TT * m;
                    const cx<T> w = row[k];
                    const T sc = act ? vy[k] : T(0);
                    v[m] = mul_ipow<T>(mk<T>(sc * w.x, sc * w.y), r2);
                }
                if constexpr (kTwReg<T>) TF::template run_reg<PRED>(v, tt, sm, twreg, act);
                else TF::template run<PRED>(v, tt, sm, a.twr, act);
                if (act) {
#pragma unroll
                    for (int e = 0; e < E; ++e) sm[TF::out_padded(tt, e)] = v[e];
                }
            };
            for (int j0 = 0; j0 < gc2; j0 += nt) {
                if (j0 + nt <= gc2) round(j0, std::false_type{});
                else round(j0, std::true_type{});
            }
            __syncthreads();   // the group's rows are complete (and, after the last, stg[buf] is read)
            if (threadIdx.x == 0 && g2 + gc2 == K2 && r1 + 2 < K1) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar[buf], ROW_BYTES);
                bulk_copy_g2s(stg + buf * P1, rows + (int64_t)(r1 + 2) * a.L, ROW_BYTES, &mbar[buf]);
            }
            // the gather; ONE: all K2 y-ranks in one group (g2 = 0, gc2 = K2), so that its
            // tests reduce to constants where the group is the whole
            auto gather = [&](auto one) {
                constexpr bool ONE = decltype(one)::value;
                const int gb = ONE ? 0 : g2, ge = ONE ? K2 : g2 + gc2;   // ranks [gb, ge)
                const bool first = r1 == 0 && (ONE || g2 == 0);   // no partial sum yet
                const bool fin = r1 + 1 == K1 && (ONE || ge == K2);   // the sums are complete
                // software-pipelined: the next sample's t, d^x, d^y and partial sum are loaded
                // while this one is formed
                int tn = 0;
                T dxn = T(0), dyn = T(0);
                cx<T> accn = mk<T>(0, 0);
                if (i0 + (int)threadIdx.x < i1) {
                    const int i = i0 + threadIdx.x;
                    tn = a.tsorted[i];
                    dxn = a.dsorted[i];
                    dyn = a.dsorted2[i];
                    if (!first) accn = a.fscr[i];
                }
#pragma unroll 1
                for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                    const int n1 = tn >> a.lg2;   // t^y
                    const T dx = dxn, dy = dyn;
                    cx<T> acc = accn;
                    if (i + (int)blockDim.x < i1) {
                        const int in = i + blockDim.x;
                        tn = a.tsorted[in];
                        dxn = a.dsorted[in];
                        dyn = a.dsorted2[in];
                        if (!first) accn = a.fscr[in];
                    }
                    if (!idx_ok(n1 >= 0 && n1 < a.L1, a.err)) continue;
                    // mu^x_r1 = sum_p beta^x_r1p T_p(d^x / gamma_x), mu^y_r2 likewise in y
                    T Tp[KM];
                    const T xi = dx * invg;
                    Tp[0] = T(1);
                    if (KM > 1) Tp[1] = xi;
#pragma unroll
                    for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * xi, Tp[q - 1], -Tp[q - 2]);
                    T mux = T(0);
#pragma unroll
                    for (int q = 0; q < KM; ++q)
                        if (((q ^ r1) & 1) == 0) mux = fma(beta_at(betax, r1, q), Tp[q], mux);
                    const T eta = dy * invg2;
                    Tp[0] = T(1);
                    if (KM > 1) Tp[1] = eta;
#pragma unroll
                    for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * eta, Tp[q - 1], -Tp[q - 2]);
                    cx<T> S = mk<T>(0, 0);
#pragma unroll
                    for (int r2 = 0; r2 < KM; ++r2) {
                        if (r2 >= gb && r2 < ge) {
                            T mu = T(0);
#pragma unroll
                            for (int q = (r2 & 1); q < KM; q += 2) mu = fma(beta_at(betay, r2, q), Tp[q], mu);
                            const cx<T> x = slots[(r2 - gb) * a.S + padi<E>(n1)];
                            S.x = fma(mu, x.x, S.x);
                            S.y = fma(mu, x.y, S.y);
                        }
                    }
                    acc.x = fma(mux, S.x, acc.x);
                    acc.y = fma(mux, S.y, acc.y);
                    if (!fin) {
                        a.fscr[i] = acc;
                    } else {
                        T sn, cs;
                        sincospi_t<T>(dx + dy, &sn, &cs);
                        const int j = a.perm[i];
                        if (idx_ok(j >= 0 && j < a.M, a.err))
                            a.out[j] = from_cx<T>(mk<T>(fma(acc.x, cs, acc.y * sn), fma(acc.y, cs, -acc.x * sn)));
                    }
                }
            };
            if (G2 >= K2) gather(std::true_type{});
            else gather(std::false_type{});
            __syncthreads();   // the slots are rewritten by the next group
        }
    }
}

// ---- 2D adjoint row pass (section 4: eq. (4.4) conjugated and reversed) ---------------
// One CTA per x-grid row s1 = b; the row's samples are sorted by t^y.  For each x-rank r1
// and each group of y-ranks, one slot per r2 receives
//     Z_r1r2[t^y] = sum over the row's samples j at t^y of mu^x_r1 mu^y_r2 e^{+i pi (d^x + d^y)} g_j
// (a segmented sum over the sorted samples: the thread at the start of each run of equal
// t^y adds up the run, so there are no atomics and the order is fixed), then the teams
// inverse-transform the slots over t^y (length L1), scale by (-i)^r2 T_r2(2 k2 / n - 1)
// (the conjugate of the forward's y-scale) and the y-ranks are summed into the row
//     W'_r1[s1][k2] = sum_r2 (-i)^r2 T_r2(z^y_k2) (L1 IDFT Z_r1r2)[k2],
// written in pass B's column-tiled layout [k2 / CQ][s1][k2 % CQ] for the column pass.
// h_j = e^{+i pi (d^x + d^y)} g_j is formed once (r1 = 0, first group) in sorted order in
// fscr and read back later by the same thread (the run of each sample has a fixed owner).
// Shared memory: an accumulator row (L1) for the groups' partial sums, then G2 slots.
template <typename T, int P1, int KM, typename BT>
__device__ __forceinline__ void passA2d_body(const PassArgs<T> &a, const BT &betax, const BT &betay,
                                             const int b) {
    constexpr int E = e_of<T, P1, PK_ROW_ADJ>();
    using TF = TeamFft<T, P1, E, true>;
    constexpr int TT = TF::TT;
    cx<T> *smem = smem_base<T>();
    const int team = threadIdx.x / TT, tt = threadIdx.x % TT;
    const int nt = blockDim.x / TT;
    const int K1 = a.K, K2 = a.K2;
    const int G2 = a.G > 0 ? min(a.G, K2) : K2;
    cx<T> *accrow = smem;        // sum over the y-ranks of the groups so far (one row)
    cx<T> *slots = smem + P1;    // G2 slots of S
    int i0 = a.bstart[b], i1 = a.bstart[b + 1];
    if (!idx_ok(i0 >= 0 && i0 <= i1 && i1 <= a.M, a.err)) i1 = i0 = 0;   // no samples (barriers follow)
    const T invg = a.inv_gamma, invg2 = a.inv_gamma2;
    for (int r1 = 0; r1 < K1; ++r1) {
        for (int g2 = 0; g2 < K2; g2 += G2) {
            const int gc2 = min(G2, K2 - g2);
            const bool first = r1 == 0 && g2 == 0;
            for (int idx = threadIdx.x; idx < gc2 * a.S; idx += blockDim.x) slots[idx] = mk<T>(0, 0);
            __syncthreads();
#pragma unroll 1
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int t = a.tsorted[i];
                if (i > i0 && a.tsorted[i - 1] == t) continue;   // inside a run: its start adds it up
                cx<T> acc[KM];
#pragma unroll
                for (int r2 = 0; r2 < KM; ++r2) acc[r2] = mk<T>(0, 0);
#pragma unroll 1
                for (int i2 = i; i2 < i1; ++i2) {
                    if (i2 > i && a.tsorted[i2] != t) break;
                    const T dx = a.dsorted[i2], dy = a.dsorted2[i2];
                    cx<T> h;
                    if (first) {
                        const int j = a.perm[i2];
                        const cx<T> gg = idx_ok(j >= 0 && j < a.M, a.err) ? to_cx<T>(a.in[j]) : mk<T>(0, 0);
                        T sn, cs;
                        sincospi_t<T>(dx + dy, &sn, &cs);
                        h = mk<T>(fma(gg.x, cs, -gg.y * sn), fma(gg.y, cs, gg.x * sn));   // g e^{+i pi (dx + dy)}
                        a.fscr[i2] = h;
                    } else {
                        h = a.fscr[i2];
                    }
                    // mu^x_r1 = sum_p beta^x_r1p T_p(d^x / gamma_x), mu^y_r2 likewise in y
                    T Tp[KM];
                    const T xi = dx * invg;
                    Tp[0] = T(1);
                    if (KM > 1) Tp[1] = xi;
#pragma unroll
                    for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * xi, Tp[q - 1], -Tp[q - 2]);
                    T mux = T(0);
#pragma unroll
                    for (int q = 0; q < KM; ++q)
                        if (((q ^ r1) & 1) == 0) mux = fma(beta_at(betax, r1, q), Tp[q], mux);
                    h = mk<T>(mux * h.x, mux * h.y);
                    const T eta = dy * invg2;
                    Tp[0] = T(1);
                    if (KM > 1) Tp[1] = eta;
#pragma unroll
                    for (int q = 2; q < KM; ++q) Tp[q] = fma(T(2) * eta, Tp[q - 1], -Tp[q - 2]);
#pragma unroll
                    for (int r2 = 0; r2 < KM; ++r2) {
                        if (r2 >= g2 && r2 < g2 + gc2) {
                            T mu = T(0);
#pragma unroll
                            for (int q = (r2 & 1); q < KM; q += 2) mu = fma(beta_at(betay, r2, q), Tp[q], mu);
                            acc[r2].x = fma(mu, h.x, acc[r2].x);
                            acc[r2].y = fma(mu, h.y, acc[r2].y);
                        }
                    }
                }
                const int n1 = t >> a.lg2;   // t^y
                if (!idx_ok(n1 >= 0 && n1 < P1 && (t & (a.L2 - 1)) == b, a.err)) continue;
#pragma unroll
                for (int r2 = 0; r2 < KM; ++r2)
                    if (r2 >= g2 && r2 < g2 + gc2) slots[(r2 - g2) * a.S + padi<E>(n1)] = acc[r2];
            }
            __syncthreads();
            // this lane's stage twiddles, loaded once for all its row FFTs of this group
            typename TF::Tw twreg;
            if constexpr (kTwReg<T>) TF::load_tw(twreg, tt, a.twr);
            auto round = [&](const int j0, auto pred) {   // one r2 per team; PRED: idle teams
                constexpr bool PRED = decltype(pred)::value;
                const int jj = j0 + team;
                const bool act = !PRED || jj < gc2;
                const int r2 = g2 + (act ? jj : 0);
                cx<T> *sm = slots + (act ? jj : 0) * a.S;
                cx<T> v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    if (!act) v[m] = mk<T>(0, 0);
                    else if constexpr (TT % E == 0) v[m] = sm[padi_run<E, TT>(padi<E>(tt), m)];
                    else v[m] = sm[padi<E>(tt + TT * m)];
                }
                __syncthreads();   // the slot is read before the transform reuses it
                if constexpr (kTwReg<T>) TF::template run_reg<PRED>(v, tt, sm, twreg, act);
                else TF::template run<PRED>(v, tt, sm, a.twr, act);
                if (act) {
                    const T *vy = a.vy + (int64_t)r2 * P1;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const T sc = vy[TF::out_index(tt, e)];
                        const cx<T> y = mul_ipow<T>(v[e], -r2);
                        sm[TF::out_padded(tt, e)] = mk<T>(sc * y.x, sc * y.y);
                    }
                }
            };
            for (int j0 = 0; j0 < gc2; j0 += nt) {
                if (j0 + nt <= gc2) round(j0, std::false_type{});
                else round(j0, std::true_type{});
            }
            __syncthreads();
            // the sum over this group's y-ranks, in r2 order; after the last group the row
            // goes out, column-tiled: W'_r1[k2 / CQ][s1][k2 % CQ]
            const bool last = g2 + gc2 == K2;
            cx<T> *dst = a.Y + (int64_t)r1 * a.L + b * a.CQ;
            for (int k2 = threadIdx.x; k2 < P1; k2 += blockDim.x) {
                cx<T> sum = g2 == 0 ? mk<T>(0, 0) : accrow[k2];
                for (int jj = 0; jj < gc2; ++jj) sum = cadd<T>(sum, slots[jj * a.S + padi<E>(k2)]);
                if (last) dst[(k2 >> a.lgCQ) * (a.L2 << a.lgCQ) + (k2 & (a.CQ - 1))] = sum;
                else accrow[k2] = sum;
            }
            __syncthreads();   // the slots and the row are rewritten by the next group
        }
    }
}

// ---- kernels ----------------------------------------------------------------------
// One plan per launch: the arguments are kernel parameters.
template <typename T, int P2>
__global__ void __launch_bounds__(256, 2) k_pass1(const __grid_constant__ PassArgs<T> a) {
    pass1_body<T, P2>(a, blockIdx.x, blockIdx.y);
}
// Two CTAs per SM for the FP64 row pass (its rank groups are sized for that); the FP32
// one is left to the compiler (it stays below 128 registers).
template <typename T> struct Pass2MinBlocks { static constexpr int v = 2; };
template <> struct Pass2MinBlocks<float> { static constexpr int v = 1; };
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256, Pass2MinBlocks<T>::v) k_pass2(const __grid_constant__ PassArgs<T> a,
                                               const __grid_constant__ Beta<T, KM> beta) {
    pass2_body<T, P1, KM>(a, beta, blockIdx.x);
}
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256) k_passA(const __grid_constant__ PassArgs<T> a,
                                               const __grid_constant__ Beta<T, KM> beta) {
    passA_body<T, P1, KM>(a, beta, blockIdx.x);
}
template <typename T, int P2>
__global__ void __launch_bounds__(PassBBounds<T>::threads, PassBBounds<T>::blocks) k_passB(const __grid_constant__ PassArgs<T> a) {
    passB_body<T, P2>(a, blockIdx.x, blockIdx.y);
}
// the 2D transform (section 4): column pass and row pass
template <typename T, int P2>
__global__ void __launch_bounds__(256, 2) k_pass1_2d(const __grid_constant__ PassArgs<T> a) {
    pass1_body<T, P2, true>(a, blockIdx.x, blockIdx.y);
}
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256) k_pass2d(const __grid_constant__ PassArgs<T> a,
                                                const __grid_constant__ Beta<T, KM> betax,
                                                const __grid_constant__ Beta<T, KM> betay) {
    pass2d_body<T, P1, KM>(a, betax, betay, blockIdx.x);
}

// the 2D adjoint (section 4): row pass and column pass
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256) k_passA2d(const __grid_constant__ PassArgs<T> a,
                                                 const __grid_constant__ Beta<T, KM> betax,
                                                 const __grid_constant__ Beta<T, KM> betay) {
    passA2d_body<T, P1, KM>(a, betax, betay, blockIdx.x);
}
template <typename T, int P2>
__global__ void __launch_bounds__(PassBBounds<T>::threads, PassBBounds<T>::blocks) k_passB2d(const __grid_constant__ PassArgs<T> a) {
    passB_body<T, P2, true>(a, blockIdx.x, blockIdx.y);
}

// Many independent plans per launch (a batch of uneven problems): blockIdx.z is the
// problem.  The problems of one launch share the grid length L, and so every launch
// dimension but the rank count; each reads its own arguments (buffers, K, M, tables)
// from args[z], and its input and output at in + in_off, out + out_off.  CTAs beyond a
// problem's own rank count or rank split return before any barrier.
// A batched launch's data pointers: problem z reads in + in_off + z in_stride and writes
// out (and, when not null, out2) + out_off + z out_stride.  Batches of uneven problems
// carry their offsets in the arguments (strides 0); batches of coefficient vectors on one
// plan pass the call's leading dimensions as strides, so that their arguments do not
// depend on the call and are built once.
struct ManyIO {
    const void *in;
    void *out;
    void *out2;
    int64_t in_stride, out_stride;
};

// The problem's arguments, copied to shared memory sa (all threads, then a barrier).
template <typename T>
__device__ __forceinline__ void many_args(PassArgs<T> &sa, const PassArgs<T> *__restrict__ args, const ManyIO &io) {
    static_assert(sizeof(PassArgs<T>) % 8 == 0, "copied in 8-byte words");
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&args[blockIdx.z]);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(PassArgs<T>) / 8); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t z = blockIdx.z;
        sa.in = (const io_c<T> *)io.in + sa.in_off + z * io.in_stride;
        sa.out = (io_c<T> *)io.out + sa.out_off + z * io.out_stride;
        if (io.out2) sa.out2 = (io_c<T> *)io.out2 + sa.out_off + z * io.out_stride;
    }
    __syncthreads();
}
template <typename T, int KM>
__device__ __forceinline__ void stage_beta(Beta<T, KM> &sb, const Beta<T, KM> *__restrict__ betas) {
    const T *src = &betas[blockIdx.z].b[0][0];
    for (int i = threadIdx.x; i < KM * KM; i += blockDim.x) (&sb.b[0][0])[i] = src[i];
    __syncthreads();
}
template <typename T, int P2>
__global__ void __launch_bounds__(256, 2) k_pass1_many(const PassArgs<T> *__restrict__ args,
                                                       const ManyIO io) {
    __shared__ PassArgs<T> a;
    many_args<T>(a, args, io);
    if ((int)blockIdx.y >= a.nranks) return;
    pass1_body<T, P2>(a, blockIdx.x, blockIdx.y);
}
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256) k_pass2_many(const PassArgs<T> *__restrict__ args,
                                                    const Beta<T, KM> *__restrict__ betas,
                                                    const ManyIO io) {
    __shared__ Beta<T, KM> sb;
    stage_beta<T, KM>(sb, betas);
    __shared__ PassArgs<T> a;
    many_args<T>(a, args, io);
    pass2_body<T, P1, KM>(a, BetaShared<T, KM>{&sb.b[0][0]}, blockIdx.x);
}
template <typename T, int P1, int KM>
__global__ void __launch_bounds__(256) k_passA_many(const PassArgs<T> *__restrict__ args,
                                                    const Beta<T, KM> *__restrict__ betas,
                                                    const ManyIO io) {
    __shared__ Beta<T, KM> sb;
    stage_beta<T, KM>(sb, betas);
    __shared__ PassArgs<T> a;
    many_args<T>(a, args, io);
    passA_body<T, P1, KM>(a, BetaShared<T, KM>{&sb.b[0][0]}, blockIdx.x);
}
template <typename T, int P2>
__global__ void __launch_bounds__(PassBBounds<T>::threads, PassBBounds<T>::blocks) k_passB_many(const PassArgs<T> *__restrict__ args,
                                                       const ManyIO io) {
    __shared__ PassArgs<T> a;
    many_args<T>(a, args, io);
    if ((int)blockIdx.y >= a.SB) return;
    passB_body<T, P2>(a, blockIdx.x, blockIdx.y);
}

// ---- launchers ------------------------------------------------------------------

template <typename F>
int dispatch_P(int P, F &&f) {
    switch (P) {
        case 32: return f(std::integral_constant<int, 32>{});
        case 64: return f(std::integral_constant<int, 64>{});
        case 128: return f(std::integral_constant<int, 128>{});
        case 256: return f(std::integral_constant<int, 256>{});
        case 512: return f(std::integral_constant<int, 512>{});
        case 1024: return f(std::integral_constant<int, 1024>{});
        case 2048: return f(std::integral_constant<int, 2048>{});
        default: return NUFFT_EUNSUPPORTED;
    }
}

// The batched kernels exist for FFT lengths up to MANY_P_MAX (grids up to 2^18
// points): batching pays for problems too small to fill the GPU alone.
constexpr int MANY_P_MAX = 512;

template <typename F>
int dispatch_P_many(int P, F &&f) {
    switch (P) {
        case 32: return f(std::integral_constant<int, 32>{});
        case 64: return f(std::integral_constant<int, 64>{});
        case 128: return f(std::integral_constant<int, 128>{});
        case 256: return f(std::integral_constant<int, 256>{});
        case 512: return f(std::integral_constant<int, 512>{});
        default: return NUFFT_EUNSUPPORTED;
    }
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device.  The
// flags are atomics: two threads that plan at once may both set the attribute (the same
// value, harmless), but neither reads a torn flag.
using SmemFlags = std::atomic<int>[64];
template <typename K>
inline int set_smem(K kern, size_t bytes, int device, std::atomic<int> *done) {
    if (bytes > 48 * 1024 && device >= 0 && device < 64 && !done[device].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(SMEM_BUDGET + 16 * 1024)) != cudaSuccess) {
            (void)cudaGetLastError();
            return NUFFT_ECUDA;
        }
        done[device].store(1, std::memory_order_release);
    }
    return NUFFT_OK;
}

inline int launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// A plan table for the kernels of element type T: the double-word kernels read the
// double-word copy an FP64 plan keeps beside the native one.
template <typename T>
inline const cx<T> *tab(const void *native, const void *dw) {
    return (const cx<T> *)(std::is_same<T, dfloat>::value ? dw : native);
}

// The fields a column-pass launch adds to base_args (single and batched launches).
template <typename T>
void cols_fields(nufft_plan p, PassArgs<T> &a, bool adjoint) {
    a.C = adjoint ? p->CB : p->C1;
    a.lgC = 0;
    while ((1 << a.lgC) < a.C) ++a.lgC;
    a.S = adjoint ? p->SB : p->S1;
    a.SB = p->SBsplit;
    a.twc = adjoint ? tab<T>(p->twst2b, p->twst2b_dw) : tab<T>(p->twst2, p->twst2_dw);   // each pass's own layout
}

// The fields a row-pass launch adds to base_args (single and batched launches).
template <typename T>
int rows_fields(nufft_plan p, PassArgs<T> &a, bool adjoint) {
    a.S = adjoint ? p->SA : p->S2;
    a.twr = adjoint ? tab<T>(p->twst1a, p->twst1a_dw) : tab<T>(p->twst1, p->twst1_dw);   // each pass's own layout
    a.chunk = p->chunkA;
    a.mbar_off = (int)p->mbar_off2;
    a.G = adjoint ? p->GA : p->G;
    a.CQ = p->CB;
    a.lgCQ = 0;
    while ((1 << a.lgCQ) < a.CQ) ++a.lgCQ;
    return a.chunk > 0 ? NUFFT_OK : NUFFT_EINVAL;
}

template <typename T>
int launch_cols(nufft_plan p, const PassArgs<T> &a0, bool adjoint, cudaStream_t s) {
    return dispatch_P(p->L2, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        const int TT = adjoint ? P / e_of<T, P, PK_COL_ADJ>() : P / e_of<T, P, PK_COL_FWD>();
        PassArgs<T> a = a0;
        cols_fields<T>(p, a, adjoint);
        const size_t smem = adjoint ? p->smemB : p->smem1;
        const dim3 block(a.C * TT);
        static SmemFlags done_b{}, done_1{};
        if (adjoint) {
            auto kern = k_passB<T, P>;
            if (int rc = set_smem(kern, smem, p->device, done_b)) return rc;
            kern<<<dim3(p->L1 / a.C, p->SBsplit), block, smem, s>>>(a);
        } else {
            auto kern = k_pass1<T, P>;
            if (int rc = set_smem(kern, smem, p->device, done_1)) return rc;
            kern<<<dim3(p->L1 / a.C, a.nranks), block, smem, s>>>(a);
        }
        return launch_status();
    });
}

template <typename T, int KM>
Beta<T, KM> beta_of(nufft_plan p) {
    Beta<T, KM> beta;
    for (int r = 0; r < KM; ++r)
        for (int q = 0; q < KM; ++q) beta.b[r][q] = (T)p->beta[r][q];
    return beta;
}

template <typename T, int KM>
int launch_rows(nufft_plan p, const PassArgs<T> &a0, bool adjoint, cudaStream_t s) {
    const Beta<T, KM> beta = beta_of<T, KM>(p);
    return dispatch_P(p->L1, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        const int TT = adjoint ? P / e_of<T, P, PK_ROW_ADJ>() : P / e_of<T, P, PK_ROW_FWD>();
        PassArgs<T> a = a0;
        if (int rc = rows_fields<T>(p, a, adjoint)) return rc;
        const int nt = adjoint ? p->ntA : (a.nranks > p->K ? p->nt2d : p->nt2);
        const size_t smem2 = p->smem2;
        const dim3 block(nt * TT);
        static SmemFlags done_a{}, done_2{};
        if (adjoint) {
            auto kern = k_passA<T, P, KM>;
            if (int rc = set_smem(kern, p->smemA, p->device, done_a)) return rc;
            kern<<<dim3(p->NB), block, p->smemA, s>>>(a, beta);
        } else {
            auto kern = k_pass2<T, P, KM>;
            if (int rc = set_smem(kern, smem2, p->device, done_2)) return rc;
            kern<<<dim3(p->NB), block, smem2, s>>>(a, beta);
        }
        return launch_status();
    });
}

// Batched launches of one class of problems (same L and rank bound KM).  rep is the
// member whose geometry covers every member: the largest rank count, and with it the
// largest shared-memory layout; grid.y is the largest rank count (pass 1) or rank
// split (pass B) of the class.  args / betas: device arrays, one entry per member.
template <typename T>
int launch_cols_many(nufft_plan rep, const PassArgs<T> *args, int nprob, int ny, bool adjoint,
                     const ManyIO &io, cudaStream_t s) {
    return dispatch_P_many(rep->L2, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        const int TT = adjoint ? P / e_of<T, P, PK_COL_ADJ>() : P / e_of<T, P, PK_COL_FWD>();
        const int C = adjoint ? rep->CB : rep->C1;
        const size_t smem = adjoint ? rep->smemB : rep->smem1;
        const dim3 grid(rep->L1 / C, ny, nprob), block(C * TT);
        static SmemFlags done_b{}, done_1{};
        if (adjoint) {
            auto kern = k_passB_many<T, P>;
            if (int rc = set_smem(kern, smem, rep->device, done_b)) return rc;
            kern<<<grid, block, smem, s>>>(args, io);
        } else {
            auto kern = k_pass1_many<T, P>;
            if (int rc = set_smem(kern, smem, rep->device, done_1)) return rc;
            kern<<<grid, block, smem, s>>>(args, io);
        }
        return launch_status();
    });
}

template <typename T, int KM>
int launch_rows_many(nufft_plan rep, const PassArgs<T> *args, const Beta<T, KM> *betas, int nprob,
                     bool adjoint, const ManyIO &io, cudaStream_t s) {
    return dispatch_P_many(rep->L1, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        const int TT = adjoint ? P / e_of<T, P, PK_ROW_ADJ>() : P / e_of<T, P, PK_ROW_FWD>();
        const int nt = adjoint ? rep->ntA : rep->nt2;
        const size_t smem = adjoint ? rep->smemA : rep->smem2;
        const dim3 grid(rep->NB, 1, nprob), block(nt * TT);
        static SmemFlags done_a{}, done_2{};
        if (adjoint) {
            auto kern = k_passA_many<T, P, KM>;
            if (int rc = set_smem(kern, smem, rep->device, done_a)) return rc;
            kern<<<grid, block, smem, s>>>(args, betas, io);
        } else {
            auto kern = k_pass2_many<T, P, KM>;
            if (int rc = set_smem(kern, smem, rep->device, done_2)) return rc;
            kern<<<grid, block, smem, s>>>(args, betas, io);
        }
        return launch_status();
    });
}

// The 2D transform of plan p (section 4).  Column pass: pass 1 in its 2D mode over the
// L1 = Ly columns of length L2 = Lx, grid.y = K (the x rank).
template <typename T>
int launch_cols_2d(nufft_plan p, const PassArgs<T> &a0, cudaStream_t s) {
    PassArgs<T> a = a0;
    cols_fields<T>(p, a, false);
    return dispatch_P(p->L2, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        constexpr int TT = P / e_of<T, P, PK_COL_FWD>();
        static SmemFlags done{};
        auto kern = k_pass1_2d<T, P>;
        if (int r = set_smem(kern, p->smem1, p->device, done)) return r;
        kern<<<dim3(p->L1 / a.C, p->K), dim3(a.C * TT), p->smem1, s>>>(a);
        return launch_status();
    });
}

// Row pass of the 2D transform: one CTA per x-grid row.  beta: [r][p] of the x
// direction (K ranks) in p->beta, of y (K2) in p->beta2.
template <typename T, int KM>
int launch_rows_2d(nufft_plan p, const PassArgs<T> &a0, cudaStream_t s) {
    PassArgs<T> a = a0;
    a.S = p->S2;
    a.G = p->G2d;   // y-ranks per group
    Beta<T, KM> bx, by;
    for (int r = 0; r < KM; ++r)
        for (int q = 0; q < KM; ++q) {
            bx.b[r][q] = (T)p->beta[r][q];
            by.b[r][q] = (T)p->beta2[r][q];
        }
    return dispatch_P(p->L1, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        constexpr int TT = P / e_of<T, P, PK_ROW_FWD>();
        static SmemFlags done{};
        auto kern = k_pass2d<T, P, KM>;
        if (int r = set_smem(kern, p->smem2, p->device, done)) return r;
        kern<<<dim3(p->L2), dim3(p->nt2 * TT), p->smem2, s>>>(a, bx, by);
        return launch_status();
    });
}

// The 2D adjoint (section 4): the row pass, one CTA per x-grid row, the y-ranks in groups
// of p->G2a; then the column pass (pass B in its 2D mode) with the plan's rank split.
template <typename T, int KM>
int launch_rows_2d_adj(nufft_plan p, const PassArgs<T> &a0, cudaStream_t s) {
    PassArgs<T> a = a0;
    a.S = p->SA;
    a.G = p->G2a;
    a.twr = (const cx<T> *)p->twst1a;
    a.CQ = p->CB;
    a.lgCQ = 0;
    while ((1 << a.lgCQ) < a.CQ) ++a.lgCQ;
    Beta<T, KM> bx, by;
    for (int r = 0; r < KM; ++r)
        for (int q = 0; q < KM; ++q) {
            bx.b[r][q] = (T)p->beta[r][q];
            by.b[r][q] = (T)p->beta2[r][q];
        }
    return dispatch_P(p->L1, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        constexpr int TT = P / e_of<T, P, PK_ROW_ADJ>();
        static SmemFlags done{};
        auto kern = k_passA2d<T, P, KM>;
        if (int r = set_smem(kern, p->smemA2d, p->device, done)) return r;
        kern<<<dim3(p->L2), dim3(p->nt2a * TT), p->smemA2d, s>>>(a, bx, by);
        return launch_status();
    });
}

template <typename T>
int launch_cols_2d_adj(nufft_plan p, const PassArgs<T> &a0, cudaStream_t s) {
    PassArgs<T> a = a0;
    cols_fields<T>(p, a, true);
    return dispatch_P(p->L2, [&](auto PC) -> int {
        constexpr int P = decltype(PC)::value;
        constexpr int TT = P / e_of<T, P, PK_COL_ADJ>();
        static SmemFlags done{};
        auto kern = k_passB2d<T, P>;
        if (int r = set_smem(kern, p->smemB, p->device, done)) return r;
        kern<<<dim3(p->L1 / a.C, p->SBsplit), dim3(a.C * TT), p->smemB, s>>>(a);
        return launch_status();
    });
}

// Common arguments of every pass of plan p (defined in exec.cu).
template <typename T>
PassArgs<T> base_args(nufft_plan p);

// explicit instantiation declarations (defined in the inst_*.cu files)
#define NUFFT_DECLARE_ROWS(T, KM) \
    extern template int launch_rows<T, KM>(nufft_plan, const PassArgs<T> &, bool, cudaStream_t);
#define NUFFT_DECLARE_COLS(T) \
    extern template int launch_cols<T>(nufft_plan, const PassArgs<T> &, bool, cudaStream_t);
#define NUFFT_DECLARE_2D_T(T, KM)                                                          \
    extern template int launch_rows_2d<T, KM>(nufft_plan, const PassArgs<T> &, cudaStream_t); \
    extern template int launch_rows_2d_adj<T, KM>(nufft_plan, const PassArgs<T> &, cudaStream_t);
#define NUFFT_DECLARE_COLS_2D_T(T)                                                       \
    extern template int launch_cols_2d<T>(nufft_plan, const PassArgs<T> &, cudaStream_t); \
    extern template int launch_cols_2d_adj<T>(nufft_plan, const PassArgs<T> &, cudaStream_t);
// batched launchers: FP32 only
#define NUFFT_DECLARE_MANY(KM)                                                            \
    extern template int launch_rows_many<float, KM>(nufft_plan, const PassArgs<float> *, \
                                                    const Beta<float, KM> *, int, bool,   \
                                                    const ManyIO &, cudaStream_t);
#define NUFFT_DECLARE_2D(KM) NUFFT_DECLARE_2D_T(float, KM)
#define NUFFT_DECLARE_COLS_2D() NUFFT_DECLARE_COLS_2D_T(float)
#define NUFFT_DECLARE_COLS_MANY()                                                                  \
    extern template int launch_cols_many<float>(nufft_plan, const PassArgs<float> *, int, int, bool, \
                                                const ManyIO &, cudaStream_t);

}  // namespace nufft
