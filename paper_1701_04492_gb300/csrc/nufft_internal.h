// nufft_internal.h -- the plan object and helpers shared by the library's sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nufft.h"

namespace nufft {

constexpr int KMAX_ALL = 16;       // Table 2.1's double row caps the rank at 16
constexpr int TW_BASE = 4096;      // low level of the two-level four-step twiddle table
constexpr int LOG2_L_MIN = 10;     // grids are at least 1024 points (two passes of 32)
constexpr int LOG2_L_MAX = 22;     // two passes of at most 2048
constexpr size_t SMEM_BUDGET = 200 * 1024;

// Real coefficient table: beta[r][p] multiplies T_p(xi) in the r-th sample factor.
template <typename T, int KM>
struct Beta { T b[KM][KM]; };

}  // namespace nufft

// The plan.  Index conventions: the grid has L = L1 * L2 points; a grid index
// t = L2 n1 + n2 (n1 < L1, n2 < L2).  Pass 1 / B transform columns of length L2
// (over k2 of k = k1 + L1 k2), pass 2 / A transform rows of length L1.
// Samples are sorted by the key (bucket, n1, row) with n2 = bucket*B2 + row.
struct nufft_plan_s {
    int64_t N = 0, M = 0, L = 0;
    int L1 = 0, L2 = 0, lg1 = 0, lg2 = 0;
    int dims = 1;          // 2: the transform of section 4 (N = m, N2 = n; L2 = Lx rows, L1 = Ly)
    int prec = 0;
    int K = 1;
    int kmax = 4;          // rank rounded up to 4, 8, 12 or 16 (kernel template)
    double gamma = 0.0, eps = 0.0;
    unsigned flags = 0;
    int device = 0;

    // execution geometry (fixed at plan time)
    int B2 = 1;            // grid rows per pass-2 bucket
    int NB = 1;            // number of buckets = L2 / B2
    int G = 1;             // ranks staged together in pass 2 (up to K + 1)
    int G2d = 1;           // 2D row pass: y-ranks transformed and gathered per group
    int G2a = 1;           // 2D adjoint row pass: y-ranks scattered and transformed per group
    int nt2a = 1;          // teams per 2D adjoint row-pass CTA
    size_t smemA2d = 0;    // dynamic shared memory of the 2D adjoint row pass
    int nt2 = 1;           // teams per pass-2 CTA (forward: K ranks)
    int nt2d = 1;          // teams per pass-2 CTA in the derivative mode (K + 1 ranks)
    int GA = 1;            // ranks staged together in pass A
    int ntA = 1;           // teams per pass-A CTA
    int C1 = 1;            // columns per pass-1 CTA
    int c1_shift = 0;      // the tuners' tile axis: C1 halved c1_shift times
    int CB = 1;            // columns per pass-B CTA
    int SBsplit = 1;       // rank splits of pass B (CTAs per column block)
    int chunkA = 512;      // samples staged per chunk in pass A
    size_t mbar_off2 = 0;  // byte offset of pass 2's mbarriers in its shared memory
    size_t smem2 = 0;      // dynamic shared memory of pass 2
    size_t smemA = 0;      // of pass A
    size_t smem1 = 0;      // of pass 1
    size_t smemB = 0;      // of pass B
    int S1 = 0, SB = 0, S2 = 0, SA = 0;   // slot strides (elements): pass 1, B, 2, A

    double beta[nufft::KMAX_ALL][nufft::KMAX_ALL] = {};   // [r][p] = w_r w_p alpha_pr
    double alpha[nufft::KMAX_ALL][nufft::KMAX_ALL] = {};  // a_pr = i^r alpha_pr

    // device memory owned by the plan
    int32_t *tsorted = nullptr, *perm = nullptr, *bstart = nullptr, *t_j = nullptr;
    void *dsorted = nullptr;   // d in sorted order, plan precision
    double *d_j = nullptr;     // d in sample order, FP64 (unfused factors)
    void *twst1 = nullptr, *twst2 = nullptr;   // stage twiddle tables: pass 2 (L1), pass 1 (L2)
    void *twst1a = nullptr, *twst2b = nullptr; // and pass A (L1), pass B (L2): each pass's own E
    void *twhi = nullptr, *twlo = nullptr;     // four-step twiddle, two levels
    // FP64 plans: the same four stage tables and four-step levels in double-word form,
    // for the double-word kernels of the fused FP64 exec
    void *twst1_dw = nullptr, *twst1a_dw = nullptr, *twst2_dw = nullptr, *twst2b_dw = nullptr;
    void *twhi_dw = nullptr, *twlo_dw = nullptr;
    void *Y = nullptr;         // (K + 1) * L complex: intermediate between the passes
    void *fscr = nullptr;      // M complex: partial sums when G < K
    void *cstage = nullptr, *fstage = nullptr;   // exec_host staging
    void *U = nullptr, *V = nullptr, *Xg = nullptr;   // unfused comparator
    void *part = nullptr;      // pass B partial sums, SBsplit x L complex
    int *counters = nullptr;   // pass B tickets, one per column block
    int *err = nullptr;        // device error word: bounded waits that timed out
    void *Ufac = nullptr;      // FP64 plans: u_r in sorted order, M x K complex (double-word)
    void *Vfac = nullptr;      // FP64 plans: v_r, K x N real (double-word)
    int64_t work_bytes = 0;

    // the 2D transform: the y direction (x uses N, K, gamma, beta, t_j, d_j, dsorted)
    int64_t N2 = 0;            // n
    int K2 = 1;
    double gamma2 = 0.0;
    double beta2[nufft::KMAX_ALL][nufft::KMAX_ALL] = {};
    double alpha2[nufft::KMAX_ALL][nufft::KMAX_ALL] = {};
    int32_t *t2_j = nullptr;   // t^y in sample order
    double *d2_j = nullptr;    // d^y in sample order
    void *dsorted2 = nullptr;  // d^y in sorted order
    void *vy = nullptr;        // T_r2(2 k2 / n - 1), K2 x L1

    // the inverse transform (section 3.3), built by the first nufft2_inverse call
    nufft_plan_s *inv_fft = nullptr;   // FFT of P >= 2N points (a gamma = 0 plan)
    int64_t inv_P = 0;
    void *inv_lam = nullptr, *inv_x = nullptr, *inv_z = nullptr;   // P complex each
    void *inv_r = nullptr, *inv_p = nullptr, *inv_ap = nullptr;    // N complex each
    double *inv_part = nullptr, *inv_scal = nullptr;               // reductions, scalars
    double *inv_host = nullptr;                                    // pinned readback

    // nufft2_step_host (made by nufft2_plan_reserve): device copies of g, f', A^H g and
    // gx; a copy stream and events
    void *st_g = nullptr, *st_fp = nullptr, *st_gc = nullptr, *st_gx = nullptr;
    cudaStream_t st_copy = nullptr;
    cudaEvent_t st_ev[6] = {};

    // batches of coefficient vectors on this plan (shared samples), for up to sb_cap
    // members (made by nufft2_plan_reserve): per-member slices of the intermediate,
    // partial sums, pass B's partials and tickets; the members' kernel arguments (six
    // sets of sb_cap: forward, forward with f', adjoint; two passes each) and
    // coefficient tables
    int64_t sb_cap = 0;
    void *sb_Y = nullptr, *sb_fscr = nullptr, *sb_part = nullptr;
    int *sb_cnt = nullptr;
    void *sb_args = nullptr, *sb_beta = nullptr;

    // NUFFT_PLAN_TIMING: events around each launch of the last exec call
    cudaEvent_t ev[8] = {};
    int nev = 0;       // events recorded by the last exec call
};

namespace nufft {
// The current device's SM count, for launch-geometry choices at plan time (152 on
// GB300, which is also the value taken if the query fails: the choices are heuristics).
inline int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        (void)cudaGetLastError();
        return 152;
    }
    return sms;
}

// Record the next timing event (no-op without NUFFT_PLAN_TIMING).
inline int mark(nufft_plan p, cudaStream_t s, bool first) {
    if (!(p->flags & NUFFT_PLAN_TIMING)) return NUFFT_OK;
    if (first) p->nev = 0;
    if (p->nev >= 8) return NUFFT_OK;
    if (cudaEventRecord(p->ev[p->nev], s) != cudaSuccess) { (void)cudaGetLastError(); return NUFFT_ECUDA; }
    ++p->nev;
    return NUFFT_OK;
}
}  // namespace nufft

namespace nufft {

// plan.cu: a plan with a given layout (the autotuners' axes): grid size L (0: the
// default), the four-step split, pass 1's columns per CTA halved c1_shift times
struct Layout {
    int64_t L = 0;
    bool long_cols = false;
    int c1_shift = 0;
};
int plan_layout(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps, int prec,
                const Layout &lay, unsigned flags, cudaStream_t s);

// hooks.cu: cudaMalloc, unless a test has injected a failure (nufft_test_fail_alloc)
cudaError_t dev_malloc(void **p, size_t bytes);

// host_math.cpp
double bessel_j_int(int n, double z);
void chebyshev_alpha(int K, double gamma, double *alpha /* K*K, [p*K + r] */);
double tail_bound(int K, double gamma);
int choose_rank(double eps, double gamma);
void twiddle(int64_t n, int64_t m, double *c, double *s);   // exp(-2 pi i m / n)

// exec_*.cu
template <typename T> int exec_forward(nufft_plan p, const void *c, void *f, cudaStream_t s);
template <typename T> int exec_adjoint(nufft_plan p, const void *g, void *c, cudaStream_t s);
template <typename T> int exec_dx(nufft_plan p, const void *c, const void *g, void *gx, int acc,
                                  cudaStream_t s);
template <typename T> int exec_unfused(nufft_plan p, const void *c, void *f, cudaStream_t s);
template <typename T> int plan_geometry(nufft_plan p);
template <typename T> int plan_unfused_factors(nufft_plan p, cudaStream_t s);
template <typename T> int plan_factor_tables(nufft_plan p, cudaStream_t s);
int reserve_step_host(nufft_plan p, cudaStream_t s);   // exec.cu: nufft2_step_host's buffers

}  // namespace nufft

#define NUFFT_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) {                               \
            (void)cudaGetLastError();                          \
            return e_ == cudaErrorMemoryAllocation ? NUFFT_ENOMEM : NUFFT_ECUDA; \
        }                                                      \
    } while (0)
