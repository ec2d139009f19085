// noalloc.cu -- the forward transform for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another runtime's
// memory pool or allocator callback, plug-ins whose host forbids device
// allocation, or code that must not allocate on a latency-critical path.  For
// them nufft2_exec_noalloc computes the same FP32 NUFFT-II as nufft2_plan +
// nufft2_exec, without a plan: everything the transform needs between its kernels
// lives in one file-scope device array, g_scratch, of fixed size (about 17 MiB,
// held by every GPU that loads the library until the process exits).
//
// The host never dereferences g_scratch: on the first call on each device, with
// that device current, cudaGetSymbolAddress gives its device address, which is
// cached per device and passed to the kernels.  Every call synchronises its stream
// (to read gamma, and at the end to read the error word), so no call can be made
// inside a stream capture.  Every call reuses the same array (it keeps the previous
// call's contents; the words that must start at zero are cleared on each call),
// so calls whose work overlaps on the GPU race with each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "passes.cuh"

namespace nufft {

NUFFT_DECLARE_ROWS(float, 4)
NUFFT_DECLARE_ROWS(float, 8)
NUFFT_DECLARE_ROWS(float, 12)
NUFFT_DECLARE_ROWS(float, 16)
NUFFT_DECLARE_COLS(float)

namespace {

constexpr int NA_LOG2_MAX = 16;
constexpr int64_t NA_LMAX = (int64_t)1 << NA_LOG2_MAX;   // grid points, frequencies, samples
constexpr int64_t NA_MMAX = NA_LMAX;
constexpr int NA_KMAX = KMAX_ALL;

// Byte layout of the scratch array (every part 256-byte aligned).
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_Y = 0;                                                     // K x L complex
constexpr size_t OFF_X = OFF_Y + al256((size_t)NA_KMAX * NA_LMAX * 8);          // K x L complex
constexpr size_t OFF_T = OFF_X + al256((size_t)NA_KMAX * NA_LMAX * 8);          // M int32
constexpr size_t OFF_D = OFF_T + al256((size_t)NA_MMAX * 4);                    // M double
constexpr size_t OFF_TW1 = OFF_D + al256((size_t)NA_MMAX * 8);                  // stage twiddles, rows
constexpr size_t OFF_TW2 = OFF_TW1 + al256((size_t)2 * 256 * 8);               // stage twiddles, columns
constexpr size_t OFF_TWHI = OFF_TW2 + al256((size_t)2 * 256 * 8);              // four-step, high level
constexpr size_t OFF_TWLO = OFF_TWHI + al256((size_t)(NA_LMAX / 4096 + 1) * 8);
constexpr size_t OFF_BSTART = OFF_TWLO + al256((size_t)4096 * 8);               // zeros (unused buckets)
constexpr size_t OFF_WORDS = OFF_BSTART + al256((size_t)(256 + 1) * 4);        // gamma bits, flags
constexpr size_t SCRATCH_BYTES = OFF_WORDS + 256;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// per device: the device address of g_scratch
std::mutex g_mu;
void *g_addr[64] = {};

int scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return NUFFT_EUNSUPPORTED;
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return NUFFT_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return NUFFT_OK;
}

// s = rint(L x), t = s mod L, d = (L x - s) N / L, gamma = max |d| (eqs. (2.8)-(2.9))
__global__ void na_round(const double *__restrict__ x, int64_t M, double Ld, double ratio,
                         int32_t *__restrict__ t_out, double *__restrict__ d_out,
                         unsigned long long *__restrict__ gamma_bits, int *__restrict__ bad) {
    unsigned long long local = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double Lx = Ld * x[j];
        if (!isfinite(Lx) || fabs(Lx) >= 4503599627370496.0) {
            atomicOr(bad, 1);
            t_out[j] = 0;
            d_out[j] = 0.0;
            continue;
        }
        const double s = rint(Lx);
        const double t = s - floor(s / Ld) * Ld;
        const double d = (Lx - s) * ratio;
        t_out[j] = (int32_t)t;
        d_out[j] = d;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(d));
        local = bits > local ? bits : local;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, local, o);
        local = v > local ? v : local;
    }
    if ((threadIdx.x & 31) == 0 && local) atomicMax(gamma_bits, local);
}

// Twiddle tables, computed in FP64 with sincospi and rounded to FP32:
//   stage table of a length-P team FFT (layout of TeamFft: stage 1 radix R1 after
//   R0 points, stage 2 radix R2 after R0 R1 points, entry (i - 1) NS + j), and the
//   two-level four-step table w_L^m = hi[m >> 12] lo[m & 4095].
__device__ float2 w_exact(long long n, long long m) {
    double s, c;
    sincospi(2.0 * (double)(m % n) / (double)n, &s, &c);
    return make_float2((float)c, (float)(-s));
}

__global__ void na_tables(int P1, int EM1, int P2, int EM2, int64_t L, float2 *tw1, float2 *tw2, float2 *hi,
                          float2 *lo, int32_t *bstart, int nb1) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int pass = 0; pass < 2; ++pass) {
        const int P = pass ? P2 : P1;
        float2 *tw = pass ? tw2 : tw1;
        const int EM = pass ? EM2 : EM1;
        const int E = P < EM ? P : EM, TT = P / E;
        const int R0 = E, R1 = TT > 1 ? (TT < E ? TT : E) : 1, R2 = TT / R1;
        const int n1 = (R1 - 1) * R0, n2 = R2 > 1 ? (R2 - 1) * R0 * R1 : 0;
        for (int q = tid; q < n1; q += nth) tw[q] = w_exact((long long)R0 * R1, (long long)(q / R0 + 1) * (q % R0));
        for (int q = tid; q < n2; q += nth) {
            const int NS = R0 * R1;
            tw[n1 + q] = w_exact((long long)NS * R2, (long long)(q / NS + 1) * (q % NS));
        }
        if (n1 + n2 == 0 && tid == 0) tw[0] = make_float2(1.f, 0.f);
    }
    const long long nlo = L < 4096 ? L : 4096, nhi = L / 4096 > 1 ? L / 4096 : 1;
    for (long long q = tid; q < nlo; q += nth) lo[q] = w_exact(L, q);
    for (long long q = tid; q < nhi; q += nth) hi[q] = w_exact(L, q * 4096);
    for (int q = tid; q <= nb1; q += nth) bstart[q] = 0;
}

// f_j = exp(-i pi d_j) sum_r mu_r(xi_j) X_r[t_j] in sample order (eq. (2.11), step 2)
template <int KM>
__global__ void na_gather(const float2 *__restrict__ X, const int32_t *__restrict__ t,
                          const double *__restrict__ d, int64_t M, int64_t L, int K, float inv_gamma,
                          const Beta<float, KM> beta, float2 *__restrict__ f) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float dj = (float)d[j];
        const float xi = dj * inv_gamma;
        float Tp[KM];
        Tp[0] = 1.f;
        if (KM > 1) Tp[1] = xi;
#pragma unroll
        for (int q = 2; q < KM; ++q) Tp[q] = fmaf(2.f * xi, Tp[q - 1], -Tp[q - 2]);
        float2 acc = make_float2(0.f, 0.f);
        const int tj = t[j];
#pragma unroll
        for (int r = 0; r < KM; ++r) {
            if (r < K) {
                float mu = 0.f;
#pragma unroll
                for (int q = (r & 1); q < KM; q += 2) mu = fmaf(beta.b[r][q], Tp[q], mu);
                const float2 x = X[(int64_t)r * L + tj];
                acc.x = fmaf(mu, x.x, acc.x);
                acc.y = fmaf(mu, x.y, acc.y);
            }
        }
        float sn, cs;
        sincospif(dj, &sn, &cs);
        f[j] = make_float2(fmaf(acc.x, cs, acc.y * sn), fmaf(acc.y, cs, -acc.x * sn));
    }
}

template <int KM>
int gather_launch(const float2 *X, const int32_t *t, const double *d, int64_t M, int64_t L, int K,
                  float inv_gamma, const double (&beta)[KMAX_ALL][KMAX_ALL], float2 *f, cudaStream_t s) {
    Beta<float, KM> b;
    for (int r = 0; r < KM; ++r)
        for (int q = 0; q < KM; ++q) b.b[r][q] = (float)beta[r][q];
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 152 * 8));
    na_gather<KM><<<grid, 256, 0, s>>>(X, t, d, M, L, K, inv_gamma, b, f);
    return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

}  // namespace
}  // namespace nufft

extern "C" int nufft2_exec_noalloc(int64_t N, int64_t M, const double *x_dev, double eps,
                                   const void *c_dev, void *f_dev, void *stream) {
    using namespace nufft;
    if (N < 1 || M < 0 || !(eps > 0.0 && eps < 1.0) || !c_dev || (M > 0 && (!x_dev || !f_dev)))
        return NUFFT_EINVAL;
    if (N > NA_LMAX || M > NA_MMAX) return NUFFT_EUNSUPPORTED;   // beyond the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return NUFFT_ECUDA; }
    unsigned char *base = nullptr;
    if (int rc = scratch_address(dev, &base)) return rc;
    if (M == 0) return NUFFT_OK;
    cudaStream_t s = (cudaStream_t)stream;

    // the plan lives on the host stack; its device pointers point into the scratch
    nufft_plan_s pl;
    pl.N = N;
    pl.M = M;
    pl.L = (int64_t)1 << LOG2_L_MIN;
    while (pl.L < N) pl.L <<= 1;
    if (pl.L > NA_LMAX) return NUFFT_EUNSUPPORTED;
    int lg = 0;
    while (((int64_t)1 << lg) < pl.L) ++lg;
    pl.lg1 = (lg + 1) / 2;
    pl.lg2 = lg / 2;
    pl.L1 = 1 << pl.lg1;
    pl.L2 = 1 << pl.lg2;
    pl.prec = NUFFT_F32;
    pl.eps = eps;
    pl.device = dev;

    int32_t *t = (int32_t *)(base + OFF_T);
    double *d = (double *)(base + OFF_D);
    unsigned long long *gbits = (unsigned long long *)(base + OFF_WORDS);
    int *bad = (int *)(base + OFF_WORDS + 8);
    int *err = (int *)(base + OFF_WORDS + 16);
    NUFFT_CUDA_TRY(cudaMemsetAsync(base + OFF_WORDS, 0, 256, s));   // gamma, flags start at zero
    const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 152 * 8));
    na_round<<<rgrid, 256, 0, s>>>(x_dev, M, (double)pl.L, (double)N / (double)pl.L, t, d, gbits, bad);
    NUFFT_CUDA_TRY(cudaGetLastError());
    unsigned long long hw[2] = {0, 0};
    NUFFT_CUDA_TRY(cudaMemcpyAsync(hw, base + OFF_WORDS, sizeof(hw), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if ((int)(hw[1] & 0xffffffffu)) return NUFFT_EINVAL;   // non-finite or too large x
    double gamma;
    std::memcpy(&gamma, &hw[0], sizeof(gamma));
    pl.gamma = gamma;
    pl.K = choose_rank(eps, gamma);
    pl.kmax = std::min(KMAX_ALL, ((pl.K + 3) / 4) * 4);
    if (gamma == 0.0) {
        pl.beta[0][0] = 1.0;
    } else {
        double al[KMAX_ALL * KMAX_ALL];
        chebyshev_alpha(pl.K, gamma, al);
        for (int r = 0; r < pl.K; ++r)
            for (int q = 0; q < pl.K; ++q)
                pl.beta[r][q] = (r == 0 ? 0.5 : 1.0) * (q == 0 ? 0.5 : 1.0) * al[q * pl.K + r];
    }
    if (int rc = plan_geometry<float>(&pl)) return rc;
    if (pl.NB + 1 > 257) return NUFFT_EUNSUPPORTED;

    float2 *tw1 = (float2 *)(base + OFF_TW1), *tw2 = (float2 *)(base + OFF_TW2);
    float2 *hi = (float2 *)(base + OFF_TWHI), *lo = (float2 *)(base + OFF_TWLO);
    int32_t *bstart = (int32_t *)(base + OFF_BSTART);
    // pass 2 (rows) and pass 1 (columns), each with its own values per thread
    na_tables<<<16, 256, 0, s>>>(pl.L1, EmaxT<float, PK_ROW_FWD>::v, pl.L2, EmaxT<float, PK_COL_FWD>::v, pl.L, tw1,
                                 tw2, hi, lo, bstart, pl.NB);
    pl.twst1 = tw1;   // the launchers take each pass's table from the plan
    pl.twst2 = tw2;
    NUFFT_CUDA_TRY(cudaGetLastError());

    PassArgs<float> a{};
    a.in = (const float2 *)c_dev;
    a.Y = (float2 *)(base + OFF_Y);
    a.out = (float2 *)(base + OFF_X);
    a.bstart = bstart;
    a.twc = tw2;
    a.twr = tw1;
    a.twhi = hi;
    a.twlo = lo;
    a.err = err;
    a.N = N;
    a.M = M;
    a.L = pl.L;
    a.L1 = pl.L1;
    a.L2 = pl.L2;
    a.lg1 = pl.lg1;
    a.lg2 = pl.lg2;
    a.K = pl.K;
    a.nranks = pl.K;
    a.piN = (float)(3.14159265358979323846 * (double)N);
    a.G = pl.G;
    a.B2 = pl.B2;
    a.mode = MODE_PLAIN_OUT;
    a.inv_gamma = gamma > 0.0 ? (float)(1.0 / gamma) : 0.f;
    // step 1: X_r = F_L (v_r o c) for all r, natural order, in the scratch
    if (int rc = launch_cols<float>(&pl, a, false, s)) return rc;
    int rc = NUFFT_EUNSUPPORTED;
    switch (pl.kmax) {
        case 4: rc = launch_rows<float, 4>(&pl, a, false, s); break;
        case 8: rc = launch_rows<float, 8>(&pl, a, false, s); break;
        case 12: rc = launch_rows<float, 12>(&pl, a, false, s); break;
        case 16: rc = launch_rows<float, 16>(&pl, a, false, s); break;
    }
    if (rc) return rc;
    // step 2: gather, U-scale, rank-sum
    const float2 *X = (const float2 *)(base + OFF_X);
    switch (pl.kmax) {
        case 4: rc = gather_launch<4>(X, t, d, M, pl.L, pl.K, a.inv_gamma, pl.beta, (float2 *)f_dev, s); break;
        case 8: rc = gather_launch<8>(X, t, d, M, pl.L, pl.K, a.inv_gamma, pl.beta, (float2 *)f_dev, s); break;
        case 12: rc = gather_launch<12>(X, t, d, M, pl.L, pl.K, a.inv_gamma, pl.beta, (float2 *)f_dev, s); break;
        default: rc = gather_launch<16>(X, t, d, M, pl.L, pl.K, a.inv_gamma, pl.beta, (float2 *)f_dev, s); break;
    }
    if (rc) return rc;
    // the passes' bounded waits and (NUFFT_CHECK builds) index checks report into the
    // error word; the caller has no plan to ask, so it is read here, once the work is done
    int h = 0;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return (h & ERR_TIMEOUT) ? NUFFT_ETIMEOUT : NUFFT_ECHECK;
    return NUFFT_OK;
}
