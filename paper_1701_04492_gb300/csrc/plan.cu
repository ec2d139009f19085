// plan.cu -- the planning stage (section 2.3 "Planning the transform").
//
// Device work, FP64: s = rint(L x), t = s mod L, delta = L x - s (eqs. (2.8)-(2.9)),
// d = delta N / L and gamma = max |d| (section 2.1.2).  Host work, FP64: the rank K
// and the coefficients a_pr of eq. (2.6).  Then a stable LSD radix sort groups the
// samples by the pass-2 tile that holds their grid point, and the twiddle tables
// are built.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "async_copy.cuh"
#include "fft_team.cuh"
#include "fill.cuh"
#include "nufft_internal.h"
#include "nvtx_range.h"

namespace nufft {
namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_CHUNK = 4096;          // elements per CTA
constexpr int SORT_BITS = 8;
constexpr int SORT_BINS = 1 << SORT_BITS;

// ---- eqs. (2.8)-(2.9) ---------------------------------------------------------

__global__ void k_round(const double *__restrict__ x, int64_t M, double Ld, int64_t L,
                        double ratio, int32_t *__restrict__ t_out, double *__restrict__ d_out,
                        unsigned long long *__restrict__ gamma_bits, int *__restrict__ bad) {
    unsigned long long local = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double xj = x[j];
        const double Lx = Ld * xj;                     // exact: L is a power of two
        if (!isfinite(Lx) || fabs(Lx) >= 4503599627370496.0) {   // 2^52
            atomicOr(bad, 1);
            t_out[j] = 0;
            d_out[j] = 0.0;
            continue;
        }
        const double s = rint(Lx);                      // nearest, ties to even
        const double q = floor(s / Ld);                 // exact quotient of a power of two
        const double t = s - q * Ld;                    // Euclidean: t in [0, L)
        const double delta = Lx - s;                    // exact, |delta| <= 1/2
        const double d = delta * ratio;
        t_out[j] = (int32_t)t;
        d_out[j] = d;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(d));
        local = bits > local ? bits : local;
    }
    // warp max, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, local, o);
        local = v > local ? v : local;
    }
    if ((threadIdx.x & 31) == 0 && local) atomicMax(gamma_bits, local);
}

// ---- stable LSD radix sort of (key, index) ---------------------------------------

__device__ __forceinline__ int32_t sort_key(int32_t t, int lg1, int lg2, int B2) {
    const int32_t n2 = t & ((1 << lg2) - 1);
    const int32_t n1 = t >> lg2;
    const int32_t bucket = n2 / B2;
    const int32_t row = n2 - bucket * B2;
    return (bucket << lg1) * B2 + n1 * B2 + row;
}

__global__ void k_keys(const int32_t *__restrict__ t, int64_t M, int lg1, int lg2, int B2,
                       int32_t *__restrict__ key, int32_t *__restrict__ val) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        key[j] = sort_key(t[j], lg1, lg2, B2);
        val[j] = (int32_t)j;
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_hist(const int32_t *__restrict__ key, int64_t M,
                                                      int shift, int nchunks,
                                                      int32_t *__restrict__ counts) {
    __shared__ int h[SORT_BINS];
    for (int i = threadIdx.x; i < SORT_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int i = threadIdx.x; i < SORT_CHUNK; i += blockDim.x) {
        const int64_t j = base + i;
        if (j < M) atomicAdd(&h[(key[j] >> shift) & (SORT_BINS - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SORT_BINS; i += blockDim.x)
        counts[(int64_t)i * nchunks + blockIdx.x] = h[i];
}

// Exclusive scan of n counts by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(int32_t *__restrict__ counts, int64_t n) {
    __shared__ int64_t part[1024];
    const int64_t seg = (n + 1023) / 1024;
    const int64_t lo = threadIdx.x * seg, hi = min(n, lo + seg);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - s;   // exclusive prefix of this segment
    for (int64_t i = lo; i < hi; ++i) {
        const int32_t c = counts[i];
        counts[i] = (int32_t)run;
        run += c;
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_scatter(const int32_t *__restrict__ kin,
                                                         const int32_t *__restrict__ vin, int64_t M,
                                                         int shift, int nchunks,
                                                         const int32_t *__restrict__ offsets,
                                                         int32_t *__restrict__ kout,
                                                         int32_t *__restrict__ vout) {
    constexpr int NW = SORT_THREADS / 32;
    constexpr int PER_WARP = SORT_CHUNK / NW;
    __shared__ int wc[NW][SORT_BINS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < NW * SORT_BINS; i += blockDim.x) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK + w * PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    // 1) per-warp digit counts
    for (int s = 0; s < PER_WARP; s += 32) {
        const int64_t j = base + s + lane;
        const int dg = j < M ? ((kin[j] >> shift) & (SORT_BINS - 1)) : SORT_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < SORT_BINS && (peers & lt) == 0) wc[w][dg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // 2) turn counts into start positions: chunk offset + earlier warps of this chunk
    for (int dg = threadIdx.x; dg < SORT_BINS; dg += blockDim.x) {
        int run = offsets[(int64_t)dg * nchunks + blockIdx.x];
        for (int ww = 0; ww < NW; ++ww) {
            const int c = wc[ww][dg];
            wc[ww][dg] = run;
            run += c;
        }
    }
    __syncthreads();
    // 3) stable placement, in input order within each warp
    for (int s = 0; s < PER_WARP; s += 32) {
        const int64_t j = base + s + lane;
        const int dg = j < M ? ((kin[j] >> shift) & (SORT_BINS - 1)) : SORT_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < SORT_BINS) {
            const int pos = wc[w][dg] + __popc(peers & lt);
            kout[pos] = kin[j];
            vout[pos] = vin[j];
        }
        __syncwarp();
        if (dg < SORT_BINS && (peers & lt) == 0) wc[w][dg] += __popc(peers);
        __syncwarp();
    }
}

template <typename T>
__global__ void k_build(const int32_t *__restrict__ perm, const int32_t *__restrict__ t_j,
                        const double *__restrict__ d_j, int64_t M, int32_t *__restrict__ tsorted,
                        T *__restrict__ dsorted) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = perm[i];
        tsorted[i] = t_j[j];
        dsorted[i] = (T)d_j[j];
    }
}

// bstart[b] = first sorted position whose bucket is >= b, b = 0..NB.
__global__ void k_bstart(const int32_t *__restrict__ keys, int64_t M, int bucket_shift, int NB,
                         int32_t *__restrict__ bstart) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int prev = i == 0 ? -1 : (keys[i - 1] >> bucket_shift);
        const int cur = i == M ? NB : (keys[i] >> bucket_shift);
        for (int b = prev + 1; b <= cur; ++b) bstart[b] = (int32_t)i;
    }
}

int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <typename T>
int upload_table(void **dst, const std::vector<double> &re, const std::vector<double> &im,
                 cudaStream_t s, int64_t *bytes) {
    const size_t n = re.size();
    std::vector<T> h(2 * n);
    for (size_t i = 0; i < n; ++i) { h[2 * i] = (T)re[i]; h[2 * i + 1] = (T)im[i]; }
    NUFFT_CUDA_TRY(dev_malloc((void **)dst, h.size() * sizeof(T)));
    *bytes += (int64_t)(h.size() * sizeof(T));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));   // h goes out of scope
    return NUFFT_OK;
}

// Stage twiddles of a length-P team FFT (the schedule of TeamFft in fft_team.cuh:
// radices E, then min(E, P/E), then the rest): stage s >= 1 with radix R after NS
// points holds w_{NS R}^{i j} at offset + (i - 1) NS + j.
template <typename T>
int stage_table(int P, int EM, void **dst, cudaStream_t s, int64_t *bytes) {
    const int E = std::min(EM, P), TT = P / E;
    const int R0 = E, R1 = TT > 1 ? std::min(E, TT) : 1, R2 = TT / R1;
    std::vector<double> re, im;
    auto add_stage = [&](int R, int NS) {
        for (int i = 1; i < R; ++i)
            for (int j = 0; j < NS; ++j) {
                double c, sn;
                twiddle((int64_t)NS * R, (int64_t)i * j, &c, &sn);
                re.push_back(c);
                im.push_back(sn);
            }
    };
    if (R1 > 1) add_stage(R1, R0);
    if (R2 > 1) add_stage(R2, R0 * R1);
    if (re.empty()) { re.push_back(1.0); im.push_back(0.0); }
    return upload_table<T>(dst, re, im, s, bytes);
}

template <typename T>
int build_tables(nufft_plan p, cudaStream_t s) {
    // each pass's stage table for its own values per thread
    int rc = stage_table<T>(p->L1, EmaxT<T, PK_ROW_FWD>::v, &p->twst1, s, &p->work_bytes);
    if (rc) return rc;
    if ((rc = stage_table<T>(p->L1, EmaxT<T, PK_ROW_ADJ>::v, &p->twst1a, s, &p->work_bytes))) return rc;
    if ((rc = stage_table<T>(p->L2, EmaxT<T, PK_COL_FWD>::v, &p->twst2, s, &p->work_bytes))) return rc;
    if ((rc = stage_table<T>(p->L2, EmaxT<T, PK_COL_ADJ>::v, &p->twst2b, s, &p->work_bytes))) return rc;
    std::vector<double> re, im;
    // four-step twiddle w_L^m = w_L^(4096 m_hi) * w_L^(m_lo), m = 4096 m_hi + m_lo
    const int64_t nlo = std::min<int64_t>(p->L, TW_BASE);
    const int64_t nhi = std::max<int64_t>(1, p->L / TW_BASE);
    re.assign(nlo, 0.0); im.assign(nlo, 0.0);
    for (int64_t m = 0; m < nlo; ++m) twiddle(p->L, m, &re[m], &im[m]);
    if ((rc = upload_table<T>(&p->twlo, re, im, s, &p->work_bytes))) return rc;
    std::vector<double> rel = re, iml = im;
    re.assign(nhi, 0.0); im.assign(nhi, 0.0);
    for (int64_t m = 0; m < nhi; ++m) twiddle(p->L, m * TW_BASE, &re[m], &im[m]);
    if ((rc = upload_table<T>(&p->twhi, re, im, s, &p->work_bytes))) return rc;
    if constexpr (std::is_same<T, double>::value) {
        // the double-word copies for the fused FP64 exec (same entries, rounded to hi + lo)
        if ((rc = stage_table<dfloat>(p->L1, EmaxT<dfloat, PK_ROW_FWD>::v, &p->twst1_dw, s, &p->work_bytes))) return rc;
        if ((rc = stage_table<dfloat>(p->L1, EmaxT<dfloat, PK_ROW_ADJ>::v, &p->twst1a_dw, s, &p->work_bytes))) return rc;
        if ((rc = stage_table<dfloat>(p->L2, EmaxT<dfloat, PK_COL_FWD>::v, &p->twst2_dw, s, &p->work_bytes))) return rc;
        if ((rc = stage_table<dfloat>(p->L2, EmaxT<dfloat, PK_COL_ADJ>::v, &p->twst2b_dw, s, &p->work_bytes))) return rc;
        if ((rc = upload_table<dfloat>(&p->twlo_dw, rel, iml, s, &p->work_bytes))) return rc;
        if ((rc = upload_table<dfloat>(&p->twhi_dw, re, im, s, &p->work_bytes))) return rc;
    }
    return NUFFT_OK;
}

// Bucket the samples: a stable LSD radix sort by (bucket, n1, row) of the grid index
// t_j, then t and d (and d2, for the 2D transform) in sorted order and the bucket
// boundaries.
template <typename T>
int sort_samples(nufft_plan p, cudaStream_t s) {
    const int64_t M = p->M;
    struct Scratch {
        int32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *cnt = nullptr;
        ~Scratch() { cudaFree(ka); cudaFree(va); cudaFree(kb); cudaFree(vb); cudaFree(cnt); }
    } sc;
    const size_t Mi = (size_t)std::max<int64_t>(M, 1);
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->tsorted, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->perm, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->dsorted, Mi * sizeof(T)));
    if (p->dims == 2) NUFFT_CUDA_TRY(dev_malloc((void **)&p->dsorted2, Mi * sizeof(T)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->bstart, (size_t)(p->NB + 1) * sizeof(int32_t)));
    p->work_bytes += (int64_t)(Mi * (2 * sizeof(int32_t) + sizeof(T)) + (p->NB + 1) * sizeof(int32_t));
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.ka, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.va, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.kb, Mi * sizeof(int32_t)));
    const int nchunks = (int)std::max<int64_t>(1, (M + SORT_CHUNK - 1) / SORT_CHUNK);
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.cnt, (size_t)SORT_BINS * nchunks * sizeof(int32_t)));
    int32_t *kin = sc.ka, *vin = sc.va, *kout = sc.kb, *vout = p->perm;
    if (M > 0) {
        k_keys<<<grid_for(M, 256), 256, 0, s>>>(p->t_j, M, p->lg1, p->lg2, p->B2, kin, vin);
        NUFFT_CUDA_TRY(cudaGetLastError());
        const int lgL = p->lg1 + p->lg2;
        const int passes = (lgL + SORT_BITS - 1) / SORT_BITS;
        NUFFT_CUDA_TRY(dev_malloc((void **)&sc.vb, Mi * sizeof(int32_t)));
        for (int ps = 0; ps < passes; ++ps) {
            // the last pass lands in perm
            vout = (ps == passes - 1) ? p->perm : (vin == sc.va ? sc.vb : sc.va);
            kout = (kin == sc.ka) ? sc.kb : sc.ka;
            const int shift = ps * SORT_BITS;
            k_hist<<<nchunks, SORT_THREADS, 0, s>>>(kin, M, shift, nchunks, sc.cnt);
            k_scan<<<1, 1024, 0, s>>>(sc.cnt, (int64_t)SORT_BINS * nchunks);
            k_scatter<<<nchunks, SORT_THREADS, 0, s>>>(kin, vin, M, shift, nchunks, sc.cnt, kout, vout);
            NUFFT_CUDA_TRY(cudaGetLastError());
            kin = kout;
            vin = vout;
        }
        k_build<T><<<grid_for(M, 256), 256, 0, s>>>(p->perm, p->t_j, p->d_j, M, p->tsorted,
                                                    (T *)p->dsorted);
        if (p->dims == 2)   // d^y in the same order (t is written again, unchanged)
            k_build<T><<<grid_for(M, 256), 256, 0, s>>>(p->perm, p->t_j, p->d2_j, M, p->tsorted,
                                                        (T *)p->dsorted2);
        NUFFT_CUDA_TRY(cudaGetLastError());
    }
    // bucket = key >> (lg1 + log2 B2)
    int lgB2 = 0;
    while ((1 << lgB2) < p->B2) ++lgB2;
    k_bstart<<<grid_for(M + 1, 256), 256, 0, s>>>(kin, M, p->lg1 + lgB2, p->NB, p->bstart);
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));   // before the scratch is freed
    return NUFFT_OK;
}

template <typename T>
int plan_device(nufft_plan p, const double *x, cudaStream_t s) {
    const int64_t M = p->M;
    struct Scratch {
        unsigned long long *gbits = nullptr;
        int *bad = nullptr;
        ~Scratch() { cudaFree(gbits); cudaFree(bad); }
    } sc;
    const size_t Mi = (size_t)std::max<int64_t>(M, 1);
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.gbits, sizeof(unsigned long long)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.bad, sizeof(int)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->t_j, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->d_j, Mi * sizeof(double)));
    p->work_bytes += (int64_t)(Mi * (sizeof(int32_t) + sizeof(double)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(sc.gbits, 0, sizeof(unsigned long long), s));
    NUFFT_CUDA_TRY(cudaMemsetAsync(sc.bad, 0, sizeof(int), s));
    if (M > 0) {
        k_round<<<grid_for(M, 256), 256, 0, s>>>(x, M, (double)p->L, p->L,
                                                 (double)p->N / (double)p->L, p->t_j, p->d_j,
                                                 sc.gbits, sc.bad);
        NUFFT_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long gb = 0;
    int bad = 0;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(&gb, sc.gbits, sizeof(gb), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(&bad, sc.bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return NUFFT_EINVAL;
    double gamma;
    std::memcpy(&gamma, &gb, sizeof(gamma));
    p->gamma = gamma;

    // rank and coefficients (eq. (2.6)); beta folds the primes of both sums
    p->K = choose_rank(p->eps, gamma);
    p->kmax = std::min(KMAX_ALL, ((p->K + 3) / 4) * 4);
    std::memset(p->beta, 0, sizeof(p->beta));
    std::memset(p->alpha, 0, sizeof(p->alpha));
    if (gamma == 0.0) {
        p->beta[0][0] = 1.0;   // u = v = 1: one FFT
        p->alpha[0][0] = 1.0;
    } else {
        std::vector<double> al(p->K * p->K);
        chebyshev_alpha(p->K, gamma, al.data());
        for (int r = 0; r < p->K; ++r)
            for (int q = 0; q < p->K; ++q) {
                const double w = (r == 0 ? 0.5 : 1.0) * (q == 0 ? 0.5 : 1.0);
                p->alpha[q][r] = al[q * p->K + r];
                p->beta[r][q] = w * al[q * p->K + r];
            }
    }

    int rc = plan_geometry<T>(p);
    if (rc) return rc;

    if ((rc = sort_samples<T>(p, s))) return rc;

    if ((rc = build_tables<T>(p, s))) return rc;

    // work buffers
    const size_t cxs = 2 * sizeof(T);
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->Y, (size_t)(p->K + 1) * p->L * cxs));   // rank K: the derivative
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->fscr, Mi * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->cstage, (size_t)p->N * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->fstage, Mi * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->err, sizeof(int)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), s));
    if (p->SBsplit > 1) {
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->part, (size_t)p->SBsplit * p->L * cxs));
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->counters, (size_t)(p->L1 / p->CB) * sizeof(int)));
        NUFFT_CUDA_TRY(cudaMemsetAsync(p->counters, 0, (size_t)(p->L1 / p->CB) * sizeof(int), s));
        p->work_bytes += (int64_t)((size_t)p->SBsplit * p->L * cxs + (p->L1 / p->CB) * sizeof(int));
    }
    p->work_bytes += (int64_t)(((size_t)(p->K + 1) * p->L + 2 * Mi + p->N) * cxs);
    if (p->flags & NUFFT_PLAN_UNFUSED) {
        if ((rc = plan_unfused_factors<T>(p, s))) return rc;
    }
    // FP64 plans read materialised factors in the fused kernels: on this GPU FP64
    // arithmetic is scarce and bandwidth is not
    if (p->prec == NUFFT_F64) {
        if ((rc = plan_factor_tables<dfloat>(p, s))) return rc;
    }
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

void free_plan(nufft_plan p) {
    if (!p) return;
    for (void *b : {p->twst1_dw, p->twst1a_dw, p->twst2_dw, p->twst2b_dw, p->twhi_dw, p->twlo_dw})
        if (b) cudaFree(b);
    void *bufs[] = {p->tsorted, p->perm, p->bstart, p->t_j, p->dsorted, p->d_j, p->twst1,
                    p->twst2, p->twst1a, p->twst2b, p->twhi, p->twlo, p->Y, p->fscr, p->cstage, p->fstage, p->U, p->V, p->Xg,
                    p->part, p->counters, p->err, p->Ufac, p->Vfac, p->t2_j, p->d2_j, p->dsorted2, p->vy,
                    p->inv_lam, p->inv_x, p->inv_z, p->inv_r, p->inv_p, p->inv_ap, p->inv_part, p->inv_scal};
    for (void *b : bufs) if (b) cudaFree(b);
    if (p->inv_host) cudaFreeHost(p->inv_host);
    for (void *b : {p->sb_Y, p->sb_fscr, p->sb_part, (void *)p->sb_cnt, p->sb_args, p->sb_beta})
        if (b) cudaFree(b);
    for (void *b : {p->st_g, p->st_fp, p->st_gc, p->st_gx})
        if (b) cudaFree(b);
    if (p->st_copy) cudaStreamDestroy(p->st_copy);
    for (cudaEvent_t e : p->st_ev)
        if (e) cudaEventDestroy(e);
    if (p->inv_fft) free_plan(p->inv_fft);
    for (cudaEvent_t e : p->ev) if (e) cudaEventDestroy(e);
    delete p;
}

}  // namespace
}  // namespace nufft

namespace nufft {
namespace {

// ---- the 2D transform (section 4) ---------------------------------------------------

__global__ void k_combine_t(int32_t *__restrict__ t, const int32_t *__restrict__ ty, int64_t M, int lgx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
        t[j] = (ty[j] << lgx) | t[j];   // t = Lx t^y + t^x: row t^x, position t^y
}

// Rounding in each direction (eqs. (2.8)-(2.9) on the m- and n-point grids, read of
// section 4), a rank per direction at eps / 2, the combined grid index, sort, tables.
template <typename T>
int plan_device_2d(nufft_plan p, const double *x, const double *y, cudaStream_t s) {
    const int64_t M = p->M;
    const size_t Mi = (size_t)std::max<int64_t>(M, 1);
    struct Scratch {
        unsigned long long *gbits = nullptr;
        int *bad = nullptr;
        ~Scratch() { cudaFree(gbits); cudaFree(bad); }
    } sc;
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.gbits, 2 * sizeof(unsigned long long)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&sc.bad, sizeof(int)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->t_j, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->d_j, Mi * sizeof(double)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->t2_j, Mi * sizeof(int32_t)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->d2_j, Mi * sizeof(double)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(sc.gbits, 0, 2 * sizeof(unsigned long long), s));
    NUFFT_CUDA_TRY(cudaMemsetAsync(sc.bad, 0, sizeof(int), s));
    const int64_t Lx = p->L2, Ly = p->L1;
    if (M > 0) {
        k_round<<<grid_for(M, 256), 256, 0, s>>>(x, M, (double)Lx, Lx, (double)p->N / (double)Lx, p->t_j,
                                                 p->d_j, sc.gbits, sc.bad);
        k_round<<<grid_for(M, 256), 256, 0, s>>>(y, M, (double)Ly, Ly, (double)p->N2 / (double)Ly, p->t2_j,
                                                 p->d2_j, sc.gbits + 1, sc.bad);
        k_combine_t<<<grid_for(M, 256), 256, 0, s>>>(p->t_j, p->t2_j, M, p->lg2);
        NUFFT_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long gb[2] = {0, 0};
    int bad = 0;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(gb, sc.gbits, sizeof(gb), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(&bad, sc.bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return NUFFT_EINVAL;
    std::memcpy(&p->gamma, &gb[0], sizeof(double));
    std::memcpy(&p->gamma2, &gb[1], sizeof(double));
    // ranks and coefficients per direction (eq. (2.6)); beta folds both primes
    auto coeffs = [](double eps, double gamma, int *K, double (*beta)[KMAX_ALL], double (*alpha)[KMAX_ALL]) {
        *K = choose_rank(eps, gamma);
        for (int r = 0; r < KMAX_ALL; ++r)
            for (int q = 0; q < KMAX_ALL; ++q) beta[r][q] = alpha[r][q] = 0.0;
        if (gamma == 0.0) {
            beta[0][0] = alpha[0][0] = 1.0;
            return;
        }
        std::vector<double> al((size_t)*K * *K);
        chebyshev_alpha(*K, gamma, al.data());
        for (int r = 0; r < *K; ++r)
            for (int q = 0; q < *K; ++q) {
                alpha[q][r] = al[q * *K + r];
                beta[r][q] = (r == 0 ? 0.5 : 1.0) * (q == 0 ? 0.5 : 1.0) * al[q * *K + r];
            }
    };
    coeffs(p->eps / 2.0, p->gamma, &p->K, p->beta, p->alpha);
    coeffs(p->eps / 2.0, p->gamma2, &p->K2, p->beta2, p->alpha2);
    const int km = std::max(p->K, p->K2);
    p->kmax = std::min(KMAX_ALL, ((km + 3) / 4) * 4);

    // geometry: pass 1 from the 1D rules; the row pass holds two row buffers, G2d slots
    // (all K2 y-ranks when they fit, else groups of G2d) and two mbarriers, with teams
    // for G2d row FFTs per group
    if (int rc = plan_geometry<T>(p)) return rc;
    p->B2 = 1;
    p->NB = p->L2;
    {
        const int E1 = std::min(EmaxT<T, PK_ROW_FWD>::v, p->L1), TT1 = p->L1 / E1;
        auto bytes = [&](int G) {
            return ((size_t)2 * p->L1 + (size_t)G * p->S2) * 2 * sizeof(T) + 2 * sizeof(uint64_t);
        };
        int G = p->K2;
        while (G > 1 && bytes(G) > SMEM_BUDGET) --G;
        if (bytes(G) > SMEM_BUDGET) return NUFFT_EUNSUPPORTED;
        p->G2d = G;
        const int maxt = std::max(1, 256 / TT1);
        const int rounds = (G + maxt - 1) / maxt;
        int nt = (G + rounds - 1) / rounds;
        if (nt * TT1 < 64) nt = std::min(maxt, std::max(nt, (64 + TT1 - 1) / TT1));
        p->nt2 = std::max(1, nt);
        p->smem2 = bytes(G);
    }
    {
        // the adjoint row pass: an accumulator row and G2a slots (all K2 y-ranks when
        // they fit, else groups), with teams for G2a inverse row FFTs per group
        const int E1a = std::min(EmaxT<T, PK_ROW_ADJ>::v, p->L1), TT1a = p->L1 / E1a;
        auto bytes = [&](int G) { return ((size_t)p->L1 + (size_t)G * p->SA) * 2 * sizeof(T); };
        int G = p->K2;
        while (G > 1 && bytes(G) > SMEM_BUDGET) --G;
        if (bytes(G) > SMEM_BUDGET) return NUFFT_EUNSUPPORTED;
        p->G2a = G;
        const int maxt = std::max(1, 256 / TT1a);
        const int rounds = (G + maxt - 1) / maxt;
        int nt = (G + rounds - 1) / rounds;
        if (nt * TT1a < 64) nt = std::min(maxt, std::max(nt, (64 + TT1a - 1) / TT1a));
        p->nt2a = std::max(1, nt);
        p->smemA2d = bytes(G);
    }

    int rc = sort_samples<T>(p, s);
    if (rc) return rc;
    if ((rc = build_tables<T>(p, s))) return rc;
    // the y-scale T_r2(2 k2 / n - 1) for k2 < n, 0 beyond (the 1/2 of r2 = 0 is in beta)
    {
        std::vector<T> h((size_t)p->K2 * p->L1, T(0));
        for (int r = 0; r < p->K2; ++r)
            for (int64_t k = 0; k < p->N2; ++k) {
                const double z = (2.0 * (double)k - (double)p->N2) / (double)p->N2;
                double a0 = 1.0, a1 = z, tr = r == 0 ? 1.0 : z;
                for (int q = 2; q <= r; ++q) {
                    tr = 2.0 * z * a1 - a0;
                    a0 = a1;
                    a1 = tr;
                }
                h[(size_t)r * p->L1 + k] = (T)tr;
            }
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->vy, h.size() * sizeof(T)));
        NUFFT_CUDA_TRY(cudaMemcpyAsync(p->vy, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const size_t cxs = 2 * sizeof(T);
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->Y, (size_t)p->K * p->L * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->fscr, Mi * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->err, sizeof(int)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), s));
    p->work_bytes += (int64_t)(((size_t)p->K * p->L + Mi) * cxs + Mi * (2 * sizeof(int32_t) + 2 * sizeof(double)));
    if (p->SBsplit > 1) {   // the adjoint's column pass splits the x-ranks over CTAs
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->part, (size_t)p->SBsplit * p->L * cxs));
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->counters, (size_t)(p->L1 / p->CB) * sizeof(int)));
        NUFFT_CUDA_TRY(cudaMemsetAsync(p->counters, 0, (size_t)(p->L1 / p->CB) * sizeof(int), s));
        p->work_bytes += (int64_t)((size_t)p->SBsplit * p->L * cxs + (p->L1 / p->CB) * sizeof(int));
    }
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

}  // namespace
}  // namespace nufft

extern "C" int nufft2d_plan(nufft_plan *out, int64_t m, int64_t n, int64_t M, const double *x_dev,
                            const double *y_dev, double eps, int prec, unsigned flags, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2d_plan");
    using namespace nufft;
    if (!out) return NUFFT_EINVAL;
    *out = nullptr;
    if (m < 1 || n < 1 || M < 0 || M >= ((int64_t)1 << 31) || !(eps > 0.0 && eps < 1.0)) return NUFFT_EINVAL;
    if (prec != NUFFT_F32 && prec != NUFFT_F64) return NUFFT_EINVAL;
    if (M > 0 && (!x_dev || !y_dev)) return NUFFT_EINVAL;
    if (flags & ~NUFFT_PLAN_TIMING) return NUFFT_EINVAL;
    if (m > 2048 || n > 2048) return NUFFT_EUNSUPPORTED;
    int64_t Lx = 32, Ly = 32;
    while (Lx < m) Lx <<= 1;
    while (Ly < n) Ly <<= 1;
    nufft_plan p = new (std::nothrow) nufft_plan_s();
    if (!p) return NUFFT_ENOMEM;
    p->dims = 2;
    p->N = m; p->N2 = n; p->M = M; p->L = Lx * Ly; p->eps = eps; p->prec = prec; p->flags = flags;
    p->L1 = (int)Ly; p->L2 = (int)Lx;
    while ((1 << p->lg1) < p->L1) ++p->lg1;
    while ((1 << p->lg2) < p->L2) ++p->lg2;
    if (cudaGetDevice(&p->device) != cudaSuccess) { free_plan(p); return NUFFT_ECUDA; }
    if (flags & NUFFT_PLAN_TIMING)
        for (cudaEvent_t &e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); free_plan(p); return NUFFT_ECUDA; }
    const int rc = prec == NUFFT_F32 ? plan_device_2d<float>(p, x_dev, y_dev, (cudaStream_t)stream)
                                     : plan_device_2d<double>(p, x_dev, y_dev, (cudaStream_t)stream);
    if (rc != NUFFT_OK) { free_plan(p); return rc; }
    *out = p;
    return NUFFT_OK;
}

extern "C" int nufft2d_plan_info(nufft_plan p, int *Kx, int *Ky, double *gamma_x, double *gamma_y, int64_t *Lx,
                                 int64_t *Ly) {
    if (!p || p->dims != 2) return NUFFT_EINVAL;
    if (Kx) *Kx = p->K;
    if (Ky) *Ky = p->K2;
    if (gamma_x) *gamma_x = p->gamma;
    if (gamma_y) *gamma_y = p->gamma2;
    if (Lx) *Lx = p->L2;
    if (Ly) *Ly = p->L1;
    return NUFFT_OK;
}

namespace nufft {
namespace {

// One plan with layout lay (lay.L a power of two, validated by the caller): lay.long_cols
// for odd log2 L puts the longer FFT on the columns (L2 = 2 L1); lay.c1_shift halves
// pass 1's columns per CTA.
int plan_create(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps, int prec,
                const Layout &lay, unsigned flags, cudaStream_t s) {
    *out = nullptr;
    nufft_plan p = new (std::nothrow) nufft_plan_s();
    if (!p) return NUFFT_ENOMEM;
    const int64_t L = lay.L;
    p->N = N; p->M = M; p->L = L; p->eps = eps; p->prec = prec; p->flags = flags;
    p->c1_shift = lay.c1_shift;
    int lg = 0;
    while (((int64_t)1 << lg) < L) ++lg;
    p->lg1 = lay.long_cols ? lg / 2 : (lg + 1) / 2;
    p->lg2 = lg - p->lg1;
    p->L1 = 1 << p->lg1;
    p->L2 = 1 << p->lg2;
    if (cudaGetDevice(&p->device) != cudaSuccess) { free_plan(p); return NUFFT_ECUDA; }
    if (flags & NUFFT_PLAN_TIMING)
        for (cudaEvent_t &e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); free_plan(p); return NUFFT_ECUDA; }
    const int rc = prec == NUFFT_F32 ? plan_device<float>(p, x_dev, s) : plan_device<double>(p, x_dev, s);
    if (rc != NUFFT_OK) { free_plan(p); return rc; }
    *out = p;
    return NUFFT_OK;
}

// Device time (ms) of one forward and one adjoint exec of plan p on its own staging
// buffers (filled with hash values), L2 flushed before each run: the best of three
// after one warm-up.
int time_exec(nufft_plan p, void *flush, cudaStream_t s, float *ms) {
    const bool f32 = p->prec == NUFFT_F32;
    NUFFT_CUDA_TRY(f32 ? fill_hash<float>(p->cstage, 2 * p->N, s) : fill_hash<double>(p->cstage, 2 * p->N, s));
    NUFFT_CUDA_TRY(f32 ? fill_hash<float>(p->fstage, 2 * p->M, s) : fill_hash<double>(p->fstage, 2 * p->M, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return NUFFT_ECUDA;
    }
    int rc = NUFFT_OK;
    float best = 1e30f;
    for (int it = 0; it < 4 && !rc; ++it) {
        if (cudaMemsetAsync(flush, it, L2_FLUSH_BYTES, s) != cudaSuccess ||
            cudaEventRecord(e0, s) != cudaSuccess) { rc = NUFFT_ECUDA; break; }
        rc = nufft2_exec(p, p->cstage, p->fstage, s);
        if (!rc) rc = nufft1_exec(p, p->fstage, p->cstage, s);
        if (rc) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = NUFFT_ECUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (it > 0) best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = nufft2_check(p, s);
    *ms = best;
    return rc;
}

// The tuner's choices, per process: (device, N, M rounded up to a power of two, eps,
// precision, K on the default grid) -> layout.
struct TuneKey {
    int device;
    int64_t N, Mb;
    double eps;
    int prec, K;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, N, Mb, eps, prec, K) < std::tie(o.device, o.N, o.Mb, o.eps, o.prec, o.K);
    }
};
std::mutex tune_mu;
std::map<TuneKey, Layout> tune_cache;

// Autotuned planning: the candidates are the default grid L0 and the oversampled
// 2 L0 (section 2.3: a longer grid lowers gamma, and so K), each with either four-step
// split when log2 L is odd (the radices of the two passes) and with pass 1's default or
// half number of columns per CTA (the tile); the one with the fastest forward + adjoint
// is kept.
int plan_autotune(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps, int prec,
                  int64_t L0, unsigned flags, cudaStream_t s) {
    nufft_plan best = nullptr;
    Layout choice;
    choice.L = L0;
    if (int rc = plan_create(&best, N, M, x_dev, eps, prec, choice, flags, s)) return rc;
    int64_t Mb = 1;
    while (Mb < M) Mb <<= 1;
    const TuneKey key{best->device, N, Mb, eps, prec, best->K};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        auto it = tune_cache.find(key);
        if (it != tune_cache.end()) { choice = it->second; cached = true; }
    }
    if (cached) {
        if (choice.L == L0 && !choice.long_cols && choice.c1_shift == 0) { *out = best; return NUFFT_OK; }
        free_plan(best);
        return plan_create(out, N, M, x_dev, eps, prec, choice, flags, s);
    }
    struct Flush {
        void *p = nullptr;
        ~Flush() { cudaFree(p); }
    } flush;
    if (dev_malloc((void **)&flush.p, L2_FLUSH_BYTES) != cudaSuccess) {
        (void)cudaGetLastError();
        free_plan(best);
        return NUFFT_ENOMEM;
    }
    float tbest = 0.f;
    if (int rc = time_exec(best, flush.p, s, &tbest)) { free_plan(best); return rc; }
    for (int64_t L = L0; L <= std::min<int64_t>(2 * L0, (int64_t)1 << LOG2_L_MAX); L *= 2) {
        int lg = 0;
        while (((int64_t)1 << lg) < L) ++lg;
        for (int lc = 0; lc < 2; ++lc)
            for (int c1s = 0; c1s < 2; ++c1s) {
                if ((L == L0 && lc == 0 && c1s == 0) || (lc == 1 && lg % 2 == 0)) continue;
                Layout cl;
                cl.L = L;
                cl.long_cols = lc == 1;
                cl.c1_shift = c1s;
                nufft_plan cand = nullptr;
                int rc = plan_create(&cand, N, M, x_dev, eps, prec, cl, flags, s);
                if (rc == NUFFT_EUNSUPPORTED) continue;   // e.g. the shared-memory budget
                if (rc) { free_plan(best); return rc; }
                float t = 0.f;
                if ((rc = time_exec(cand, flush.p, s, &t))) { free_plan(cand); free_plan(best); return rc; }
                if (t < tbest) {
                    free_plan(best);
                    best = cand;
                    tbest = t;
                    choice = cl;
                } else {
                    free_plan(cand);
                }
            }
    }
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        tune_cache[key] = choice;
    }
    *out = best;
    return NUFFT_OK;
}

// The tuner's table as text: a header line, then one entry per line,
//   device N Mb eps prec K -> L long_cols c1_shift
// with eps printed to 17 significant digits, so that it reads back to the same double.
constexpr const char *TUNE_HEADER = "nufft-tune-table 1";

bool tune_entry_ok(const TuneKey &k, const Layout &l) {
    const bool pow2_L = l.L > 0 && (l.L & (l.L - 1)) == 0;
    const bool pow2_M = k.Mb > 0 && (k.Mb & (k.Mb - 1)) == 0;
    return k.device >= 0 && k.N >= 1 && pow2_M && k.eps > 0.0 && k.eps < 1.0 && (k.prec == 0 || k.prec == 1) &&
           k.K >= 1 && k.K <= KMAX_ALL && pow2_L && l.L >= k.N && l.L >= ((int64_t)1 << LOG2_L_MIN) &&
           l.L <= ((int64_t)1 << LOG2_L_MAX) && (l.c1_shift == 0 || l.c1_shift == 1);
}

}  // namespace
}  // namespace nufft

extern "C" int nufft_tune_save(const char *path, int64_t *entries) {
    using namespace nufft;
    if (!path) return NUFFT_EINVAL;
    std::map<TuneKey, Layout> snap;
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        snap = tune_cache;
    }
    FILE *f = std::fopen(path, "w");
    if (!f) return NUFFT_EINVAL;
    bool ok = std::fprintf(f, "%s\n", TUNE_HEADER) > 0;
    for (const auto &e : snap) {
        const TuneKey &k = e.first;
        const Layout &l = e.second;
        ok = ok && std::fprintf(f, "%d %lld %lld %.17g %d %d -> %lld %d %d\n", k.device, (long long)k.N,
                                (long long)k.Mb, k.eps, k.prec, k.K, (long long)l.L, l.long_cols ? 1 : 0,
                                l.c1_shift) > 0;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return NUFFT_EINVAL;
    if (entries) *entries = (int64_t)snap.size();
    return NUFFT_OK;
}

extern "C" int nufft_tune_load(const char *path, int64_t *entries) {
    using namespace nufft;
    if (!path) return NUFFT_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return NUFFT_EINVAL;
    char line[512];
    bool ok = std::fgets(line, sizeof line, f) != nullptr && std::strncmp(line, TUNE_HEADER, std::strlen(TUNE_HEADER)) == 0;
    std::vector<std::pair<TuneKey, Layout>> got;
    while (ok && std::fgets(line, sizeof line, f)) {
        if (line[0] == '\n' || line[0] == '\0') continue;
        TuneKey k{};
        Layout l;
        long long N = 0, Mb = 0, L = 0;
        int lc = 0;
        char arrow[4] = {0};
        const int n = std::sscanf(line, "%d %lld %lld %lf %d %d %3s %lld %d %d", &k.device, &N, &Mb, &k.eps, &k.prec,
                                  &k.K, arrow, &L, &lc, &l.c1_shift);
        k.N = N;
        k.Mb = Mb;
        l.L = L;
        l.long_cols = lc == 1;
        ok = n == 10 && std::strcmp(arrow, "->") == 0 && (lc == 0 || lc == 1) && tune_entry_ok(k, l);
        if (ok) got.emplace_back(k, l);
    }
    std::fclose(f);
    if (!ok) return NUFFT_EINVAL;   // nothing merged from a malformed table
    std::lock_guard<std::mutex> lk(tune_mu);
    for (const auto &e : got) tune_cache[e.first] = e.second;
    if (entries) *entries = (int64_t)got.size();
    return NUFFT_OK;
}

extern "C" int nufft_tune_clear(int64_t *entries) {
    using namespace nufft;
    std::lock_guard<std::mutex> lk(tune_mu);
    if (entries) *entries = (int64_t)tune_cache.size();
    tune_cache.clear();
    return NUFFT_OK;
}

extern "C" int nufft2_plan(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps,
                           int prec, int64_t L, unsigned flags, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_plan");
    using namespace nufft;
    if (!out) return NUFFT_EINVAL;
    *out = nullptr;
    if (N < 1 || M < 0 || M >= ((int64_t)1 << 31) || !(eps > 0.0 && eps < 1.0)) return NUFFT_EINVAL;
    if (prec != NUFFT_F32 && prec != NUFFT_F64) return NUFFT_EINVAL;
    if (M > 0 && !x_dev) return NUFFT_EINVAL;
    if (flags & ~(NUFFT_PLAN_UNFUSED | NUFFT_PLAN_TIMING | NUFFT_PLAN_AUTOTUNE | NUFFT_PLAN_LONG_COLUMNS |
                  NUFFT_PLAN_HALF_TILE))
        return NUFFT_EINVAL;
    if (N > ((int64_t)1 << LOG2_L_MAX)) return NUFFT_EUNSUPPORTED;
    const bool fixed_L = L != 0;
    if (!fixed_L) {
        L = (int64_t)1 << LOG2_L_MIN;
        while (L < N) L <<= 1;
    } else {
        if (L < N || (L & (L - 1)) != 0) return NUFFT_EINVAL;
        if (L < ((int64_t)1 << LOG2_L_MIN) || L > ((int64_t)1 << LOG2_L_MAX)) return NUFFT_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned pf = flags & (NUFFT_PLAN_UNFUSED | NUFFT_PLAN_TIMING);
    if ((flags & NUFFT_PLAN_AUTOTUNE) && !fixed_L && !(flags & (NUFFT_PLAN_LONG_COLUMNS | NUFFT_PLAN_HALF_TILE)))
        return plan_autotune(out, N, M, x_dev, eps, prec, L, pf, s);
    Layout lay;
    lay.L = L;
    lay.long_cols = (flags & NUFFT_PLAN_LONG_COLUMNS) != 0;
    lay.c1_shift = (flags & NUFFT_PLAN_HALF_TILE) ? 1 : 0;
    return plan_create(out, N, M, x_dev, eps, prec, lay, pf, s);
}

namespace nufft {
// A plan with a given layout, for the batch tuner (the same checks as nufft2_plan).
int plan_layout(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps, int prec,
                const Layout &lay, unsigned flags, cudaStream_t s) {
    if (!out) return NUFFT_EINVAL;
    *out = nullptr;
    if (lay.L == 0 && !lay.long_cols && lay.c1_shift == 0)
        return nufft2_plan(out, N, M, x_dev, eps, prec, 0, flags, s);
    if (N < 1 || M < 0 || M >= ((int64_t)1 << 31) || !(eps > 0.0 && eps < 1.0)) return NUFFT_EINVAL;
    if (prec != NUFFT_F32 && prec != NUFFT_F64) return NUFFT_EINVAL;
    if (M > 0 && !x_dev) return NUFFT_EINVAL;
    Layout l = lay;
    if (l.L == 0) {
        l.L = (int64_t)1 << LOG2_L_MIN;
        while (l.L < N) l.L <<= 1;
    }
    if (l.L < N || (l.L & (l.L - 1)) != 0) return NUFFT_EINVAL;
    if (l.L < ((int64_t)1 << LOG2_L_MIN) || l.L > ((int64_t)1 << LOG2_L_MAX)) return NUFFT_EUNSUPPORTED;
    if (l.c1_shift < 0 || l.c1_shift > 4) return NUFFT_EINVAL;
    return plan_create(out, N, M, x_dev, eps, prec, l, flags & (NUFFT_PLAN_UNFUSED | NUFFT_PLAN_TIMING), s);
}
}  // namespace nufft

extern "C" int nufft2_plan_info(nufft_plan p, int *K, double *gamma, int64_t *L, int64_t *work_bytes) {
    if (!p) return NUFFT_EINVAL;
    if (K) *K = p->K;
    if (gamma) *gamma = p->gamma;
    if (L) *L = p->L;
    if (work_bytes) *work_bytes = p->work_bytes;
    return NUFFT_OK;
}

extern "C" int nufft2_plan_export(nufft_plan p, int32_t *t_dev, double *d_dev, double *alpha_host,
                                  void *stream) {
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;
    if (!p) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->M > 0 && t_dev)
        NUFFT_CUDA_TRY(cudaMemcpyAsync(t_dev, p->t_j, (size_t)p->M * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (p->M > 0 && d_dev)
        NUFFT_CUDA_TRY(cudaMemcpyAsync(d_dev, p->d_j, (size_t)p->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (alpha_host)
        for (int q = 0; q < p->K; ++q)
            for (int r = 0; r < p->K; ++r) alpha_host[q * p->K + r] = p->alpha[q][r];
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

extern "C" int nufft_kernel_times(nufft_plan p, float *ms_out, int cap, int *count) {
    if (!p || (cap > 0 && !ms_out)) return NUFFT_EINVAL;
    if (!(p->flags & NUFFT_PLAN_TIMING)) return NUFFT_ESTATE;
    const int n = p->nev > 0 ? p->nev - 1 : 0;
    if (count) *count = n;
    if (n == 0) return NUFFT_OK;
    NUFFT_CUDA_TRY(cudaEventSynchronize(p->ev[p->nev - 1]));
    for (int i = 0; i < n && i < cap; ++i) NUFFT_CUDA_TRY(cudaEventElapsedTime(&ms_out[i], p->ev[i], p->ev[i + 1]));
    return NUFFT_OK;
}

extern "C" int nufft2_check(nufft_plan p, void *stream) {
    if (!p) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        NUFFT_CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), s));
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
        return (h & nufft::ERR_TIMEOUT) ? NUFFT_ETIMEOUT : NUFFT_ECHECK;
    }
    return NUFFT_OK;
}

extern "C" int nufft_destroy(nufft_plan p) {
    nufft::free_plan(p);
    return NUFFT_OK;
}

extern "C" const char *nufft_strerror(int code) {
    switch (code) {
        case NUFFT_OK: return "ok";
        case NUFFT_EINVAL: return "invalid argument";
        case NUFFT_ENOMEM: return "out of memory";
        case NUFFT_ECUDA: return "CUDA error";
        case NUFFT_EUNSUPPORTED: return "unsupported size";
        case NUFFT_ESTATE: return "plan lacks the option this call needs";
        case NUFFT_ETIMEOUT: return "a device-side wait timed out; results of the affected calls are invalid";
        case NUFFT_ECHECK: return "an index check failed (NUFFT_CHECK build); results of the affected calls are invalid";
        default: return "unknown status";
    }
}
