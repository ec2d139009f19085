// shared_batch.cu -- B coefficient vectors on one plan (the same samples) in one
// launch per pass.
//
// Each member b gets its own slice of a per-plan workspace (the rank intermediate, the
// partial sums of the row passes, pass B's partials and tickets) and reads the plan's
// sorted samples, tables and coefficients; the batched kernels (blockIdx.z = the
// member) read the members' arguments from a device array built on each call.  The
// batched kernels exist for FP32 plans whose FFT lengths are at most 512 (grids up to
// 2^18 points); other plans run the members one after another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "passes.cuh"
#include "nvtx_range.h"

namespace nufft {
NUFFT_DECLARE_COLS_MANY()
NUFFT_DECLARE_MANY(4)
NUFFT_DECLARE_MANY(8)
NUFFT_DECLARE_MANY(12)
NUFFT_DECLARE_MANY(16)

namespace {

// Coefficients per member: N, or m n for a 2D plan.
int64_t ncoef(nufft_plan p) { return p->dims == 2 ? p->N * p->N2 : p->N; }

bool batchable(nufft_plan p) {
    return p->prec == NUFFT_F32 && p->dims == 1 && p->M > 0 && std::max(p->L1, p->L2) <= MANY_P_MAX;
}

// The per-member argument arrays, each `cap` entries, in the order of ArgSet.
enum ArgSet { AS_FWD1 = 0, AS_FWD2, AS_DER1, AS_DER2, AS_ADJA, AS_ADJB, AS_COUNT };

// A member's arguments: its workspace slice.  Its data pointers come from the launch
// (ManyIO: the call's base pointers and leading dimensions), so the arguments do not
// depend on the call and are built once, by nufft2_plan_reserve.
PassArgs<float> member(nufft_plan p, int64_t b) {
    PassArgs<float> a = base_args<float>(p);
    a.Y = (cx<float> *)p->sb_Y + b * (int64_t)(p->K + 1) * p->L;
    a.fscr = (cx<float> *)p->sb_fscr + b * p->M;
    a.part = (cx<float> *)p->sb_part + b * (int64_t)std::max(1, p->SBsplit) * p->L;
    a.counters = p->sb_cnt + b * (int64_t)(p->L1 / p->CB);
    a.in_off = 0;
    a.out_off = 0;
    return a;
}

// The workspace and the member arguments for up to B members: the plan stage of the
// batch calls (allocates, uploads, synchronises), so that the exec calls do neither.
int reserve_batch(nufft_plan p, int64_t B, cudaStream_t s) {
    if (B <= p->sb_cap) return NUFFT_OK;
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));   // the old workspace may be in use
    for (void *q : {p->sb_Y, p->sb_fscr, p->sb_part, (void *)p->sb_cnt, p->sb_args, p->sb_beta})
        if (q) cudaFree(q);
    p->sb_Y = p->sb_fscr = p->sb_part = p->sb_args = p->sb_beta = nullptr;
    p->sb_cnt = nullptr;
    p->sb_cap = 0;
    const size_t cxs = 8, nb = (size_t)B;
    const size_t ncnt = (size_t)(p->L1 / p->CB);
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_Y, nb * (size_t)(p->K + 1) * p->L * cxs));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_fscr, nb * (size_t)p->M * cxs));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_part, nb * (size_t)std::max(1, p->SBsplit) * p->L * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->sb_cnt, nb * ncnt * sizeof(int)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(p->sb_cnt, 0, nb * ncnt * sizeof(int), s));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_args, AS_COUNT * nb * sizeof(PassArgs<float>)));
    const int km = p->kmax;
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_beta, nb * (size_t)km * km * sizeof(float)));
    // beta for every member (the batched kernels index it by member), laid out as
    // Beta<float, kmax>: kmax x kmax row-major
    std::vector<float> be(nb * (size_t)km * km);
    for (size_t b = 0; b < nb; ++b)
        for (int r = 0; r < km; ++r)
            for (int q = 0; q < km; ++q) be[(b * km + r) * km + q] = (float)p->beta[r][q];
    std::vector<PassArgs<float>> v(AS_COUNT * nb);
    for (size_t b = 0; b < nb; ++b) {
        const PassArgs<float> a = member(p, (int64_t)b);
        PassArgs<float> d = a;   // the forward with f': K + 1 ranks
        d.mode |= MODE_DERIV;
        d.nranks = p->K + 1;
        PassArgs<float> f1 = a, f2 = a, d1 = d, d2 = d, aA = a, aB = a;
        cols_fields<float>(p, f1, false);
        cols_fields<float>(p, d1, false);
        cols_fields<float>(p, aB, true);
        if (int rc = rows_fields<float>(p, f2, false)) return rc;
        if (int rc = rows_fields<float>(p, d2, false)) return rc;
        if (int rc = rows_fields<float>(p, aA, true)) return rc;
        v[AS_FWD1 * nb + b] = f1;
        v[AS_FWD2 * nb + b] = f2;
        v[AS_DER1 * nb + b] = d1;
        v[AS_DER2 * nb + b] = d2;
        v[AS_ADJA * nb + b] = aA;
        v[AS_ADJB * nb + b] = aB;
    }
    NUFFT_CUDA_TRY(cudaMemcpy(p->sb_beta, be.data(), be.size() * sizeof(float), cudaMemcpyHostToDevice));
    NUFFT_CUDA_TRY(cudaMemcpy(p->sb_args, v.data(), v.size() * sizeof(PassArgs<float>), cudaMemcpyHostToDevice));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    p->sb_cap = B;
    p->work_bytes += (int64_t)(nb * ((size_t)(p->K + 1) * p->L + p->M + (size_t)std::max(1, p->SBsplit) * p->L) * cxs);
    return NUFFT_OK;
}

const PassArgs<float> *argset(nufft_plan p, ArgSet k) {
    return (const PassArgs<float> *)p->sb_args + (int64_t)k * p->sb_cap;
}

int rows_many_km(nufft_plan p, const PassArgs<float> *args, int64_t B, bool adjoint, const ManyIO &io,
                 cudaStream_t s) {
    const void *be = p->sb_beta;
    const int n = (int)B;
    switch (p->kmax) {
        case 4: return launch_rows_many<float, 4>(p, args, (const Beta<float, 4> *)be, n, adjoint, io, s);
        case 8: return launch_rows_many<float, 8>(p, args, (const Beta<float, 8> *)be, n, adjoint, io, s);
        case 12: return launch_rows_many<float, 12>(p, args, (const Beta<float, 12> *)be, n, adjoint, io, s);
        case 16: return launch_rows_many<float, 16>(p, args, (const Beta<float, 16> *)be, n, adjoint, io, s);
        default: return NUFFT_EUNSUPPORTED;
    }
}

// Forward (deriv = false) or forward with f' (deriv = true) of B <= sb_cap members: two
// launches, no allocation, no host synchronisation.
int fwd_batch(nufft_plan p, int64_t B, const void *c, int64_t ldc, void *f, void *fp, int64_t ldf, bool deriv,
              cudaStream_t s) {
    if (B > p->sb_cap) return NUFFT_ESTATE;
    const ManyIO io{c, f, deriv ? fp : nullptr, ldc, ldf};
    const PassArgs<float> *a1 = argset(p, deriv ? AS_DER1 : AS_FWD1), *a2 = argset(p, deriv ? AS_DER2 : AS_FWD2);
    if (int rc = launch_cols_many<float>(p, a1, (int)B, deriv ? p->K + 1 : p->K, false, io, s)) return rc;
    return rows_many_km(p, a2, B, false, io, s);
}

// Adjoint of B <= sb_cap members: c_b = A^H g_b.
int adj_batch(nufft_plan p, int64_t B, const void *g, int64_t ldg, void *c, int64_t ldc, cudaStream_t s) {
    if (B > p->sb_cap) return NUFFT_ESTATE;
    const ManyIO io{g, c, nullptr, ldg, ldc};
    if (int rc = rows_many_km(p, argset(p, AS_ADJA), B, true, io, s)) return rc;
    return launch_cols_many<float>(p, argset(p, AS_ADJB), (int)B, std::max(1, p->SBsplit), true, io, s);
}

// gx_j (+)= sum_b Re(conj(g_bj) f'_bj)
template <typename T>
__global__ void k_grad_x_batch(const cx<T> *__restrict__ g, const cx<T> *__restrict__ fp, int64_t B, int64_t ld,
                               int64_t M, int acc, T *__restrict__ gx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        T s = acc ? gx[j] : T(0);
        for (int64_t b = 0; b < B; ++b) {
            const cx<T> a = g[b * ld + j], q = fp[b * ld + j];
            s += fma(a.x, q.x, a.y * q.y);
        }
        gx[j] = s;
    }
}

int grid_m(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

}  // namespace
}  // namespace nufft

using nufft::adj_batch;
using nufft::batchable;
using nufft::ncoef;

extern "C" int nufft2_plan_reserve(nufft_plan p, int64_t B_max, unsigned what, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_plan_reserve");
    if (!p || B_max < 0 || (what & ~NUFFT_RESERVE_STEP_HOST)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (B_max >= 2 && batchable(p))
        if (int rc = nufft::reserve_batch(p, B_max, s)) return rc;
    if (what & NUFFT_RESERVE_STEP_HOST) {
        if (p->dims == 2) return NUFFT_EUNSUPPORTED;
        if (int rc = nufft::reserve_step_host(p, s)) return rc;
    }
    return NUFFT_OK;
}

extern "C" int nufft2_plan_reserved(nufft_plan p, int64_t *B_max, int *step_host) {
    if (!p) return NUFFT_EINVAL;
    if (B_max) *B_max = batchable(p) ? p->sb_cap : INT64_MAX;
    if (step_host) *step_host = p->st_g && p->st_copy ? 1 : 0;
    return NUFFT_OK;
}
using nufft::fwd_batch;

extern "C" int nufft2_exec_batch(nufft_plan p, int64_t B, const void *c_dev, int64_t ldc, void *f_dev, int64_t ldf,
                                 void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_batch");
    if (!p || B < 0 || ldc < ncoef(p) || ldf < p->M) return NUFFT_EINVAL;
    if (B > 0 && (!c_dev || (p->M > 0 && !f_dev))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (B >= 2 && batchable(p)) return fwd_batch(p, B, c_dev, ldc, f_dev, nullptr, ldf, false, s);
    const size_t cxs = p->prec == NUFFT_F32 ? 8 : 16;
    for (int64_t b = 0; b < B; ++b) {
        const void *cb = (const char *)c_dev + (size_t)(b * ldc) * cxs;
        void *fb = (char *)f_dev + (size_t)(b * ldf) * cxs;
        if (int rc = nufft2_exec(p, cb, fb, stream)) return rc;
    }
    return NUFFT_OK;
}

extern "C" int nufft1_exec_batch(nufft_plan p, int64_t B, const void *g_dev, int64_t ldg, void *c_dev, int64_t ldc,
                                 void *stream) {
    nufft::NvtxRange nvtx_range_("nufft1_exec_batch");
    if (!p || B < 0 || ldc < ncoef(p) || ldg < p->M) return NUFFT_EINVAL;
    if (B > 0 && (!c_dev || (p->M > 0 && !g_dev))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (B >= 2 && batchable(p)) return adj_batch(p, B, g_dev, ldg, c_dev, ldc, s);
    const size_t cxs = p->prec == NUFFT_F32 ? 8 : 16;
    for (int64_t b = 0; b < B; ++b) {
        const void *gb = (const char *)g_dev + (size_t)(b * ldg) * cxs;
        void *cb = (char *)c_dev + (size_t)(b * ldc) * cxs;
        if (int rc = nufft1_exec(p, gb, cb, stream)) return rc;
    }
    return NUFFT_OK;
}

extern "C" int nufft2_exec_deriv_batch(nufft_plan p, int64_t B, const void *c_dev, int64_t ldc, void *f_dev,
                                       void *fprime_dev, int64_t ldf, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_deriv_batch");
    if (!p || B < 0 || ldc < p->N || ldf < p->M) return NUFFT_EINVAL;
    if (B > 0 && (!c_dev || (p->M > 0 && (!f_dev || !fprime_dev)))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (B >= 2 && batchable(p) && p->G >= p->K + 1)
        return fwd_batch(p, B, c_dev, ldc, f_dev, fprime_dev, ldf, true, s);
    const size_t cxs = p->prec == NUFFT_F32 ? 8 : 16;
    for (int64_t b = 0; b < B; ++b) {
        const void *cb = (const char *)c_dev + (size_t)(b * ldc) * cxs;
        void *fb = (char *)f_dev + (size_t)(b * ldf) * cxs;
        void *pb = (char *)fprime_dev + (size_t)(b * ldf) * cxs;
        if (int rc = nufft2_exec_deriv(p, cb, fb, pb, stream)) return rc;
    }
    return NUFFT_OK;
}

extern "C" int nufft2_grad_x_batch(nufft_plan p, int64_t B, const void *g_dev, const void *fprime_dev, int64_t ld,
                                   void *gx_dev, int accumulate, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_grad_x_batch");
    if (!p || B < 0 || ld < p->M) return NUFFT_EINVAL;
    if (p->dims == 2) return NUFFT_EUNSUPPORTED;
    if (p->M > 0 && (!g_dev || !fprime_dev || !gx_dev)) return NUFFT_EINVAL;
    if (p->M == 0) return NUFFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->prec == NUFFT_F32)
        nufft::k_grad_x_batch<float><<<nufft::grid_m(p->M), 256, 0, s>>>(
            (const nufft::cx<float> *)g_dev, (const nufft::cx<float> *)fprime_dev, B, ld, p->M, accumulate,
            (float *)gx_dev);
    else
        nufft::k_grad_x_batch<double><<<nufft::grid_m(p->M), 256, 0, s>>>(
            (const nufft::cx<double> *)g_dev, (const nufft::cx<double> *)fprime_dev, B, ld, p->M, accumulate,
            (double *)gx_dev);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}
