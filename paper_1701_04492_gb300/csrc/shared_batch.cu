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

bool batchable(nufft_plan p) {
    return p->prec == NUFFT_F32 && p->dims == 1 && p->M > 0 && std::max(p->L1, p->L2) <= MANY_P_MAX;
}

// The workspace for B members (kept, grown when a larger B comes).
int ensure_workspace(nufft_plan p, int64_t B, cudaStream_t s) {
    if (B <= p->sb_cap) return NUFFT_OK;
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));   // the old workspace may be in use
    for (void *q : {p->sb_Y, p->sb_fscr, p->sb_part, (void *)p->sb_cnt, p->sb_args, p->sb_beta})
        if (q) cudaFree(q);
    if (p->sb_host) cudaFreeHost(p->sb_host);
    p->sb_Y = p->sb_fscr = p->sb_part = p->sb_args = p->sb_beta = p->sb_host = nullptr;
    p->sb_cnt = nullptr;
    p->sb_cap = 0;
    const size_t cxs = 8, nb = (size_t)B;
    const size_t ncnt = (size_t)(p->L1 / p->CB);
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_Y, nb * (size_t)(p->K + 1) * p->L * cxs));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_fscr, nb * (size_t)p->M * cxs));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_part, nb * (size_t)std::max(1, p->SBsplit) * p->L * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->sb_cnt, nb * ncnt * sizeof(int)));
    NUFFT_CUDA_TRY(cudaMemsetAsync(p->sb_cnt, 0, nb * ncnt * sizeof(int), s));
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_args, 2 * nb * sizeof(PassArgs<float>)));
    const int km = p->kmax;
    NUFFT_CUDA_TRY(dev_malloc(&p->sb_beta, nb * (size_t)km * km * sizeof(float)));
    NUFFT_CUDA_TRY(cudaMallocHost(&p->sb_host, 2 * nb * sizeof(PassArgs<float>)));
    if (!p->sb_ev) NUFFT_CUDA_TRY(cudaEventCreateWithFlags(&p->sb_ev, cudaEventDisableTiming));
    // beta for every member (the batched kernels index it by member), laid out as
    // Beta<float, kmax>: kmax x kmax row-major
    std::vector<float> be(nb * (size_t)km * km);
    for (size_t b = 0; b < nb; ++b)
        for (int r = 0; r < km; ++r)
            for (int q = 0; q < km; ++q) be[(b * km + r) * km + q] = (float)p->beta[r][q];
    NUFFT_CUDA_TRY(cudaMemcpy(p->sb_beta, be.data(), be.size() * sizeof(float), cudaMemcpyHostToDevice));
    p->sb_cap = B;
    p->work_bytes += (int64_t)(nb * ((size_t)(p->K + 1) * p->L + p->M + (size_t)std::max(1, p->SBsplit) * p->L) * cxs);
    return NUFFT_OK;
}

// Upload the two argument arrays (first and second pass, B each) of this call.
int upload_args(nufft_plan p, const std::vector<PassArgs<float>> &v, cudaStream_t s) {
    // the staging buffer is reused: the previous call's copy must have been made
    NUFFT_CUDA_TRY(cudaEventSynchronize(p->sb_ev));
    std::copy(v.begin(), v.end(), (PassArgs<float> *)p->sb_host);
    NUFFT_CUDA_TRY(cudaMemcpyAsync(p->sb_args, p->sb_host, v.size() * sizeof(PassArgs<float>),
                                   cudaMemcpyHostToDevice, s));
    NUFFT_CUDA_TRY(cudaEventRecord(p->sb_ev, s));
    return NUFFT_OK;
}

// A member's arguments: its workspace slice; input and output offsets into the packed
// batch (the kernels add the call's base pointers).
PassArgs<float> member(nufft_plan p, int64_t b, int64_t in_off, int64_t out_off) {
    PassArgs<float> a = base_args<float>(p);
    a.Y = (cx<float> *)p->sb_Y + b * (int64_t)(p->K + 1) * p->L;
    a.fscr = (cx<float> *)p->sb_fscr + b * p->M;
    a.part = (cx<float> *)p->sb_part + b * (int64_t)std::max(1, p->SBsplit) * p->L;
    a.counters = p->sb_cnt + b * (int64_t)(p->L1 / p->CB);
    a.in_off = in_off;
    a.out_off = out_off;
    return a;
}

int rows_many_km(nufft_plan p, const PassArgs<float> *args, int64_t B, bool adjoint, const void *in, void *out,
                 cudaStream_t s) {
    const void *be = p->sb_beta;
    const int n = (int)B;
    switch (p->kmax) {
        case 4: return launch_rows_many<float, 4>(p, args, (const Beta<float, 4> *)be, n, adjoint, in, out, s);
        case 8: return launch_rows_many<float, 8>(p, args, (const Beta<float, 8> *)be, n, adjoint, in, out, s);
        case 12: return launch_rows_many<float, 12>(p, args, (const Beta<float, 12> *)be, n, adjoint, in, out, s);
        case 16: return launch_rows_many<float, 16>(p, args, (const Beta<float, 16> *)be, n, adjoint, in, out, s);
        default: return NUFFT_EUNSUPPORTED;
    }
}

// Forward (deriv = false) or forward with f' (deriv = true) of B members.
int fwd_batch(nufft_plan p, int64_t B, const void *c, int64_t ldc, void *f, void *fp, int64_t ldf, bool deriv,
              cudaStream_t s) {
    if (int rc = ensure_workspace(p, B, s)) return rc;
    std::vector<PassArgs<float>> v((size_t)(2 * B));
    for (int64_t b = 0; b < B; ++b) {
        PassArgs<float> a = member(p, b, b * ldc, b * ldf);
        if (deriv) {
            a.mode |= MODE_DERIV;
            a.nranks = p->K + 1;
            a.out2 = (cx<float> *)fp + b * ldf;
        }
        PassArgs<float> a1 = a, a2 = a;
        cols_fields<float>(p, a1, false);
        if (int rc = rows_fields<float>(p, a2, false)) return rc;
        v[(size_t)b] = a1;
        v[(size_t)(B + b)] = a2;
    }
    if (int rc = upload_args(p, v, s)) return rc;
    const PassArgs<float> *args = (const PassArgs<float> *)p->sb_args;
    if (int rc = launch_cols_many<float>(p, args, (int)B, deriv ? p->K + 1 : p->K, false, c, f, s)) return rc;
    return rows_many_km(p, args + B, B, false, c, f, s);
}

// Adjoint of B members: c_b = A^H g_b.
int adj_batch(nufft_plan p, int64_t B, const void *g, int64_t ldg, void *c, int64_t ldc, cudaStream_t s) {
    if (int rc = ensure_workspace(p, B, s)) return rc;
    std::vector<PassArgs<float>> v((size_t)(2 * B));
    for (int64_t b = 0; b < B; ++b) {
        PassArgs<float> a = member(p, b, b * ldg, b * ldc);
        PassArgs<float> aA = a, aB = a;
        if (int rc = rows_fields<float>(p, aA, true)) return rc;
        cols_fields<float>(p, aB, true);
        v[(size_t)b] = aA;
        v[(size_t)(B + b)] = aB;
    }
    if (int rc = upload_args(p, v, s)) return rc;
    const PassArgs<float> *args = (const PassArgs<float> *)p->sb_args;
    if (int rc = rows_many_km(p, args, B, true, g, c, s)) return rc;
    return launch_cols_many<float>(p, args + B, (int)B, std::max(1, p->SBsplit), true, g, c, s);
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
using nufft::fwd_batch;

extern "C" int nufft2_exec_batch(nufft_plan p, int64_t B, const void *c_dev, int64_t ldc, void *f_dev, int64_t ldf,
                                 void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_batch");
    if (!p || B < 0 || ldc < p->N || ldf < p->M) return NUFFT_EINVAL;
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
    if (!p || B < 0 || ldc < p->N || ldg < p->M) return NUFFT_EINVAL;
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
