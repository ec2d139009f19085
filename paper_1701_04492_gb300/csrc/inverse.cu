// inverse.cu -- the inverse NUFFT-II of section 3.3: conjugate gradients on the
// normal equations A^H A c = A^H f.
//
// A^H A is Toeplitz and Hermitian positive definite (A has full column rank):
// (A^H A)_jk = sum_p exp(2 pi i x_p (j - k)) = t_{j-k}, with t_d = (A^H 1)_d for d >= 0
// (A e_0 is the all-ones vector) and t_{-d} = conj(t_d).  It is applied through the
// circulant matrix of size P >= 2N - 1 whose first column is [t_0 .. t_{N-1}, 0 .., 0,
// conj(t_{N-1}) .. conj(t_1)]: with lambda = FFT_P of that column,
// (A^H A) x = IFFT_P(lambda o FFT_P([x; 0]))[0 : N], and IFFT(y) = conj(FFT(conj(y))) / P.
// The FFTs are the library's own passes on a plan of P grid points with gamma = 0
// (rank 1, unit factors): pass 1 and pass 2 writing natural order.
//
// The solver state (that FFT plan, lambda, the CG vectors) is built by the first call
// on a plan and kept until the plan is destroyed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "passes.cuh"
#include "nvtx_range.h"

namespace nufft {
NUFFT_DECLARE_COLS(float)
NUFFT_DECLARE_COLS(double)
NUFFT_DECLARE_ROWS(float, 4)
NUFFT_DECLARE_ROWS(double, 4)
NUFFT_DECLARE_ROWS(dfloat, 4)
NUFFT_DECLARE_COLS(dfloat)

namespace {

constexpr int RED_BLOCKS = 1024;   // partial sums per reduction
constexpr int RED_THREADS = 256;

// scalars of the iteration, on the device
enum { S_RS = 0, S_B2 = 1, S_ALPHA = 2, S_BETA = 3, S_PAP = 4, S_COUNT = 8 };

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;   // thread 0 holds the block's sum
}

template <typename T>
__global__ void k_ones(cx<T> *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = mk<T>(1, 0);
}

// the circulant's first column from t (N entries): t_i, zeros, conj(t_{P-i})
template <typename T>
__global__ void k_circulant(const cx<T> *__restrict__ t, int64_t N, int64_t P, cx<T> *__restrict__ col) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        cx<T> v = mk<T>(0, 0);
        if (i < N) v = t[i];
        else if (i > P - N) v = mk<T>(t[P - i].x, -t[P - i].y);
        col[i] = v;
    }
}

// Z = conj(lambda o X)
template <typename T>
__global__ void k_scale_conj(const cx<T> *__restrict__ lam, const cx<T> *__restrict__ X, int64_t P,
                             cx<T> *__restrict__ Z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> z = cmul<T>(lam[i], X[i]);
        Z[i] = mk<T>(z.x, -z.y);
    }
}

// c = 0, p = r (r holds A^H f), partial sums of |r|^2
template <typename T>
__global__ void k_init(cx<T> *__restrict__ c, const cx<T> *__restrict__ r, cx<T> *__restrict__ p, int64_t N,
                       double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> v = r[i];
        c[i] = mk<T>(0, 0);
        p[i] = v;
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Ap = conj(W[0:N]) / P, partial sums of Re <p, Ap>
template <typename T>
__global__ void k_ap_dot(const cx<T> *__restrict__ W, const cx<T> *__restrict__ p, int64_t N, T invP,
                         cx<T> *__restrict__ Ap, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> w = W[i];
        const cx<T> a = mk<T>(w.x * invP, -w.y * invP);
        Ap[i] = a;
        const cx<T> q = p[i];
        acc += (double)q.x * a.x + (double)q.y * a.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// c += alpha p, r -= alpha Ap, partial sums of |r|^2
template <typename T>
__global__ void k_update(const double *__restrict__ scal, cx<T> *__restrict__ c, cx<T> *__restrict__ r,
                         const cx<T> *__restrict__ p, const cx<T> *__restrict__ Ap, int64_t N,
                         double *__restrict__ part) {
    __shared__ double sh[32];
    const T alpha = (T)scal[S_ALPHA];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> q = p[i], a = Ap[i];
        cx<T> ci = c[i], ri = r[i];
        ci.x = fma(alpha, q.x, ci.x);
        ci.y = fma(alpha, q.y, ci.y);
        ri.x = fma(-alpha, a.x, ri.x);
        ri.y = fma(-alpha, a.y, ri.y);
        c[i] = ci;
        r[i] = ri;
        acc += (double)ri.x * ri.x + (double)ri.y * ri.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// p = r + beta p
template <typename T>
__global__ void k_direction(const double *__restrict__ scal, const cx<T> *__restrict__ r, cx<T> *__restrict__ p,
                            int64_t N) {
    const T beta = (T)scal[S_BETA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> ri = r[i], q = p[i];
        p[i] = mk<T>(fma(beta, q.x, ri.x), fma(beta, q.y, ri.y));
    }
}

// One block: the sum of the partials in a fixed order, then the step's scalars.
// op 0: rs = b2 = sum; op 1: pAp = sum, alpha = rs / pAp; op 2: beta = sum / rs, rs = sum.
__global__ void k_reduce(const double *__restrict__ part, int n, double *__restrict__ scal, int op) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x != 0) return;
    if (op == 0) {
        scal[S_RS] = acc;
        scal[S_B2] = acc;
    } else if (op == 1) {
        scal[S_PAP] = acc;
        scal[S_ALPHA] = acc > 0.0 ? scal[S_RS] / acc : 0.0;
    } else {
        scal[S_BETA] = scal[S_RS] > 0.0 ? acc / scal[S_RS] : 0.0;
        scal[S_RS] = acc;
    }
}

int grid1(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, (n + RED_THREADS - 1) / RED_THREADS));
}

// FFT_P of `in` (its first n_valid entries, zeros beyond) in natural order into `out`,
// in the plan's fused-exec arithmetic (FP32, or double-word for FP64 plans).
template <typename T>
int fft_natural(nufft_plan fp, const void *in, int64_t n_valid, void *out, cudaStream_t s) {
    using A = Arith<T>;
    PassArgs<A> a = base_args<A>(fp);
    a.in = (const io_c<A> *)in;
    a.out = (io_c<A> *)out;
    a.N = n_valid;
    a.nranks = 1;
    if (int rc = launch_cols<A>(fp, a, false, s)) return rc;
    a.mode |= MODE_PLAIN_OUT;
    return launch_rows<A, 4>(fp, a, false, s);
}

// Free the solver state (after a failed build, so that the next call starts afresh).
void drop_state(nufft_plan p) {
    for (void *q : {p->inv_lam, p->inv_x, p->inv_z, p->inv_r, p->inv_p, p->inv_ap, (void *)p->inv_part,
                    (void *)p->inv_scal})
        if (q) cudaFree(q);
    if (p->inv_host) cudaFreeHost(p->inv_host);
    if (p->inv_fft) nufft_destroy(p->inv_fft);
    p->inv_lam = p->inv_x = p->inv_z = p->inv_r = p->inv_p = p->inv_ap = nullptr;
    p->inv_part = p->inv_scal = p->inv_host = nullptr;
    p->inv_fft = nullptr;
    p->inv_P = 0;
}

template <typename T>
int build_state_impl(nufft_plan p, cudaStream_t s) {
    const size_t cxs = 2 * sizeof(T);
    int64_t P = 1024;
    while (P < 2 * p->N) P <<= 1;
    if (P > ((int64_t)1 << LOG2_L_MAX)) return NUFFT_EUNSUPPORTED;
    if (int rc = nufft2_plan(&p->inv_fft, P, 0, nullptr, 0.5, p->prec, P, 0, s)) return rc;
    if (p->inv_fft->K != 1 || p->inv_fft->kmax != 4) return NUFFT_ESTATE;
    p->inv_P = P;
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_lam, (size_t)P * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_x, (size_t)P * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_z, (size_t)P * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_r, (size_t)p->N * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_p, (size_t)p->N * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_ap, (size_t)p->N * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_part, RED_BLOCKS * sizeof(double)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->inv_scal, S_COUNT * sizeof(double)));
    NUFFT_CUDA_TRY(cudaMallocHost(&p->inv_host, 2 * sizeof(double)));
    p->work_bytes += (int64_t)((3 * (size_t)P + 3 * (size_t)p->N) * cxs);
    // t = A^H 1 (its first N entries are the Toeplitz column), then lambda
    void *ones = nullptr;
    NUFFT_CUDA_TRY(dev_malloc((void **)&ones, (size_t)std::max<int64_t>(p->M, 1) * cxs));
    k_ones<T><<<grid1(p->M), RED_THREADS, 0, s>>>((cx<T> *)ones, p->M);
    int rc = nufft1_exec(p, ones, p->inv_r, s);
    if (!rc) {
        k_circulant<T><<<grid1(P), RED_THREADS, 0, s>>>((const cx<T> *)p->inv_r, p->N, P, (cx<T> *)p->inv_z);
        rc = cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
    }
    if (!rc) rc = fft_natural<T>(p->inv_fft, p->inv_z, P, p->inv_lam, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = NUFFT_ECUDA;
    cudaFree(ones);
    return rc;
}

template <typename T>
int build_state(nufft_plan p, cudaStream_t s) {
    const int rc = build_state_impl<T>(p, s);
    if (rc) drop_state(p);
    return rc;
}

template <typename T>
int solve(nufft_plan p, const void *f, void *c, double tol, int maxit, int *iters, double *relres, cudaStream_t s) {
    if (!p->inv_fft)
        if (int rc = build_state<T>(p, s)) return rc;
    const int64_t N = p->N, P = p->inv_P;
    cx<T> *cv = (cx<T> *)c, *r = (cx<T> *)p->inv_r, *pv = (cx<T> *)p->inv_p, *ap = (cx<T> *)p->inv_ap;
    double *host = p->inv_host;
    if (int rc = nufft1_exec(p, f, r, s)) return rc;   // r = b = A^H f
    k_init<T><<<grid1(N), RED_THREADS, 0, s>>>(cv, r, pv, N, p->inv_part);
    k_reduce<<<1, RED_THREADS, 0, s>>>(p->inv_part, grid1(N), p->inv_scal, 0);
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaMemcpyAsync(host, p->inv_scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    const double b2 = host[1];
    double rs = host[0];
    int it = 0;
    while (it < maxit && b2 > 0.0 && std::sqrt(rs) > tol * std::sqrt(b2)) {
        // Ap = (A^H A) p through the circulant
        if (int rc = fft_natural<T>(p->inv_fft, pv, N, p->inv_x, s)) return rc;
        k_scale_conj<T><<<grid1(P), RED_THREADS, 0, s>>>((const cx<T> *)p->inv_lam, (const cx<T> *)p->inv_x, P,
                                                         (cx<T> *)p->inv_z);
        if (int rc = fft_natural<T>(p->inv_fft, p->inv_z, P, p->inv_x, s)) return rc;
        k_ap_dot<T><<<grid1(N), RED_THREADS, 0, s>>>((const cx<T> *)p->inv_x, pv, N, T(1.0 / (double)P), ap,
                                                     p->inv_part);
        k_reduce<<<1, RED_THREADS, 0, s>>>(p->inv_part, grid1(N), p->inv_scal, 1);
        k_update<T><<<grid1(N), RED_THREADS, 0, s>>>(p->inv_scal, cv, r, pv, ap, N, p->inv_part);
        k_reduce<<<1, RED_THREADS, 0, s>>>(p->inv_part, grid1(N), p->inv_scal, 2);
        k_direction<T><<<grid1(N), RED_THREADS, 0, s>>>(p->inv_scal, r, pv, N);
        NUFFT_CUDA_TRY(cudaGetLastError());
        NUFFT_CUDA_TRY(cudaMemcpyAsync(host, p->inv_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
        rs = host[0];
        ++it;
    }
    if (b2 == 0.0) NUFFT_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)N * 2 * sizeof(T), s));
    if (iters) *iters = it;
    if (relres) *relres = b2 > 0.0 ? std::sqrt(rs / b2) : 0.0;
    return nufft2_check(p, s);
}

}  // namespace
}  // namespace nufft

extern "C" int nufft2_inverse(nufft_plan p, const void *f_dev, void *c_dev, double tol, int maxit, int *iterations,
                              double *relres, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_inverse");
    if (!p || !c_dev || (p->M > 0 && !f_dev) || !(tol >= 0.0) || maxit < 0) return NUFFT_EINVAL;
    if (p->dims == 2) return NUFFT_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? nufft::solve<float>(p, f_dev, c_dev, tol, maxit, iterations, relres, s)
                                : nufft::solve<double>(p, f_dev, c_dev, tol, maxit, iterations, relres, s);
}
