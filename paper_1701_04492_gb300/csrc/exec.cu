// exec.cu -- the online stage: launch geometry, the exec entry points of the C ABI,
// and the unfused comparator (the section 2.3 one-liner run step by step).
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cstdint>

#include "passes.cuh"
#include "nvtx_range.h"

namespace nufft {

NUFFT_DECLARE_ROWS(float, 4)
NUFFT_DECLARE_ROWS(float, 8)
NUFFT_DECLARE_ROWS(float, 12)
NUFFT_DECLARE_ROWS(float, 16)
NUFFT_DECLARE_ROWS(double, 4)
NUFFT_DECLARE_ROWS(double, 8)
NUFFT_DECLARE_ROWS(double, 12)
NUFFT_DECLARE_ROWS(double, 16)
NUFFT_DECLARE_ROWS(dfloat, 4)
NUFFT_DECLARE_ROWS(dfloat, 8)
NUFFT_DECLARE_ROWS(dfloat, 12)
NUFFT_DECLARE_ROWS(dfloat, 16)
NUFFT_DECLARE_COLS(float)
NUFFT_DECLARE_COLS(double)
NUFFT_DECLARE_COLS(dfloat)
NUFFT_DECLARE_COLS_2D()
NUFFT_DECLARE_2D(4)
NUFFT_DECLARE_2D(8)
NUFFT_DECLARE_2D(12)
NUFFT_DECLARE_2D(16)
NUFFT_DECLARE_COLS_2D_T(double)
NUFFT_DECLARE_2D_T(double, 4)
NUFFT_DECLARE_2D_T(double, 8)
NUFFT_DECLARE_2D_T(double, 12)
NUFFT_DECLARE_2D_T(double, 16)

namespace {

// Complex elements per 128-byte shared-memory wavefront.
template <typename T> constexpr int nbank() { return 128 / (2 * (int)sizeof(T)); }

// Slot stride (elements) for a team slot of a length-P FFT: padded length, then
// nudged so that the q teams sharing a wavefront land on disjoint banks.
template <typename T>
int slot_stride(int P, int E, int q) {
    const int base = P + P / E;
    const int nb = nbank<T>();
    int s = base;
    if (q > 1) {
        const int target = nb / std::min(q, nb);
        s = base + (((target - base % nb) % nb) + nb) % nb;
    }
    // slots are bulk-copy destinations: keep every slot 16-byte aligned
    while ((s * 2 * (int)sizeof(T)) % 16 != 0) ++s;
    return s;
}

int clamp_pow2(int v, int lo, int hi) { return std::max(lo, std::min(hi, v)); }

}  // namespace

template <typename T>
int plan_geometry(nufft_plan p) {
    // values per thread of each pass's team FFT (see EmaxT) and the team sizes
    const int E1 = std::min(EmaxT<T, PK_ROW_FWD>::v, p->L1), TT1 = p->L1 / E1;      // pass 2
    const int E1a = std::min(EmaxT<T, PK_ROW_ADJ>::v, p->L1), TT1a = p->L1 / E1a;   // pass A
    const int E2 = std::min(EmaxT<T, PK_COL_FWD>::v, p->L2), TT2 = p->L2 / E2;      // pass 1
    const int E2b = std::min(EmaxT<T, PK_COL_ADJ>::v, p->L2), TT2b = p->L2 / E2b;   // pass B
    const size_t cxs = 2 * sizeof(T);
    // column passes: C columns per CTA, columns fastest across the lanes
    p->C1 = clamp_pow2((256 / TT2) >> p->c1_shift, 1, p->L1);
    // one 32 KiB tile of the adjoint intermediate: pass A writes it (each of its rows a
    // run of CB columns, a whole 32-byte sector or more), pass B fetches it by one bulk
    // copy; pass B's CTA then has CB TT2b threads (256 in FP32, 128 in FP64)
    p->CB = clamp_pow2((int)(32768 / ((size_t)p->L2 * cxs)), 1, p->L1);
    (void)TT2b;
    p->S1 = slot_stride<T>(p->L2, E2, p->C1);
    p->SB = slot_stride<T>(p->L2, E2b, p->CB);
    p->smem1 = ((size_t)p->C1 * p->S1 + (size_t)p->C1 * E2) * cxs;   // slots + four-step table
    // two tile buffers (copy landing zone and exchange slots), then two mbarriers
    p->smemB = ((2 * (size_t)p->CB * p->SB * cxs + 15) / 16) * 16 + 2 * sizeof(uint64_t);
    // rank splits of pass B, at most one rank each.  FP32: about one CTA per SM.  Every
    // further split costs a partial sum to write and add; at 2^20 (K = 12) pass B took
    // 45 us with 256 CTAs (no split), 49 with two splits and 53 with three; at 2^18 20.5 us
    // with 128 CTAs against 28.7 with 640; at 2^22 151.6 us unsplit against 190.5 with two.
    // The double-word FP64 pass B (128-thread CTAs, three per SM, several times the
    // arithmetic per element) wants about four per SM: 308 us with two splits at 2^20
    // against 342 unsplit.
    {
        const int blocks = p->L1 / p->CB, sms = device_sm_count();
        const int target = std::is_same<T, float>::value ? sms : 4 * sms;
        p->SBsplit = std::max(1, std::min(p->K, (target + blocks - 1) / blocks));
    }
    // row passes: buckets of B2 rows; G ranks staged at once by nt teams
    p->B2 = clamp_pow2(1024 / p->L1, 1, p->L2);
    p->NB = p->L2 / p->B2;
    p->S2 = slot_stride<T>(p->L1, E1, std::max(1, nbank<T>() / TT1));
    p->SA = slot_stride<T>(p->L1, E1a, std::max(1, nbank<T>() / TT1a));
    p->chunkA = 512;
    const size_t staging = (size_t)p->chunkA * (sizeof(int32_t) + sizeof(T)) + (size_t)p->chunkA * cxs;
    // one slot per staged row (idle teams need none)
    auto nslots = [&](int G) { return (size_t)G * p->B2; };
    // pass 2: slots, then (16-byte aligned) one mbarrier per slot
    auto body2 = [&](int G) { return (nslots(G) * p->S2 * cxs + 15) / 16 * 16; };
    auto bytes2 = [&](int G, int nt) { return body2(G) + nslots(G) * sizeof(uint64_t) + 0 * nt; };
    // pass A: slots, four-step tables, staged samples
    auto bytesA = [&](int G, int nt) { return (nslots(G) * p->SA + (size_t)nt * E1a) * cxs + staging; };
    // teams (of TTr threads) for J row FFTs: the fewest rounds with at most 256
    // threads, then the fewest teams that still take that many rounds
    auto teams_of = [](int TTr) {
        const int maxt = std::max(1, 256 / TTr);
        return [=](int J) {
            const int rounds = (J + maxt - 1) / maxt;
            int nt = (J + rounds - 1) / rounds;
            if (nt * TTr < 64) nt = std::min(maxt, std::max(nt, (64 + TTr - 1) / TTr));
            return std::max(1, nt);
        };
    };
    const auto teams = teams_of(TT1), teamsA = teams_of(TT1a);
    auto choose = [&](int Gmax, auto bytes, auto teams, int *Gout, int *ntout, size_t budget) -> bool {
        int G = Gmax;
        while (G > 1 && bytes(G, teams(G * p->B2)) > budget) --G;
        *Gout = G;
        *ntout = teams(G * p->B2);
        return bytes(G, *ntout) <= budget;
    };
    // pass 2 stages up to K + 1 ranks (the FP32 derivative mode adds rank K, and its
    // gather needs them all in one group).  FP64 plans (double-word passes, which take
    // the derivative another way) stage groups that let two CTAs share an SM: at 2^20
    // (K = 12) pass 2 took 639 us with all 12 ranks (192 KB, one CTA per SM) and 403 us
    // in two groups of 6, the partial sums kept in the plan's scratch between them.
    const size_t budget2 = std::is_same<T, float>::value ? SMEM_BUDGET : (size_t)110 * 1024;
    int nt_dummy = 1;
    if (!choose(p->K + 1, bytes2, teams, &p->G, &nt_dummy, budget2)) return NUFFT_EUNSUPPORTED;
    p->nt2 = teams(std::min(p->G, p->K) * p->B2);   // forward: K ranks
    p->nt2d = teams(p->G * p->B2);                  // derivative: K + 1 ranks
    p->mbar_off2 = body2(p->G);
    p->smem2 = bytes2(p->G, 1);
    // (A smaller group for the plain forward, so that four CTAs fit per SM, was faster,
    // 78 -> 74 us at 2^20, until the row passes kept their stage twiddles in registers: at
    // about 120 registers per thread four CTAs no longer fit.)
    // (Pass A keeps the full budget in both precisions: its samples are staged again per
    // group, and the FP64 pass A measured 1003 us in one group against 1139 in two.)
    if (!choose(p->K, bytesA, teamsA, &p->GA, &p->ntA, SMEM_BUDGET)) return NUFFT_EUNSUPPORTED;
    p->smemA = bytesA(p->GA, p->ntA);
    if (p->smem1 > SMEM_BUDGET || p->smemB > SMEM_BUDGET) return NUFFT_EUNSUPPORTED;
    return NUFFT_OK;
}

template <typename T>
PassArgs<T> base_args(nufft_plan p) {
    PassArgs<T> a{};
    a.Y = (cx<T> *)p->Y;
    a.fscr = (cx<T> *)p->fscr;
    a.tsorted = p->tsorted;
    a.perm = p->perm;
    a.bstart = p->bstart;
    a.dsorted = (const T *)p->dsorted;
    a.twc = tab<T>(p->twst2, p->twst2_dw);
    a.twr = tab<T>(p->twst1, p->twst1_dw);
    a.twhi = tab<T>(p->twhi, p->twhi_dw);
    a.part = (cx<T> *)p->part;
    a.counters = p->counters;
    a.err = p->err;
    a.vfac = (const T *)p->Vfac;
    a.ufac = (const cx<T> *)p->Ufac;
    a.mode = p->Ufac ? MODE_FACTORS : 0;
    a.twlo = tab<T>(p->twlo, p->twlo_dw);
    a.N = p->N;
    a.M = p->M;
    a.L = p->L;
    a.L1 = p->L1;
    a.L2 = p->L2;
    a.lg1 = p->lg1;
    a.lg2 = p->lg2;
    a.K = p->K;
    a.G = p->G;
    a.B2 = p->B2;
    a.nranks = p->K;
    a.piN = (T)(3.14159265358979323846 * (double)p->N);
    a.inv_gamma = p->gamma > 0.0 ? (T)(1.0 / p->gamma) : T(0);
    return a;
}

template PassArgs<float> base_args<float>(nufft_plan);
template PassArgs<double> base_args<double>(nufft_plan);
template PassArgs<dfloat> base_args<dfloat>(nufft_plan);

namespace {

template <typename T>
int run_rows(nufft_plan p, const PassArgs<T> &a, bool adjoint, cudaStream_t s) {
    switch (p->kmax) {
        case 4: return launch_rows<T, 4>(p, a, adjoint, s);
        case 8: return launch_rows<T, 8>(p, a, adjoint, s);
        case 12: return launch_rows<T, 12>(p, a, adjoint, s);
        case 16: return launch_rows<T, 16>(p, a, adjoint, s);
        default: return NUFFT_EUNSUPPORTED;
    }
}

// ---- unfused comparator kernels ----------------------------------------------------

// U[j][r] = sum'_p a_pr exp(-i pi d_j) T_p(d_j / gamma), FP64 (eq. (2.6)).
template <typename T>
__global__ void k_uf_U(const double *__restrict__ d, int64_t M, int K, double inv_gamma,
                       int trivial, const Beta<double, KMAX_ALL> aw, cx<T> *__restrict__ U) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (trivial) { U[j * K] = mk<T>(1, 0); continue; }
        const double xi = d[j] * inv_gamma;
        double Tp[KMAX_ALL];
        Tp[0] = 1.0;
        Tp[1] = xi;
        for (int q = 2; q < K; ++q) Tp[q] = 2.0 * xi * Tp[q - 1] - Tp[q - 2];
        double sn, cs;
        sincospi(d[j], &sn, &cs);
        for (int r = 0; r < K; ++r) {
            double s = 0.0;
            for (int q = 0; q < K; ++q) s += aw.b[r][q] * Tp[q];
            // i^r exp(-i pi d) s
            cx<double> u = mk<double>(cs * s, -sn * s);
            u = mul_ipow<double>(u, r);
            U[j * K + r] = mk<T>((T)u.x, (T)u.y);
        }
    }
}

// V[k][r] = T_r(2k/N - 1), V[k][0] = 1/2 (eq. (2.6)), FP64.
template <typename T>
__global__ void k_uf_V(int64_t N, int K, int trivial, T *__restrict__ V) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (trivial) { V[k * K] = T(1); continue; }
        const double z = double(2 * k - N) / double(N);
        double a = 1.0, b = z;
        V[k * K] = T(0.5);
        if (K > 1) V[k * K + 1] = (T)z;
        for (int r = 2; r < K; ++r) {
            const double c = 2.0 * z * b - a;
            a = b;
            b = c;
            V[k * K + r] = (T)c;
        }
    }
}

// W[r][k] = V[k][r] c_k for k < N, 0 for N <= k < L.
template <typename T>
__global__ void k_uf_vscale(const cx<T> *__restrict__ c, const T *__restrict__ V, int64_t N,
                            int64_t L, int K, cx<T> *__restrict__ W) {
    const int64_t tot = (int64_t)K * L;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / L);
        const int64_t k = idx - (int64_t)r * L;
        cx<T> w = mk<T>(0, 0);
        if (k < N) {
            const T v = V[k * K + r];
            const cx<T> cc = c[k];
            w = mk<T>(v * cc.x, v * cc.y);
        }
        W[idx] = w;
    }
}

// Xg[r][j] = X[r][t_j]  (the row gather I_L(t,:))
template <typename T>
__global__ void k_uf_gather(const cx<T> *__restrict__ X, const int32_t *__restrict__ t, int64_t M,
                            int64_t L, int K, cx<T> *__restrict__ Xg) {
    const int64_t tot = (int64_t)K * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / M);
        const int64_t j = idx - (int64_t)r * M;
        Xg[idx] = X[(int64_t)r * L + t[j]];
    }
}

// f_j = sum_r U[j][r] Xg[r][j]  ((U .* X) * ones(K))
template <typename T>
__global__ void k_uf_ranksum(const cx<T> *__restrict__ U, const cx<T> *__restrict__ Xg, int64_t M,
                             int K, cx<T> *__restrict__ f) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        cx<T> acc = mk<T>(0, 0);
        for (int r = 0; r < K; ++r) acc = cadd<T>(acc, cmul<T>(U[j * K + r], Xg[(int64_t)r * M + j]));
        f[j] = acc;
    }
}

int grid1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

// Factor tables of the fused path's MODE_FACTORS, FP64 (eq. (2.6)):
//   Vfac[r][k] = v_r(k) = T_r(2k/N - 1) (v_0 = 1/2), rank-major;
//   Ufac[i][r] = u_r(perm[i]) = sum'_p a_pr exp(-i pi d) T_p(d / gamma), sorted order.
template <typename T>
__global__ void k_fac_V(int64_t N, int K, int trivial, T *__restrict__ V) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (trivial) { V[k] = T(1); continue; }
        const double z = double(2 * k - N) / double(N);
        double a = 1.0, b = z;
        V[k] = T(0.5);
        if (K > 1) V[N + k] = (T)z;
        for (int r = 2; r < K; ++r) {
            const double c = 2.0 * z * b - a;
            a = b;
            b = c;
            V[(int64_t)r * N + k] = (T)c;
        }
    }
}

template <typename T>
__global__ void k_fac_U(const io_r<T> *__restrict__ dsorted, int64_t M, int K, double inv_gamma, int trivial,
                        const Beta<double, KMAX_ALL> aw, cx<T> *__restrict__ U) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (trivial) { U[i * K] = mk<T>(1, 0); continue; }
        const double d = (double)dsorted[i];
        const double xi = d * inv_gamma;
        double Tp[KMAX_ALL];
        Tp[0] = 1.0;
        Tp[1] = xi;
        for (int q = 2; q < K; ++q) Tp[q] = 2.0 * xi * Tp[q - 1] - Tp[q - 2];
        double sn, cs;
        sincospi(d, &sn, &cs);
        for (int r = 0; r < K; ++r) {
            double sum = 0.0;
            for (int q = 0; q < K; ++q) sum += aw.b[r][q] * Tp[q];
            const cx<double> u = mul_ipow<double>(mk<double>(cs * sum, -sn * sum), r);
            U[i * K + r] = mk<T>(T(u.x), T(u.y));
        }
    }
}

}  // namespace

template <typename T>
int plan_factor_tables(nufft_plan p, cudaStream_t s) {
    const size_t cxs = 2 * sizeof(T);
    const int64_t M = std::max<int64_t>(p->M, 1);
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->Ufac, (size_t)M * p->K * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->Vfac, (size_t)p->N * p->K * sizeof(T)));
    p->work_bytes += (int64_t)((size_t)M * p->K * cxs + (size_t)p->N * p->K * sizeof(T));
    Beta<double, KMAX_ALL> aw{};
    for (int r = 0; r < p->K; ++r)
        for (int q = 0; q < p->K; ++q) aw.b[r][q] = (q == 0 ? 0.5 : 1.0) * p->alpha[q][r];
    const int trivial = p->gamma == 0.0;
    const double inv_gamma = trivial ? 0.0 : 1.0 / p->gamma;
    if (p->M > 0)
        k_fac_U<T><<<grid1d(p->M), 256, 0, s>>>((const io_r<T> *)p->dsorted, p->M, p->K, inv_gamma, trivial, aw,
                                                (cx<T> *)p->Ufac);
    k_fac_V<T><<<grid1d(p->N), 256, 0, s>>>(p->N, p->K, trivial, (T *)p->Vfac);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template int plan_factor_tables<dfloat>(nufft_plan, cudaStream_t);

namespace {
}  // namespace

template <typename T>
int plan_unfused_factors(nufft_plan p, cudaStream_t s) {
    const size_t cxs = 2 * sizeof(T);
    const int64_t M = std::max<int64_t>(p->M, 1);
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->U, (size_t)M * p->K * cxs));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->V, (size_t)p->N * p->K * sizeof(T)));
    NUFFT_CUDA_TRY(dev_malloc((void **)&p->Xg, (size_t)p->K * p->L * cxs));
    p->work_bytes += (int64_t)((size_t)M * p->K * cxs + (size_t)p->N * p->K * sizeof(T) +
                               (size_t)p->K * p->L * cxs);
    if ((size_t)p->K * p->M > (size_t)(p->K + 1) * p->L) {   // the gathered K x M block reuses Y
        cudaFree(p->Y);
        p->Y = nullptr;
        NUFFT_CUDA_TRY(dev_malloc((void **)&p->Y, (size_t)p->K * p->M * cxs));
        p->work_bytes += (int64_t)(((size_t)p->K * p->M - (size_t)(p->K + 1) * p->L) * cxs);
    }
    Beta<double, KMAX_ALL> aw{};
    for (int r = 0; r < p->K; ++r)
        for (int q = 0; q < p->K; ++q) aw.b[r][q] = (q == 0 ? 0.5 : 1.0) * p->alpha[q][r];
    const int trivial = p->gamma == 0.0;
    const double inv_gamma = trivial ? 0.0 : 1.0 / p->gamma;
    if (p->M > 0)
        k_uf_U<T><<<grid1d(p->M), 256, 0, s>>>(p->d_j, p->M, p->K, inv_gamma, trivial, aw, (cx<T> *)p->U);
    k_uf_V<T><<<grid1d(p->N), 256, 0, s>>>(p->N, p->K, trivial, (T *)p->V);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

// The 2D transform (section 4, eq. (4.4)): FP32 plans only.
template <typename T>
int exec_forward_2d(nufft_plan p, const void *C, void *f, cudaStream_t s) {
    if (p->M == 0) return NUFFT_OK;
    PassArgs<T> a = base_args<T>(p);
    a.in = (const cx<T> *)C;
    a.out = (cx<T> *)f;
    a.ncol = (int)p->N2;
    a.ldc = (int)p->N2;
    a.K2 = p->K2;
    a.dsorted2 = (const T *)p->dsorted2;
    a.vy = (const T *)p->vy;
    a.inv_gamma2 = p->gamma2 > 0.0 ? (T)(1.0 / p->gamma2) : T(0);
    if (int rc = mark(p, s, true)) return rc;
    if (int rc = launch_cols_2d<T>(p, a, s)) return rc;
    if (int rc = mark(p, s, false)) return rc;
    int rc = NUFFT_EUNSUPPORTED;
    switch (p->kmax) {
        case 4: rc = launch_rows_2d<T, 4>(p, a, s); break;
        case 8: rc = launch_rows_2d<T, 8>(p, a, s); break;
        case 12: rc = launch_rows_2d<T, 12>(p, a, s); break;
        case 16: rc = launch_rows_2d<T, 16>(p, a, s); break;
        default: break;
    }
    if (rc) return rc;
    return mark(p, s, false);
}

// The 2D adjoint, C = A^H g (section 4, eq. (4.4) conjugated and reversed): the row
// pass (scatter, inverse FFTs over t^y, y-scale, sum over r2), then the column pass
// (inverse FFTs over s1, x-scale, sum over r1).  C is m x n row-major.
template <typename T>
int exec_adjoint_2d(nufft_plan p, const void *g, void *C, cudaStream_t s) {
    if (p->M == 0) {
        NUFFT_CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)p->N * p->N2 * 2 * sizeof(T), s));
        return NUFFT_OK;
    }
    PassArgs<T> a = base_args<T>(p);
    a.in = (const cx<T> *)g;
    a.out = (cx<T> *)C;
    a.ncol = (int)p->N2;
    a.ldc = (int)p->N2;
    a.K2 = p->K2;
    a.dsorted2 = (const T *)p->dsorted2;
    a.vy = (const T *)p->vy;
    a.inv_gamma2 = p->gamma2 > 0.0 ? (T)(1.0 / p->gamma2) : T(0);
    if (int rc = mark(p, s, true)) return rc;
    int rc = NUFFT_EUNSUPPORTED;
    switch (p->kmax) {
        case 4: rc = launch_rows_2d_adj<T, 4>(p, a, s); break;
        case 8: rc = launch_rows_2d_adj<T, 8>(p, a, s); break;
        case 12: rc = launch_rows_2d_adj<T, 12>(p, a, s); break;
        case 16: rc = launch_rows_2d_adj<T, 16>(p, a, s); break;
        default: break;
    }
    if (rc) return rc;
    if (int rc2 = mark(p, s, false)) return rc2;
    if (int rc2 = launch_cols_2d_adj<T>(p, a, s)) return rc2;
    return mark(p, s, false);
}

template <typename T>
int exec_forward(nufft_plan p, const void *c, void *f, cudaStream_t s) {
    if (p->dims == 2) return exec_forward_2d<T>(p, c, f, s);
    if (p->M == 0) return NUFFT_OK;
    using A = Arith<T>;
    PassArgs<A> a = base_args<A>(p);
    a.in = (const io_c<A> *)c;
    a.out = (io_c<A> *)f;
    if (int rc = mark(p, s, true)) return rc;
    if (int rc = launch_cols<A>(p, a, false, s)) return rc;
    if (int rc = mark(p, s, false)) return rc;
    if (int rc = run_rows<A>(p, a, false, s)) return rc;
    return mark(p, s, false);
}

template <typename T>
int exec_adjoint(nufft_plan p, const void *g, void *c, cudaStream_t s) {
    if (p->dims == 2) return exec_adjoint_2d<T>(p, g, c, s);
    if (p->M == 0) {
        NUFFT_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)p->N * 2 * sizeof(T), s));
        return NUFFT_OK;
    }
    using A = Arith<T>;
    PassArgs<A> a = base_args<A>(p);
    a.in = (const io_c<A> *)g;
    a.out = (io_c<A> *)c;
    if (int rc = mark(p, s, true)) return rc;
    if (int rc = run_rows<A>(p, a, true, s)) return rc;
    if (int rc = mark(p, s, false)) return rc;
    if (int rc = launch_cols<A>(p, a, true, s)) return rc;
    return mark(p, s, false);
}

template <typename T>
int exec_dx(nufft_plan p, const void *c, const void *g, void *gx, int acc, cudaStream_t s) {
    if (p->M == 0) return NUFFT_OK;
    using A = Arith<T>;
    PassArgs<A> a = base_args<A>(p);
    a.in = (const io_c<A> *)c;
    a.g = (const io_c<A> *)g;
    a.gx = (io_r<A> *)gx;
    a.accumulate = acc;
    if (!kFactors<A> && p->G >= p->K + 1) {
        a.mode |= MODE_DERIV | MODE_GX;
        a.nranks = p->K + 1;
        a.out = nullptr;
        a.out2 = nullptr;
    } else {
        a.mode |= MODE_PRESCALE | MODE_GX;
    }
    if (int rc = mark(p, s, true)) return rc;
    if (int rc = launch_cols<A>(p, a, false, s)) return rc;
    if (int rc = mark(p, s, false)) return rc;
    if (int rc = run_rows<A>(p, a, false, s)) return rc;
    return mark(p, s, false);
}

// f = A c and f' = df/dx (the derivative of eq. (1.2) with respect to each x_j).
template <typename T>
int exec_deriv(nufft_plan p, const void *c, void *f, void *fprime, cudaStream_t s) {
    if (p->M == 0) return NUFFT_OK;
    using A = Arith<T>;
    if (!kFactors<A> && p->G >= p->K + 1) {
        PassArgs<A> a = base_args<A>(p);
        a.in = (const io_c<A> *)c;
        a.out = (io_c<A> *)f;
        a.out2 = (io_c<A> *)fprime;
        a.mode |= MODE_DERIV;
        a.nranks = p->K + 1;
        if (int rc = mark(p, s, true)) return rc;
        if (int rc = launch_cols<A>(p, a, false, s)) return rc;
        if (int rc = mark(p, s, false)) return rc;
        if (int rc = run_rows<A>(p, a, false, s)) return rc;
        return mark(p, s, false);
    }
    // otherwise: the forward, then A((-2 pi i k) o c)
    if (int rc = exec_forward<T>(p, c, f, s)) return rc;
    PassArgs<A> a = base_args<A>(p);
    a.in = (const io_c<A> *)c;
    a.out = (io_c<A> *)fprime;
    a.mode |= MODE_PRESCALE;
    if (int rc = launch_cols<A>(p, a, false, s)) return rc;
    return run_rows<A>(p, a, false, s);
}

// gx_j (+)= Re(conj(g_j) f'_j)
template <typename T>
__global__ void k_grad_x(const cx<T> *__restrict__ g, const cx<T> *__restrict__ fp, int64_t M, int acc,
                         T *__restrict__ gx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> a = g[j], b = fp[j];
        const T re = fma(a.x, b.x, a.y * b.y);
        gx[j] = acc ? gx[j] + re : re;
    }
}

template <typename T>
int exec_grad_x(nufft_plan p, const void *g, const void *fprime, void *gx, int acc, cudaStream_t s) {
    if (p->M == 0) return NUFFT_OK;
    k_grad_x<T><<<grid1d(p->M), 256, 0, s>>>((const cx<T> *)g, (const cx<T> *)fprime, p->M, acc, (T *)gx);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template <typename T>
int exec_unfused(nufft_plan p, const void *c, void *f, cudaStream_t s) {
    if (!(p->flags & NUFFT_PLAN_UNFUSED)) return NUFFT_ESTATE;
    if (p->M == 0) return NUFFT_OK;
    cx<T> *W = (cx<T> *)p->Xg;   // K x L: scaled columns, later the FFT outputs X
    k_uf_vscale<T><<<grid1d((int64_t)p->K * p->L), 256, 0, s>>>((const cx<T> *)c, (const T *)p->V,
                                                                p->N, p->L, p->K, W);
    NUFFT_CUDA_TRY(cudaGetLastError());
    PassArgs<T> a = base_args<T>(p);
    a.in = W;
    a.out = W;
    a.mode |= MODE_PLAIN_IN | MODE_PLAIN_OUT;
    if (int rc = launch_cols<T>(p, a, false, s)) return rc;   // W -> Y
    if (int rc = run_rows<T>(p, a, false, s)) return rc;      // Y -> X (in W)
    cx<T> *Xg = (cx<T> *)p->Y;
    k_uf_gather<T><<<grid1d((int64_t)p->K * p->M), 256, 0, s>>>(W, p->t_j, p->M, p->L, p->K, Xg);
    k_uf_ranksum<T><<<grid1d(p->M), 256, 0, s>>>((const cx<T> *)p->U, Xg, p->M, p->K, (cx<T> *)f);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template int plan_geometry<float>(nufft_plan);
template int plan_geometry<double>(nufft_plan);
template int plan_unfused_factors<float>(nufft_plan, cudaStream_t);
template int plan_unfused_factors<double>(nufft_plan, cudaStream_t);

}  // namespace nufft

// ---- C ABI --------------------------------------------------------------------------

using nufft::exec_adjoint;
using nufft::exec_dx;
using nufft::exec_forward;
using nufft::exec_unfused;

extern "C" int nufft2_exec(nufft_plan p, const void *c_dev, void *f_dev, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec");
    if (!p || !c_dev || (p->M > 0 && !f_dev)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? exec_forward<float>(p, c_dev, f_dev, s)
                                : exec_forward<double>(p, c_dev, f_dev, s);
}

extern "C" int nufft1_exec(nufft_plan p, const void *g_dev, void *c_dev, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft1_exec");
    if (!p || !c_dev || (p->M > 0 && !g_dev)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? exec_adjoint<float>(p, g_dev, c_dev, s)
                                : exec_adjoint<double>(p, g_dev, c_dev, s);
}

extern "C" int nufft2_exec_dx(nufft_plan p, const void *c_dev, const void *g_dev, void *gx_dev,
                              int accumulate, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_dx");
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;   // the 2D transform has its forward and adjoint only
    if (!p || !c_dev || (p->M > 0 && (!g_dev || !gx_dev))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? exec_dx<float>(p, c_dev, g_dev, gx_dev, accumulate, s)
                                : exec_dx<double>(p, c_dev, g_dev, gx_dev, accumulate, s);
}

extern "C" int nufft2_exec_deriv(nufft_plan p, const void *c_dev, void *f_dev, void *fprime_dev,
                                 void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_deriv");
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;   // the 2D transform has its forward and adjoint only
    if (!p || !c_dev || (p->M > 0 && (!f_dev || !fprime_dev))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? nufft::exec_deriv<float>(p, c_dev, f_dev, fprime_dev, s)
                                : nufft::exec_deriv<double>(p, c_dev, f_dev, fprime_dev, s);
}

extern "C" int nufft2_grad_x(nufft_plan p, const void *g_dev, const void *fprime_dev, void *gx_dev,
                             int accumulate, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_grad_x");
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;   // the 2D transform has its forward and adjoint only
    if (!p || (p->M > 0 && (!g_dev || !fprime_dev || !gx_dev))) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? nufft::exec_grad_x<float>(p, g_dev, fprime_dev, gx_dev, accumulate, s)
                                : nufft::exec_grad_x<double>(p, g_dev, fprime_dev, gx_dev, accumulate, s);
}

extern "C" int nufft2_exec_host(nufft_plan p, const void *c_host, void *f_host, void *stream) {
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;   // the 2D transform has its forward and adjoint only
    if (!p || !c_host || (p->M > 0 && !f_host)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cxs = p->prec == NUFFT_F32 ? 8 : 16;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(p->cstage, c_host, (size_t)p->N * cxs, cudaMemcpyHostToDevice, s));
    if (int rc = nufft2_exec(p, p->cstage, p->fstage, stream)) return rc;
    if (p->M > 0)
        NUFFT_CUDA_TRY(cudaMemcpyAsync(f_host, p->fstage, (size_t)p->M * cxs, cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

extern "C" int nufft2_exec_unfused(nufft_plan p, const void *c_dev, void *f_dev, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_unfused");
    if (p && p->dims == 2) return NUFFT_EUNSUPPORTED;   // the 2D transform has its forward and adjoint only
    if (!p || !c_dev || (p->M > 0 && !f_dev)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? exec_unfused<float>(p, c_dev, f_dev, s)
                                : exec_unfused<double>(p, c_dev, f_dev, s);
}

namespace nufft {
namespace {

// One training step with host buffers: upload g and c, the adjoint, the forward with f'
// and dL/dx, download A^H g, f and gx.  The adjoint needs only g, so it runs while c is
// still arriving; the copies run on the plan's own stream, each as soon as its data is
// ready (A^H g leaves during the forward, f during dL/dx), and the caller's stream waits
// for the last one.
template <typename T>
int step_host(nufft_plan p, const void *c_h, const void *g_h, void *f_h, void *gc_h, void *gx_h, cudaStream_t s) {
    const size_t cxs = 2 * sizeof(T);
    if (!p->st_g || !p->st_copy) return NUFFT_ESTATE;   // nufft2_plan_reserve makes the buffers
    cudaStream_t cs = p->st_copy;
    cudaEvent_t *ev = p->st_ev;   // 0 start / gx ready, 1 g in, 2 c in, 3 A^H g ready, 4 f ready, 5 all out
    // c goes up first and the forward starts as soon as it is in, while g follows; f and
    // gx come down while the adjoint runs, so that only the first upload and A^H g's
    // download stay outside the kernels' time
    NUFFT_CUDA_TRY(cudaEventRecord(ev[0], s));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(cs, ev[0], 0));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(p->cstage, c_h, (size_t)p->N * cxs, cudaMemcpyHostToDevice, cs));
    NUFFT_CUDA_TRY(cudaEventRecord(ev[2], cs));
    if (p->M > 0) NUFFT_CUDA_TRY(cudaMemcpyAsync(p->st_g, g_h, (size_t)p->M * cxs, cudaMemcpyHostToDevice, cs));
    NUFFT_CUDA_TRY(cudaEventRecord(ev[1], cs));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(s, ev[2], 0));
    if (int rc = exec_deriv<T>(p, p->cstage, p->fstage, p->st_fp, s)) return rc;
    NUFFT_CUDA_TRY(cudaEventRecord(ev[4], s));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(s, ev[1], 0));
    if (int rc = exec_grad_x<T>(p, p->st_g, p->st_fp, p->st_gx, 0, s)) return rc;
    NUFFT_CUDA_TRY(cudaEventRecord(ev[0], s));   // gx ready
    if (int rc = exec_adjoint<T>(p, p->st_g, p->st_gc, s)) return rc;
    NUFFT_CUDA_TRY(cudaEventRecord(ev[3], s));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(cs, ev[4], 0));
    if (p->M > 0) NUFFT_CUDA_TRY(cudaMemcpyAsync(f_h, p->fstage, (size_t)p->M * cxs, cudaMemcpyDeviceToHost, cs));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(cs, ev[0], 0));
    if (p->M > 0) NUFFT_CUDA_TRY(cudaMemcpyAsync(gx_h, p->st_gx, (size_t)p->M * sizeof(T), cudaMemcpyDeviceToHost, cs));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(cs, ev[3], 0));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(gc_h, p->st_gc, (size_t)p->N * cxs, cudaMemcpyDeviceToHost, cs));
    NUFFT_CUDA_TRY(cudaEventRecord(ev[5], cs));
    NUFFT_CUDA_TRY(cudaStreamWaitEvent(s, ev[5], 0));
    return NUFFT_OK;
}

}  // namespace

// nufft2_step_host's device copies of g, f', A^H g and gx, its copy stream and events
// (once per plan; part of nufft2_plan_reserve, the plan stage).
int reserve_step_host(nufft_plan p, cudaStream_t s) {
    if (p->st_g && p->st_copy) return NUFFT_OK;
    const size_t rs = p->prec == NUFFT_F32 ? 4 : 8, cxs = 2 * rs, Mi = (size_t)std::max<int64_t>(p->M, 1);
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (!p->st_g) NUFFT_CUDA_TRY(dev_malloc(&p->st_g, Mi * cxs));
    if (!p->st_fp) NUFFT_CUDA_TRY(dev_malloc(&p->st_fp, Mi * cxs));
    if (!p->st_gc) NUFFT_CUDA_TRY(dev_malloc(&p->st_gc, (size_t)p->N * cxs));
    if (!p->st_gx) NUFFT_CUDA_TRY(dev_malloc(&p->st_gx, Mi * rs));
    for (cudaEvent_t &e : p->st_ev)
        if (!e) NUFFT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    NUFFT_CUDA_TRY(cudaStreamCreateWithFlags(&p->st_copy, cudaStreamNonBlocking));   // last: marks it complete
    p->work_bytes += (int64_t)(Mi * (2 * cxs + rs) + (size_t)p->N * cxs);
    return NUFFT_OK;
}

}  // namespace nufft

extern "C" int nufft2_step_host(nufft_plan p, const void *c_host, const void *g_host, void *f_host, void *gc_host,
                                void *gx_host, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_step_host");
    if (!p || !c_host || !gc_host || (p->M > 0 && (!g_host || !f_host || !gx_host))) return NUFFT_EINVAL;
    if (p->dims == 2) return NUFFT_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NUFFT_F32 ? nufft::step_host<float>(p, c_host, g_host, f_host, gc_host, gx_host, s)
                                : nufft::step_host<double>(p, c_host, g_host, f_host, gc_host, gx_host, s);
}
