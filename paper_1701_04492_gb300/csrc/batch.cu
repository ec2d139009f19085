// batch.cu -- many independent NUFFT-II problems of uneven sizes in few launches.
//
// Each problem has its own plan (rounding, rank, sort, tables: section 2.3's
// planning stage, one per problem).  Problems whose grids have the same length L and
// four-step split and whose ranks share a rank bound KM form a class; one launch per pass then covers a
// whole class (blockIdx.z = the problem), reading each problem's arguments from a
// device array built here once.  Batched launches exist for FP32 problems on grids
// of up to 2^18 points; a larger problem fills the GPU alone, and an FP64 problem
// (or any problem with NUFFT_BATCH_PER_PROBLEM) runs with its own plan's launches,
// a class of its own.  Inputs and outputs are packed: problem i's coefficients
// start at sum_{j<i} N_j, its samples at sum_{j<i} M_j.
//
// With NUFFT_BATCH_GRAPH, a call whose pointers equal the previous call's replays a
// CUDA graph of all launches, each class a parallel branch; the graph is captured on
// the first such call (the eager call before it has set every kernel attribute).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "fill.cuh"
#include "passes.cuh"
#include "persist.cuh"
#include "nvtx_range.h"

namespace nufft {
NUFFT_DECLARE_COLS_MANY()
NUFFT_DECLARE_MANY(4)
NUFFT_DECLARE_MANY(8)
NUFFT_DECLARE_MANY(12)
NUFFT_DECLARE_MANY(16)
}  // namespace nufft

struct nufft_batch_s {
    struct Class {
        int64_t L = 0;
        int KM = 0;
        int lg1 = 0;            // the four-step split (log2 of the row length)
        int C1 = 0;             // pass 1's columns per CTA
        bool single = false;    // one large problem: its own plan's launches
        std::vector<int> idx;   // members (problem indices)
        int rep = -1;           // member whose launch geometry covers the class
        int ny1 = 1, nyB = 1;   // grid.y of pass 1 (largest K) and pass B (largest split)
        void *a1 = nullptr, *a2 = nullptr, *aA = nullptr, *aB = nullptr, *betas = nullptr;
        cudaStream_t st = nullptr;   // its branch while a graph is captured
        cudaEvent_t done = nullptr;
    };
    int prec = 0;
    unsigned flags = 0;
    std::vector<nufft_plan> plans;
    std::vector<int64_t> offN, offM;   // count + 1 prefix sums
    std::vector<Class> cls;
    // graph state, [0] forward, [1] adjoint
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    const void *gin[2] = {nullptr, nullptr};
    void *gout[2] = {nullptr, nullptr};
    const void *lastin[2] = {nullptr, nullptr};
    void *lastout[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    // NUFFT_BATCH_PERSISTENT: every batched class of a direction in one persistent launch
    // ([0] forward, [1] adjoint): its device state, grid and shared memory
    bool persist = false;
    nufft::PState pst[2] = {};
    int pgrid[2] = {0, 0};
    size_t psmem[2] = {0, 0};
    std::vector<void *> pbufs;   // device allocations of the persistent state
};

namespace nufft {
namespace {

void free_batch(nufft_batch b) {
    if (!b) return;
    for (auto &c : b->cls) {
        for (void *q : {c.a1, c.a2, c.aA, c.aB, c.betas})
            if (q) cudaFree(q);
        if (c.st) cudaStreamDestroy(c.st);
        if (c.done) cudaEventDestroy(c.done);
    }
    for (cudaGraphExec_t g : b->gexec)
        if (g) cudaGraphExecDestroy(g);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    for (void *q : b->pbufs)
        if (q) cudaFree(q);
    for (nufft_plan p : b->plans)
        if (p) nufft_destroy(p);
    delete b;
}

template <typename V>
int upload(void **dst, const std::vector<V> &h) {
    NUFFT_CUDA_TRY(dev_malloc((void **)dst, h.size() * sizeof(V)));
    NUFFT_CUDA_TRY(cudaMemcpy(*dst, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return NUFFT_OK;
}

// The four argument arrays and the coefficient tables of one class.
template <typename T, int KM>
int build_class(nufft_batch b, nufft_batch_s::Class &c) {
    std::vector<PassArgs<T>> v1, v2, vA, vB;
    std::vector<Beta<T, KM>> be;
    // pass B's rank split for the class: about one CTA per SM over all its problems (as
    // for a single plan), at most any member's own split (whose partial-sum buffer it uses)
    nufft_plan r = b->plans[c.rep];
    const int blocks = (int)(r->L1 / r->CB) * (int)c.idx.size();
    int sb = (device_sm_count() + blocks - 1) / blocks;
    for (int i : c.idx) sb = std::min(sb, b->plans[i]->SBsplit);
    sb = std::max(1, sb);
    c.nyB = sb;
    for (int i : c.idx) {
        nufft_plan p = b->plans[i];
        const PassArgs<T> a = base_args<T>(p);
        PassArgs<T> x1 = a, x2 = a, xA = a, xB = a;
        cols_fields<T>(p, x1, false);
        if (int rc = rows_fields<T>(p, x2, false)) return rc;
        if (int rc = rows_fields<T>(p, xA, true)) return rc;
        cols_fields<T>(p, xB, true);
        xB.SB = sb;
        // forward: in = c, out = f; adjoint: in = g, out = c
        x1.in_off = x2.in_off = b->offN[i];
        x1.out_off = x2.out_off = b->offM[i];
        xA.in_off = xB.in_off = b->offM[i];
        xA.out_off = xB.out_off = b->offN[i];
        v1.push_back(x1);
        v2.push_back(x2);
        vA.push_back(xA);
        vB.push_back(xB);
        be.push_back(beta_of<T, KM>(p));
        c.ny1 = std::max(c.ny1, p->K);
    }
    if (int rc = upload(&c.a1, v1)) return rc;
    if (int rc = upload(&c.a2, v2)) return rc;
    if (int rc = upload(&c.aA, vA)) return rc;
    if (int rc = upload(&c.aB, vB)) return rc;
    return upload(&c.betas, be);
}

int build_class_f32(nufft_batch b, nufft_batch_s::Class &c) {
    switch (c.KM) {
        case 4: return build_class<float, 4>(b, c);
        case 8: return build_class<float, 8>(b, c);
        case 12: return build_class<float, 12>(b, c);
        case 16: return build_class<float, 16>(b, c);
        default: return NUFFT_EUNSUPPORTED;
    }
}

int rows_many(const nufft_batch_s::Class &c, nufft_plan rep, const void *args, bool adjoint,
              const void *in, void *out, cudaStream_t s) {
    using T = float;
    const int n = (int)c.idx.size();
    const PassArgs<T> *a = (const PassArgs<T> *)args;
    const ManyIO io{in, out, nullptr, 0, 0};   // the problems' offsets are in their arguments
    switch (c.KM) {
        case 4: return launch_rows_many<T, 4>(rep, a, (const Beta<T, 4> *)c.betas, n, adjoint, io, s);
        case 8: return launch_rows_many<T, 8>(rep, a, (const Beta<T, 8> *)c.betas, n, adjoint, io, s);
        case 12: return launch_rows_many<T, 12>(rep, a, (const Beta<T, 12> *)c.betas, n, adjoint, io, s);
        case 16: return launch_rows_many<T, 16>(rep, a, (const Beta<T, 16> *)c.betas, n, adjoint, io, s);
        default: return NUFFT_EUNSUPPORTED;
    }
}

// The launches of one class, in order, on stream s: two batched launches, or a
// single problem's own exec call.
template <typename T>
int class_launches(nufft_batch b, const nufft_batch_s::Class &c, bool adjoint, const void *in,
                   void *out, cudaStream_t s) {
    nufft_plan rep = b->plans[c.rep];
    const int n = (int)c.idx.size();
    if (c.single) {
        const size_t cxs = 2 * sizeof(T);
        const int i = c.idx[0];
        const char *src = (const char *)in + (size_t)(adjoint ? b->offM[i] : b->offN[i]) * cxs;
        char *dst = (char *)out + (size_t)(adjoint ? b->offN[i] : b->offM[i]) * cxs;
        return adjoint ? nufft1_exec(rep, src, dst, s) : nufft2_exec(rep, src, dst, s);
    }
    if constexpr (std::is_same<T, float>::value) {
        const ManyIO io{in, out, nullptr, 0, 0};
        if (!adjoint) {
            if (int rc = launch_cols_many<T>(rep, (const PassArgs<T> *)c.a1, n, c.ny1, false, io, s)) return rc;
            return rows_many(c, rep, c.a2, false, in, out, s);
        }
        if (int rc = rows_many(c, rep, c.aA, true, in, out, s)) return rc;
        return launch_cols_many<T>(rep, (const PassArgs<T> *)c.aB, n, c.nyB, true, io, s);
    } else {
        return NUFFT_EUNSUPPORTED;   // FP64 classes are single problems
    }
}

// The persistent launch of one direction (every batched class), if the batch has one.
int persistent_launch(nufft_batch b, bool adjoint, const void *in, void *out, cudaStream_t s) {
    const int dir = adjoint ? 1 : 0;
    if (!b->persist || b->pst[dir].n_items == 0) return NUFFT_OK;
    return launch_persistent(dir, b->pst[dir], b->pgrid[dir], b->psmem[dir], ManyIO{in, out, nullptr, 0, 0}, s);
}

template <typename T>
int launch_all(nufft_batch b, bool adjoint, const void *in, void *out, cudaStream_t s) {
    for (const auto &c : b->cls) {
        if (b->persist && !c.single) continue;   // in the persistent launch
        if (int rc = class_launches<T>(b, c, adjoint, in, out, s)) return rc;
    }
    return persistent_launch(b, adjoint, in, out, s);
}

// Capture every class as a parallel branch of one graph (fork from b->cap, join back).
template <typename T>
int capture(nufft_batch b, int dir, const void *in, void *out) {
    if (b->gexec[dir]) {
        cudaGraphExecDestroy(b->gexec[dir]);
        b->gexec[dir] = nullptr;
    }
    NUFFT_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = NUFFT_OK;
    if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) rc = NUFFT_ECUDA;
    for (auto &c : b->cls) {
        if (rc) break;
        if (b->persist && !c.single) continue;   // in the persistent launch, below
        if (cudaStreamWaitEvent(c.st, b->fork, 0) != cudaSuccess) { rc = NUFFT_ECUDA; break; }
        rc = class_launches<T>(b, c, dir == 1, in, out, c.st);
        if (!rc && (cudaEventRecord(c.done, c.st) != cudaSuccess ||
                    cudaStreamWaitEvent(b->cap, c.done, 0) != cudaSuccess))
            rc = NUFFT_ECUDA;
    }
    if (!rc) rc = persistent_launch(b, dir == 1, in, out, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (!rc && e != cudaSuccess) rc = NUFFT_ECUDA;
    if (!rc && cudaGraphInstantiate(&b->gexec[dir], g, 0) != cudaSuccess) {
        b->gexec[dir] = nullptr;
        rc = NUFFT_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    if (rc) (void)cudaGetLastError();
    b->gin[dir] = in;
    b->gout[dir] = out;
    return rc;
}

template <typename T>
int exec_many(nufft_batch b, bool adjoint, const void *in, void *out, cudaStream_t s) {
    const int dir = adjoint ? 1 : 0;
    if (b->flags & NUFFT_BATCH_GRAPH) {
        if (b->gexec[dir] && b->gin[dir] == in && b->gout[dir] == out) {
            NUFFT_CUDA_TRY(cudaGraphLaunch(b->gexec[dir], s));
            return NUFFT_OK;
        }
        if (b->lastin[dir] == in && b->lastout[dir] == out) {   // second call: capture
            if (int rc = capture<T>(b, dir, in, out)) return rc;
            NUFFT_CUDA_TRY(cudaGraphLaunch(b->gexec[dir], s));
            return NUFFT_OK;
        }
    }
    b->lastin[dir] = in;
    b->lastout[dir] = out;
    return launch_all<T>(b, adjoint, in, out, s);
}

}  // namespace
}  // namespace nufft

using nufft::free_batch;

namespace nufft {
namespace {

// The persistent kernel's CTAs (128 registers, 256 threads) fit two per SM only with at most
// this much shared memory each; its dynamic shared memory is the largest any item needs, so
// the row passes' rank groups and pass 1's columns per CTA are re-chosen to stay within it.
constexpr size_t PERSIST_SMEM_CAP = 110 * 1024;

// Pass A's arguments and shared memory in a CTA of 256 threads (the persistent kernel):
// 256 / TT teams, each with its four-step table, and the largest rank group that fits.
PassArgs<float> passA_persistent(nufft_plan p, size_t *smem) {
    PassArgs<float> a = base_args<float>(p);
    (void)rows_fields<float>(p, a, true);
    const int E = std::min<int>(EmaxT<float, PK_ROW_ADJ>::v, p->L1), TT = p->L1 / E, nt = 256 / TT;
    const size_t staging = (size_t)p->chunkA * (sizeof(int32_t) + sizeof(float)) + (size_t)p->chunkA * 8;
    auto bytes = [&](int G) { return ((size_t)G * p->B2 * p->SA + (size_t)nt * E) * 8 + staging; };
    int G = p->GA;
    while (G > 1 && bytes(G) > PERSIST_SMEM_CAP) --G;
    a.G = G;
    *smem = bytes(G);
    return a;
}

// Pass 1's arguments with its columns per CTA halved until its slots and four-step table
// stay within PERSIST_SMEM_CAP (a class launch may take more shared memory, and run one
// CTA per SM, but the persistent kernel's size is every item's); with fewer columns the
// extra threads of the 256-thread CTA shadow roles.  The slot stride is kept.
PassArgs<float> pass1_persistent(nufft_plan p, size_t *smem) {
    PassArgs<float> a = base_args<float>(p);
    cols_fields<float>(p, a, false);
    const size_t E2 = (size_t)std::min<int>(EmaxT<float, PK_COL_FWD>::v, p->L2);
    auto bytes = [&](int C) { return ((size_t)C * a.S + (size_t)C * E2) * sizeof(float2); };
    while (a.C > 1 && bytes(a.C) > PERSIST_SMEM_CAP) {
        a.C /= 2;
        --a.lgC;
    }
    *smem = bytes(a.C);
    return a;
}

// Pass 2's arguments with its rank group re-chosen to stay within PERSIST_SMEM_CAP (its
// slots, then one mbarrier per slot); a group smaller than K keeps partial sums in fscr.
PassArgs<float> pass2_persistent(nufft_plan p, size_t *smem) {
    PassArgs<float> a = base_args<float>(p);
    (void)rows_fields<float>(p, a, false);
    auto body = [&](int G) { return ((size_t)G * p->B2 * p->S2 * 8 + 15) / 16 * 16; };
    auto bytes = [&](int G) { return body(G) + (size_t)G * p->B2 * sizeof(uint64_t); };
    int G = std::min(p->G, p->K);   // the plain forward stages K ranks
    while (G > 1 && bytes(G) > PERSIST_SMEM_CAP) --G;
    a.G = G;
    a.mbar_off = (int)body(G);
    *smem = bytes(G);
    return a;
}

template <typename D, typename V>
int upload_persist(nufft_batch b, D **dst, const std::vector<V> &h) {
    void *q = nullptr;
    NUFFT_CUDA_TRY(dev_malloc(&q, std::max<size_t>(1, h.size()) * sizeof(V)));
    b->pbufs.push_back(q);
    if (!h.empty()) NUFFT_CUDA_TRY(cudaMemcpy(q, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    *dst = (D *)q;
    return NUFFT_OK;
}

// The persistent launches' state (NUFFT_BATCH_PERSISTENT): per direction, the class table
// (the class launches' argument arrays; pass A's rebuilt for 256-thread CTAs), the work
// items -- every first-pass block of every problem, largest problems first, then every
// second-pass block in the same order -- the first-pass counts each problem's second pass
// waits for, the coefficients as 16 x 16 tables, the counters, and the grid (the CTAs
// that fit on the device at once).
int build_persistent(nufft_batch b) {
    const int nprob = (int)b->plans.size();
    std::vector<Beta<float, 16>> be((size_t)nprob);
    for (int i = 0; i < nprob; ++i)
        for (int r = 0; r < 16; ++r)
            for (int q = 0; q < 16; ++q) be[i].b[r][q] = (float)b->plans[i]->beta[r][q];
    const Beta<float, 16> *dbe = nullptr;
    if (int rc = upload_persist(b, &dbe, be)) return rc;
    int *done = nullptr, *ctl = nullptr;
    if (int rc = upload_persist(b, &done, std::vector<int>((size_t)nprob, 0))) return rc;
    if (int rc = upload_persist(b, &ctl, std::vector<int>(4, 0))) return rc;
    int dev = 0, sms = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    NUFFT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // problems of batched classes, largest grid first (they take longest)
    std::vector<std::pair<int, int>> order;   // (class, member)
    for (int c = 0; c < (int)b->cls.size(); ++c)
        if (!b->cls[c].single)
            for (int m = 0; m < (int)b->cls[c].idx.size(); ++m) order.push_back({c, m});
    std::stable_sort(order.begin(), order.end(), [&](const std::pair<int, int> &u, const std::pair<int, int> &v) {
        return b->cls[u.first].L > b->cls[v.first].L;
    });
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<PClass> pc(b->cls.size());
        std::vector<int> c1(b->cls.size(), 1);   // pass 1's columns per CTA, per class
        std::vector<PItem> first, second;
        std::vector<int> need((size_t)nprob, 0);
        size_t smem = 0;
        for (int c = 0; c < (int)b->cls.size(); ++c) {
            auto &cl = b->cls[c];
            if (cl.single) continue;
            nufft_plan r = b->plans[cl.rep];
            pc[c].P_rows = r->L1;
            pc[c].P_cols = r->L2;
            pc[c].km = cl.KM <= 8 ? 8 : cl.KM <= 12 ? 12 : 16;
            if (dir == 0) {
                std::vector<PassArgs<float>> v1, v2;
                for (int i : cl.idx) {
                    size_t sm = 0;
                    PassArgs<float> a = pass1_persistent(b->plans[i], &sm);
                    a.in_off = b->offN[i];
                    a.out_off = b->offM[i];
                    v1.push_back(a);
                    smem = std::max(smem, sm);
                    a = pass2_persistent(b->plans[i], &sm);
                    a.in_off = b->offN[i];
                    a.out_off = b->offM[i];
                    v2.push_back(a);
                    smem = std::max(smem, sm);
                }
                const PassArgs<float> *d1 = nullptr, *d2 = nullptr;
                if (int rc = upload_persist(b, &d1, v1)) return rc;
                if (int rc = upload_persist(b, &d2, v2)) return rc;
                pc[c].args[0] = d1;
                pc[c].args[1] = d2;
                c1[c] = v1.empty() ? r->C1 : v1[0].C;
            } else {
                std::vector<PassArgs<float>> vA;
                for (int i : cl.idx) {
                    size_t sm = 0;
                    PassArgs<float> a = passA_persistent(b->plans[i], &sm);
                    a.in_off = b->offM[i];
                    a.out_off = b->offN[i];
                    vA.push_back(a);
                    smem = std::max(smem, sm);
                }
                const PassArgs<float> *dA = nullptr;
                if (int rc = upload_persist(b, &dA, vA)) return rc;
                pc[c].args[0] = dA;
                pc[c].args[1] = (const PassArgs<float> *)cl.aB;
                smem = std::max(smem, r->smemB);
            }
        }
        // a row of nbx blocks in items of up to `per` consecutive blocks: problems with many
        // blocks take several per item, so that the per-item work (the ticket, the arguments,
        // the barriers) is a small part of it
        auto add_row = [&](std::vector<PItem> &v, int kind, const std::pair<int, int> &cm, int i, int nbx, int by) {
            const int per = nbx >= 256 ? 4 : nbx >= 64 ? 2 : 1;
            for (int bx = 0; bx < nbx; bx += per)
                v.push_back(PItem{kind, cm.first, cm.second, i, bx, by, std::min(per, nbx - bx)});
        };
        for (const auto &cm : order) {
            const auto &cl = b->cls[cm.first];
            const int i = cl.idx[cm.second];
            nufft_plan p = b->plans[i];
            if (p->M == 0 && dir == 0) continue;   // nothing to transform (its f is empty)
            if (dir == 0) {
                const int nbx = p->L1 / c1[cm.first];
                for (int by = 0; by < p->K; ++by) add_row(first, 0, cm, i, nbx, by);
                need[i] = nbx * p->K;
                add_row(second, 1, cm, i, p->NB, 0);
            } else {
                add_row(first, 0, cm, i, p->NB, 0);
                need[i] = p->NB;
                for (int by = 0; by < cl.nyB; ++by) add_row(second, 1, cm, i, p->L1 / p->CB, by);
            }
        }
        first.insert(first.end(), second.begin(), second.end());
        PState &st = b->pst[dir];
        if (int rc = upload_persist(b, &st.items, first)) return rc;
        const PClass *dpc = nullptr;
        if (int rc = upload_persist(b, &dpc, pc)) return rc;
        const int *dneed = nullptr;
        if (int rc = upload_persist(b, &dneed, need)) return rc;
        st.n_items = (int)first.size();
        st.classes = dpc;
        st.betas = dbe;
        st.done = done;
        st.need = dneed;
        st.ctl = ctl + 2 * dir;
        st.nprob = nprob;
        b->psmem[dir] = smem;
        int per_sm = 0;
        if (int rc = persistent_blocks_per_sm(dir, smem, &per_sm)) return rc;
        if (per_sm < 1) return NUFFT_EUNSUPPORTED;
        b->pgrid[dir] = per_sm * sms;
    }
    b->persist = true;
    return NUFFT_OK;
}

// A batch from per-problem inputs: sample pointers xs[i], layouts lays (or NULL: each
// problem's default).  flags may hold NUFFT_PLAN_AUTOTUNE for the problems' own plans.
// Inputs are validated by the caller.
int plan_many_core(nufft_batch *out, int64_t count, const int64_t *N_host, const int64_t *M_host,
                   const Layout *lays, const double *const *xs, const double *eps_host, int prec, unsigned flags,
                   void *stream) {
    *out = nullptr;
    nufft_batch b = new (std::nothrow) nufft_batch_s();
    if (!b) return NUFFT_ENOMEM;
    b->prec = prec;
    b->flags = flags;
    b->plans.assign((size_t)count, nullptr);
    b->offN.assign((size_t)count + 1, 0);
    b->offM.assign((size_t)count + 1, 0);
    for (int64_t i = 0; i < count; ++i) {
        b->offN[i + 1] = b->offN[i] + N_host[i];
        b->offM[i + 1] = b->offM[i] + M_host[i];
    }
    for (int64_t i = 0; i < count; ++i) {
        const int rc = plan_layout(&b->plans[i], N_host[i], M_host[i], xs[i], eps_host[i], prec,
                                   lays ? lays[i] : Layout{}, flags & NUFFT_PLAN_AUTOTUNE, (cudaStream_t)stream);
        if (rc) { free_batch(b); return rc; }
    }
    // classes: same L and rank bound; the representative has the largest K
    for (int64_t i = 0; i < count; ++i) {
        nufft_plan p = b->plans[i];
        const bool single = prec == NUFFT_F64 || (flags & NUFFT_BATCH_PER_PROBLEM) ||
                            std::max(p->L1, p->L2) > MANY_P_MAX;
        auto it = std::find_if(b->cls.begin(), b->cls.end(), [&](const nufft_batch_s::Class &c) {
            return !single && !c.single && c.L == p->L && c.KM == p->kmax && c.lg1 == p->lg1 && c.C1 == p->C1;
        });
        if (it == b->cls.end()) {
            b->cls.emplace_back();
            it = b->cls.end() - 1;
            it->L = p->L;
            it->KM = p->kmax;
            it->lg1 = p->lg1;
            it->C1 = p->C1;
            it->single = single;
        }
        it->idx.push_back((int)i);
        if (it->rep < 0 || b->plans[it->rep]->K < p->K) it->rep = (int)i;
    }
    // every member must fit the representative's shared-memory layouts (pass 2: its
    // own slots and mbarriers; pass A: its slots plus the launch's team tables);
    // a member that does not becomes a class of its own
    std::vector<nufft_batch_s::Class> own_classes;
    for (auto &c : b->cls) {
        if (c.single) continue;
        nufft_plan r = b->plans[c.rep];
        const size_t E1 = (size_t)std::min<int>(EmaxT<float, PK_ROW_ADJ>::v, r->L1);   // pass A's tables
        for (size_t q = 0; q < c.idx.size();) {
            nufft_plan m = b->plans[c.idx[q]];
            const size_t needA = m->smemA + (size_t)std::max(0, r->ntA - m->ntA) * E1 * 8;
            if (m->smem2 <= r->smem2 && needA <= r->smemA && m->smem1 <= r->smem1 && m->smemB <= r->smemB) {
                ++q;
                continue;
            }
            nufft_batch_s::Class own;
            own.L = m->L;
            own.KM = m->kmax;
            own.single = true;
            own.idx.push_back(c.idx[q]);
            own.rep = c.idx[q];
            c.idx.erase(c.idx.begin() + (long)q);
            own_classes.push_back(own);
        }
    }
    b->cls.insert(b->cls.end(), own_classes.begin(), own_classes.end());
    for (auto &c : b->cls) {
        const int rc = c.single ? NUFFT_OK : build_class_f32(b, c);
        if (rc) { free_batch(b); return rc; }
        if (flags & NUFFT_BATCH_GRAPH) {
            if (cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) {
                (void)cudaGetLastError();
                free_batch(b);
                return NUFFT_ECUDA;
            }
        }
    }
    if (flags & NUFFT_BATCH_GRAPH) {
        if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            free_batch(b);
            return NUFFT_ECUDA;
        }
    }
    if (flags & NUFFT_BATCH_PERSISTENT) {
        if (int rc = build_persistent(b)) {
            free_batch(b);
            return rc;
        }
    }
    *out = b;
    return NUFFT_OK;
}

// Device time (ms) of one forward and one adjoint of the whole batch on scratch
// buffers c (sum N) and f (sum M) holding hash values, L2 flushed before each run:
// the best of three after a warm-up.
int time_batch(nufft_batch b, void *c, void *f, void *flush, cudaStream_t s, float *ms) {
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
        rc = exec_many<float>(b, false, c, f, s);
        if (!rc) rc = exec_many<float>(b, true, f, c, s);
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
    if (!rc) rc = nufft_batch_check(b, s);
    *ms = best;
    return rc;
}

// The batch autotuner (FP32 batched launches).  What a layout costs in a batch is its
// share of a full GPU, not its latency alone, so layouts are compared class by class
// on the batched launches themselves: for each class of the default layout (grid L0,
// rows the longer FFT), its members are planned again on the oversampled grid 2 L0
// (section 2.3: a longer grid lowers gamma and so K) and with the other four-step
// split where log2 L is odd, each candidate batch is timed (forward + adjoint), and
// the fastest layout is kept for those members.  Timed alone, a class measures what
// it costs when classes run one after another; in a graph they overlap, so the batch
// with the chosen layouts is then timed as a whole (graph or direct launches, as the
// batch will run) against the default batch, and the faster batch is kept.
int tune_many(nufft_batch *out, int64_t count, const int64_t *N, const int64_t *M, const double *const *xs,
              const double *eps, unsigned flags, cudaStream_t s) {
    nufft_batch b0 = nullptr;
    if (int rc = plan_many_core(&b0, count, N, M, nullptr, xs, eps, NUFFT_F32, flags, s)) return rc;
    std::vector<Layout> lay((size_t)count);
    for (int64_t i = 0; i < count; ++i) lay[i].L = b0->plans[i]->L;
    void *c = nullptr, *f = nullptr, *flush = nullptr;
    const size_t cn = (size_t)std::max<int64_t>(b0->offN.back(), 1), fm = (size_t)std::max<int64_t>(b0->offM.back(), 1);
    int rc = NUFFT_OK;
    if (dev_malloc((void **)&c, cn * 8) != cudaSuccess || dev_malloc((void **)&f, fm * 8) != cudaSuccess ||
        dev_malloc((void **)&flush, L2_FLUSH_BYTES) != cudaSuccess ||
        fill_hash<float>(c, 2 * (int64_t)cn, s) != cudaSuccess || fill_hash<float>(f, 2 * (int64_t)fm, s) != cudaSuccess)
        rc = NUFFT_ECUDA;
    bool changed = false;
    const int64_t L_max_batched = (int64_t)MANY_P_MAX * MANY_P_MAX;
    for (size_t k = 0; k < b0->cls.size() && !rc; ++k) {
        const auto &cl = b0->cls[k];
        if (cl.single) continue;
        const size_t n = cl.idx.size();
        std::vector<int64_t> sN(n), sM(n);
        std::vector<const double *> sx(n);
        std::vector<double> se(n);
        for (size_t q = 0; q < n; ++q) {
            const int i = cl.idx[q];
            sN[q] = N[i]; sM[q] = M[i]; sx[q] = xs[i]; se[q] = eps[i];
        }
        float tbest = 1e30f;
        Layout best;
        best.L = cl.L;
        for (int64_t Lc = cl.L; Lc <= std::min<int64_t>(2 * cl.L, L_max_batched) && !rc; Lc *= 2) {
            int lg = 0;
            while (((int64_t)1 << lg) < Lc) ++lg;
            for (int lcc = 0; lcc < 2 && !rc; ++lcc)
                for (int c1s = 0; c1s < 2 && !rc; ++c1s) {
                    if (lcc == 1 && lg % 2 == 0) continue;
                    Layout cand;
                    cand.L = Lc;
                    cand.long_cols = lcc == 1;
                    cand.c1_shift = c1s;
                    std::vector<Layout> sl(n, cand);
                    nufft_batch t = nullptr;
                    int r2 = plan_many_core(&t, (int64_t)n, sN.data(), sM.data(), sl.data(), sx.data(), se.data(),
                                            NUFFT_F32, flags & ~NUFFT_BATCH_GRAPH, s);
                    if (r2 == NUFFT_EUNSUPPORTED || r2 == NUFFT_EINVAL) continue;
                    if (r2) { rc = r2; break; }
                    float ms = 0.f;
                    r2 = time_batch(t, c, f, flush, s, &ms);
                    free_batch(t);
                    if (r2) { rc = r2; break; }
                    // the default layout wins ties: a new layout must save 3 %
                    if (Lc == cl.L && lcc == 0 && c1s == 0) tbest = ms;
                    else if (ms < 0.97f * tbest) { tbest = ms; best = cand; }
                }
        }
        if (best.L != cl.L || best.long_cols || best.c1_shift) {
            changed = true;
            for (int i : cl.idx) lay[i] = best;
        }
    }
    nufft_batch b1 = nullptr;
    float t0 = 0.f, t1 = 0.f;
    if (!rc && changed) rc = plan_many_core(&b1, count, N, M, lay.data(), xs, eps, NUFFT_F32, flags, s);
    if (!rc && changed) rc = time_batch(b0, c, f, flush, s, &t0);
    if (!rc && changed) rc = time_batch(b1, c, f, flush, s, &t1);
    cudaFree(c);
    cudaFree(f);
    cudaFree(flush);
    if (rc) { free_batch(b0); free_batch(b1); return rc; }
    if (changed && t1 < t0) {
        free_batch(b0);
        *out = b1;
    } else {
        free_batch(b1);
        *out = b0;
    }
    return NUFFT_OK;
}

}  // namespace
}  // namespace nufft

extern "C" int nufft2_plan_many(nufft_batch *out, int64_t count, const int64_t *N_host,
                                const int64_t *M_host, const int64_t *L_host, const double *x_dev,
                                const double *eps_host, int prec, unsigned flags, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_plan_many");
    using namespace nufft;
    if (!out) return NUFFT_EINVAL;
    *out = nullptr;
    if (count < 1 || count > 65535 || !N_host || !M_host || !eps_host) return NUFFT_EINVAL;
    if (prec != NUFFT_F32 && prec != NUFFT_F64) return NUFFT_EINVAL;
    if (flags & ~(NUFFT_BATCH_GRAPH | NUFFT_BATCH_PER_PROBLEM | NUFFT_PLAN_AUTOTUNE | NUFFT_BATCH_PERSISTENT))
        return NUFFT_EINVAL;
    int64_t totM = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (M_host[i] < 0 || M_host[i] >= ((int64_t)1 << 31)) return NUFFT_EINVAL;
        totM += M_host[i];
    }
    if (totM > 0 && !x_dev) return NUFFT_EINVAL;
    std::vector<const double *> xs((size_t)count, nullptr);
    int64_t off = 0;
    for (int64_t i = 0; i < count; ++i) {
        xs[i] = M_host[i] > 0 ? x_dev + off : nullptr;
        off += M_host[i];
    }
    const bool batched = prec == NUFFT_F32 && !(flags & NUFFT_BATCH_PER_PROBLEM);
    bool L_free = true;   // no grid size fixed by the caller
    for (int64_t i = 0; L_host && i < count; ++i) L_free = L_free && L_host[i] == 0;
    if ((flags & NUFFT_PLAN_AUTOTUNE) && batched && L_free)
        return tune_many(out, count, N_host, M_host, xs.data(), eps_host, flags & ~NUFFT_PLAN_AUTOTUNE,
                         (cudaStream_t)stream);
    std::vector<Layout> lays;
    if (L_host) {
        lays.resize((size_t)count);
        for (int64_t i = 0; i < count; ++i) lays[i].L = L_host[i];
    }
    return plan_many_core(out, count, N_host, M_host, L_host ? lays.data() : nullptr, xs.data(), eps_host, prec, flags,
                          stream);
}

extern "C" int nufft_batch_info(nufft_batch b, int64_t *classes, int64_t *total_N, int64_t *total_M,
                                int *K_host, int64_t *L_host) {
    if (!b) return NUFFT_EINVAL;
    if (classes) *classes = (int64_t)b->cls.size();
    if (total_N) *total_N = b->offN.back();
    if (total_M) *total_M = b->offM.back();
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (K_host) K_host[i] = b->plans[i]->K;
        if (L_host) L_host[i] = b->plans[i]->L;
    }
    return NUFFT_OK;
}

extern "C" int nufft_batch_launches(nufft_batch b, int64_t *per_direction) {
    if (!b || !per_direction) return NUFFT_EINVAL;
    int64_t n = 0;
    for (const auto &c : b->cls) n += (b->persist && !c.single) ? 0 : 2;
    if (b->persist) n += 1;
    *per_direction = n;
    return NUFFT_OK;
}

extern "C" int nufft2_exec_many(nufft_batch b, const void *c_dev, void *f_dev, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_many");
    if (!b || !c_dev || (b->offM.back() > 0 && !f_dev)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return b->prec == NUFFT_F32 ? nufft::exec_many<float>(b, false, c_dev, f_dev, s)
                                : nufft::exec_many<double>(b, false, c_dev, f_dev, s);
}

extern "C" int nufft1_exec_many(nufft_batch b, const void *g_dev, void *c_dev, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft1_exec_many");
    if (!b || !c_dev || (b->offM.back() > 0 && !g_dev)) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return b->prec == NUFFT_F32 ? nufft::exec_many<float>(b, true, g_dev, c_dev, s)
                                : nufft::exec_many<double>(b, true, g_dev, c_dev, s);
}

extern "C" int nufft2_exec_each(nufft_batch b, const void *c_dev, void *f_dev, int adjoint, void *stream) {
    nufft::NvtxRange nvtx_range_("nufft2_exec_each");
    if (!b || !c_dev || (b->offM.back() > 0 && !f_dev)) return NUFFT_EINVAL;
    const size_t cxs = b->prec == NUFFT_F32 ? 8 : 16;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        const char *cb = (const char *)c_dev + (size_t)b->offN[i] * cxs;
        char *fb = (char *)f_dev + (size_t)b->offM[i] * cxs;
        const int rc = adjoint ? nufft1_exec(b->plans[i], fb, (void *)cb, stream)
                               : nufft2_exec(b->plans[i], cb, fb, stream);
        if (rc) return rc;
    }
    return NUFFT_OK;
}

extern "C" int nufft_batch_check(nufft_batch b, void *stream) {
    if (!b) return NUFFT_EINVAL;
    int worst = NUFFT_OK;
    for (nufft_plan p : b->plans) {
        const int rc = nufft2_check(p, stream);
        if (rc && !worst) worst = rc;
    }
    return worst;
}

extern "C" int nufft_batch_destroy(nufft_batch b) {
    free_batch(b);
    return NUFFT_OK;
}
