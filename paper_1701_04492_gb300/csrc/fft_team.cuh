// fft_team.cuh -- in-register DFTs and a Stockham FFT executed by a team of threads.
//
// A length-P transform (P a power of two, P <= E^3) is done by TT = P/E threads,
// each holding E complex values in registers.  Stage s applies radix R_s
// butterflies (R_0 = E, then E or the remainder); between stages the data moves
// through the team's shared-memory slot.  The formulation is the self-sorting
// (Stockham) one: virtual butterfly v of a stage with radix R, after NS points
// of sub-transforms, reads x[v + (P/R) i], multiplies input i by w_{NS R}^{i (v mod NS)}
// and writes output i to (v / NS) NS R + (v mod NS) + NS i.  Input and output are in
// natural order.
//
//   input layout : thread tt holds x[tt + TT m], m = 0..E-1      (strided by TT)
//   output layout: register e holds X[out_index(tt, e)]
//
// Every thread of the CTA (of the warp, for warp-contained teams) must call run() the same
// number of times (it synchronises between stages); teams with no work run on a scratch slot.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "dfloat.cuh"

namespace nufft {

// A complex double-word value: 16 bytes, so that it moves as one vector access.
struct __align__(16) cdf {
    dfloat x, y;
};

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<dfloat> { using type = cdf; };
template <typename T> using cx = typename CxT<T>::type;

// The types the caller's arrays hold for an element type T: complex64 / float for FP32,
// complex128 / double for FP64 and for the double-word kernels (which convert on load
// and on store).
template <typename T> struct IoT { using c = cx<T>; using r = T; };
template <> struct IoT<dfloat> { using c = double2; using r = double; };
template <typename T> using io_c = typename IoT<T>::c;
template <typename T> using io_r = typename IoT<T>::r;

// Read-only loads of complex values (16-byte double-word values as one vector load).
__device__ __forceinline__ float2 ldg_cx(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_cx(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ cdf ldg_cx(const cdf *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    cdf r;
    r.x = dfloat(v.x, v.y);
    r.y = dfloat(v.z, v.w);
    return r;
}
// Loads that bypass L1 (partial sums written by other CTAs of the same launch).
__device__ __forceinline__ float2 ldcg_cx(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg_cx(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ cdf ldcg_cx(const cdf *p) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    cdf r;
    r.x = dfloat(v.x, v.y);
    r.y = dfloat(v.z, v.w);
    return r;
}

template <typename T> __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// a * b
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
    return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// the double-word products as one dot2 per component
template <> __device__ __forceinline__ cdf cmul<dfloat>(cdf a, cdf b) {
    cdf r;
    r.x = dot2(a.x, b.x, -a.y, b.y);
    r.y = dot2(a.x, b.y, a.y, b.x);
    return r;
}
template <> __device__ __forceinline__ cdf cmulc<dfloat>(cdf a, cdf b) {
    cdf r;
    r.x = dot2(a.x, b.x, a.y, b.y);
    r.y = dot2(a.y, b.x, -a.x, b.y);
    return r;
}
// a * i^q  (q mod 4)
template <typename T> __device__ __forceinline__ cx<T> mul_ipow(cx<T> a, int q) {
    switch (q & 3) {
        case 0: return a;
        case 1: return mk<T>(-a.y, a.x);
        case 2: return mk<T>(-a.x, -a.y);
        default: return mk<T>(a.y, -a.x);
    }
}

// cos(2 pi m / 32) for m in [0, 8], from the half-angle values of pi/16.
__host__ __device__ constexpr double cos32_oct(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.98078528040323044912618223613424
         : m == 2 ? 0.92387953251128675612818318939679
         : m == 3 ? 0.83146961230254523707878837761791
         : m == 4 ? 0.70710678118654752440084436210485
         : m == 5 ? 0.55557023301960222474283081394853
         : m == 6 ? 0.38268343236508977172845998403040
         : m == 7 ? 0.19509032201612826784828486847702
                  : 0.0;
}
__host__ __device__ constexpr double cos32(int m) {
    return (m & 31) <= 8  ? cos32_oct(m & 31)
         : (m & 31) <= 16 ? -cos32_oct(16 - (m & 31))
         : (m & 31) <= 24 ? -cos32_oct((m & 31) - 16)
                          : cos32_oct(32 - (m & 31));
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// a * exp(-+ 2 pi i m / 32): forward (INV = false) uses the negative exponent.
template <bool INV, typename T>
__device__ __forceinline__ cx<T> mul_w32(cx<T> a, int m) {
    m &= 31;
    if (m == 0) return a;
    if (m == 16) return mk<T>(-a.x, -a.y);
    if (m == 8) return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
    if (m == 24) return INV ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
    const T c = (T)cos32(m);
    const T s = (T)(INV ? sin32(m) : -sin32(m));   // exp(i s') with s' = -+ angle
    if constexpr (std::is_same<T, dfloat>::value) {
        cdf r;
        r.x = dot2(c, a.x, -s, a.y);
        r.y = dot2(c, a.y, s, a.x);
        return r;
    }
    if (m == 4 || m == 12 || m == 20 || m == 28) {
        // |c| = |s| = 1/sqrt(2): (c a.x - s a.y, c a.y + s a.x) with shared products
        return mk<T>(c * a.x - s * a.y, c * a.y + s * a.x);
    }
    return mk<T>(fma(c, a.x, -s * a.y), fma(c, a.y, s * a.x));
}

__host__ __device__ constexpr int bitrev_c(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// f(std::integral_constant<int, i>) for i = 0..N-1, indices known to the compiler.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// In-place DFT of R points held in registers, natural order in and out:
// radix-2 decimation in time on the bit-reversed renaming of the inputs, fully
// unrolled, so at most R + 2 complex values are live.
template <int R, bool INV, typename T>
struct Dft {
    __device__ __forceinline__ static void run(cx<T> (&s)[R]) {
        constexpr int LG = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
        cx<T> t[R];
        static_for<R>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int j = bitrev_c(i, LG);
            t[i] = s[j];
        });
#pragma unroll
        for (int h = 1; h < R; h *= 2) {
#pragma unroll
            for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    const cx<T> a = t[g + k];
                    const cx<T> b = mul_w32<INV, T>(t[g + k + h], k * (16 / h));   // w_{2h}^k
                    t[g + k] = cadd<T>(a, b);
                    t[g + k + h] = csub<T>(a, b);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) s[i] = t[i];
    }
};

// The double-word DFT: the same radix-2 decimation in time, with the lazy double-word
// operations along its chains and one renormalisation of each output.
template <bool INV>
__device__ __forceinline__ cdf mul_w32_lazy(cdf a, int m) {
    m &= 31;
    if (m == 0) return a;
    cdf r;
    if (m == 16) { r.x = -a.x; r.y = -a.y; return r; }
    if (m == 8) { if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r; }
    if (m == 24) { if (INV) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; } return r; }
    const dfloat c(cos32(m));
    const dfloat sn(INV ? sin32(m) : -sin32(m));
    r.x = dot2_lazy(c, a.x, -sn, a.y);
    r.y = dot2_lazy(c, a.y, sn, a.x);
    return r;
}
template <int R, bool INV>
struct Dft<R, INV, dfloat> {
    __device__ __forceinline__ static void run(cdf (&s)[R]) {
        constexpr int LG = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
        cdf t[R];
        static_for<R>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int j = bitrev_c(i, LG);
            t[i] = s[j];
        });
#pragma unroll
        for (int h = 1; h < R; h *= 2) {
#pragma unroll
            for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    const cdf a = t[g + k];
                    const cdf b = mul_w32_lazy<INV>(t[g + k + h], k * (16 / h));
                    t[g + k].x = add_lazy(a.x, b.x);
                    t[g + k].y = add_lazy(a.y, b.y);
                    t[g + k + h].x = sub_lazy(a.x, b.x);
                    t[g + k + h].y = sub_lazy(a.y, b.y);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            s[i].x = renorm(t[i].x);
            s[i].y = renorm(t[i].y);
        }
    }
};

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// Shared-memory index with one pad element per E elements (bank-conflict relief).
template <int E> __device__ __forceinline__ int padi(int o) { return o + (o >> ilog2c(E)); }
template <int E> __host__ __device__ constexpr int padded_len(int P) { return P + P / E; }

// padi(base + STEP * i) = padi(base) + i (STEP + STEP / E) whenever STEP is a
// multiple of E (adding a multiple of E leaves the low bits of base alone), so a
// strided run of padded indices is one per-thread base plus compile-time offsets.
template <int E, int STEP>
__device__ __forceinline__ int padi_run(int pbase, int i) {
    if constexpr (STEP % E == 0) {
        return pbase + i * (STEP + STEP / E);
    } else {
        (void)pbase;
        return -1;   // not used: callers check STEP % E first
    }
}

// The passes, for the choice of their team FFT's values per thread E.
enum PassKind : int { PK_COL_FWD = 0, PK_ROW_FWD = 1, PK_ROW_ADJ = 2, PK_COL_ADJ = 3 };

// E per pass (the FFT length is P <= E^3; a team has P / E threads).  FP32: the row
// passes and the adjoint column pass take E = 16 (twice the threads, one more exchange),
// measured faster at 2^20 (pass 2 74 -> 68 us, pass A 101 -> 93 us, pass B 72 -> 64 us);
// pass 1 was faster with E = 32 (50 against 58 us).  FP64: E = 16.
template <typename T> struct EmaxBase;
template <> struct EmaxBase<float> {
    __host__ __device__ static constexpr int of(int kind) { return kind == PK_COL_FWD ? 32 : 16; }
};
template <> struct EmaxBase<double> {
    __host__ __device__ static constexpr int of(int) { return 16; }
};
template <> struct EmaxBase<dfloat> {
    __host__ __device__ static constexpr int of(int) { return 16; }
};
template <typename T, int KIND> struct EmaxT { static constexpr int v = EmaxBase<T>::of(KIND); };
template <typename T, int P, int KIND> __host__ __device__ constexpr int e_of() {
    return P < EmaxT<T, KIND>::v ? P : EmaxT<T, KIND>::v;
}

// The barrier between the stages of a team FFT.  WS: every team is a run of lanes inside
// one warp (row passes with at most 32 threads per team), so the warp's own barrier orders
// the team's shared-memory exchange; otherwise the whole CTA synchronises (column passes,
// whose teams are spread across warps, and teams of more than one warp).
template <bool WS>
__device__ __forceinline__ void team_sync() {
    if constexpr (WS) {
        // the lanes that exist in this warp (a CTA of, say, 240 threads ends in a half warp)
        const unsigned n = min(32u, blockDim.x - (threadIdx.x & ~31u));
        __syncwarp(n == 32u ? 0xffffffffu : (1u << n) - 1u);
    } else {
        __syncthreads();
    }
}

template <typename T, int P, int E, bool INV>
struct TeamFft {
    static_assert(P % E == 0, "P must be a multiple of E");
    static constexpr int TT = P / E;
    static constexpr int R0 = E;
    static constexpr int REM1 = TT;
    static constexpr int R1 = REM1 > E ? E : REM1;
    static constexpr int R2 = REM1 / R1;
    static_assert(R2 <= E, "P too large for E");
    static constexpr int RL = R2 > 1 ? R2 : (R1 > 1 ? R1 : R0);  // last radix
    static constexpr int NSL = P / RL;                            // sub-transform size before it

    // Output index of register e after run(): tt + TT q(e).
    __device__ __forceinline__ static int out_index(int tt, int e) {
        const int b = e / RL, i = e % RL;
        return tt + TT * b + NSL * i;
    }
    __host__ __device__ static constexpr int out_q(int e) { return e / RL + (E / RL) * (e % RL); }

    // Stage twiddles w_{NS R}^{i j} live in one table per FFT length, stage s >= 1
    // at offset TW_OFF_s, entry (i - 1) NS + j: lanes with consecutive j read
    // consecutive entries.
    static constexpr int TW_OFF1 = 0;
    static constexpr int TW_OFF2 = (R1 - 1) * R0;
    static constexpr int TW_SIZE = (R1 - 1) * R0 + (R2 > 1 ? (R2 - 1) * R0 * R1 : 0);

    template <int R, int NS, int OFF>
    __device__ __forceinline__ static void stage(cx<T> (&a)[E], int tt, const cx<T>* __restrict__ tw) {
#pragma unroll
        for (int b = 0; b < E / R; ++b) {
            cx<T> s[R];
#pragma unroll
            for (int i = 0; i < R; ++i) s[i] = a[b * R + i];
            if (NS > 1) {
                const int v = tt + TT * b;
                const int j = v & (NS - 1);
#pragma unroll
                for (int i = 1; i < R; ++i) {
                    const cx<T> w = ldg_cx(&tw[OFF + (i - 1) * NS + j]);
                    s[i] = INV ? cmulc<T>(s[i], w) : cmul<T>(s[i], w);
                }
            }
            Dft<R, INV, T>::run(s);
#pragma unroll
            for (int i = 0; i < R; ++i) a[b * R + i] = s[i];
        }
    }

    // A thread's stage twiddles depend only on its lane tt, not on the transform, so a
    // thread that runs several transforms can load them once into registers (Tw) and
    // reuse them: stage 1 (radix R1 after R0 points), then stage 2 (radix R2 after R0 R1).
    static constexpr int NW1 = R1 > 1 ? (E / R1) * (R1 - 1) : 0;
    static constexpr int NW2 = R2 > 1 ? (E / R2) * (R2 - 1) : 0;
    struct Tw {
        cx<T> w[NW1 + NW2 > 0 ? NW1 + NW2 : 1];
    };
    __device__ __forceinline__ static void load_tw(Tw& t, int tt, const cx<T>* __restrict__ tw) {
        if constexpr (R1 > 1) {
#pragma unroll
            for (int b = 0; b < E / R1; ++b) {
                const int j = (tt + TT * b) & (R0 - 1);
#pragma unroll
                for (int i = 1; i < R1; ++i) t.w[b * (R1 - 1) + i - 1] = ldg_cx(&tw[TW_OFF1 + (i - 1) * R0 + j]);
            }
        }
        if constexpr (R2 > 1) {
            constexpr int NS = R0 * R1;
#pragma unroll
            for (int b = 0; b < E / R2; ++b) {
                const int j = (tt + TT * b) & (NS - 1);
#pragma unroll
                for (int i = 1; i < R2; ++i) t.w[NW1 + b * (R2 - 1) + i - 1] = ldg_cx(&tw[TW_OFF2 + (i - 1) * NS + j]);
            }
        }
    }
    template <int R, int NS, int WOFF>
    __device__ __forceinline__ static void stage_reg(cx<T> (&a)[E], const Tw& t) {
#pragma unroll
        for (int b = 0; b < E / R; ++b) {
            cx<T> s[R];
#pragma unroll
            for (int i = 0; i < R; ++i) s[i] = a[b * R + i];
#pragma unroll
            for (int i = 1; i < R; ++i) {
                const cx<T> w = t.w[WOFF + b * (R - 1) + i - 1];
                s[i] = INV ? cmulc<T>(s[i], w) : cmul<T>(s[i], w);
            }
            Dft<R, INV, T>::run(s);
#pragma unroll
            for (int i = 0; i < R; ++i) a[b * R + i] = s[i];
        }
    }

    // Write the outputs of a stage (radix R after NS) to sm; read the inputs of the
    // next stage (radix Rn).
    // PRED: a round in which some teams are idle.  A thread with act = false (an idle
    // team) then only takes part in the barriers, so every thread meets the same
    // barriers.  Full rounds take PRED = false: stores guarded by a branch cost about a
    // quarter of a row pass's time, since the stage arithmetic can no longer be
    // scheduled around them.
    template <int R, int NS, int Rn, bool PRED, bool WS>
    __device__ __forceinline__ static void exchange(cx<T> (&a)[E], int tt, cx<T>* sm, bool act) {
        static_assert(NS == 1 || NS % E == 0, "later stages follow a radix-E stage");
#pragma unroll
        for (int b = 0; b < E / R; ++b) {
            const int v = tt + TT * b;
            if constexpr (NS == 1) {
                // first stage (R = E): o = v E + i, padded v (E + 1) + i
                static_assert(R == E, "the first stage has radix E");
                const int pb = v * (E + 1);
                if (!PRED || act) {
#pragma unroll
                    for (int i = 0; i < R; ++i) sm[pb + i] = a[b * R + i];
                }
            } else {
                const int o0 = (v / NS) * NS * R + (v % NS);
                const int pb = padi<E>(o0);
                if (!PRED || act) {
#pragma unroll
                    for (int i = 0; i < R; ++i) sm[padi_run<E, NS>(pb, i)] = a[b * R + i];
                }
            }
        }
        team_sync<WS>();
        constexpr int Vn = P / Rn;
        static_assert(Vn % E == 0, "exchange strides are multiples of E");
#pragma unroll
        for (int b = 0; b < E / Rn; ++b) {
            const int v = tt + TT * b;
            const int pb = padi<E>(v);
            // loads stay unconditional (an idle team reads its in-bounds slot and
            // discards the values), so independent loads can be scheduled around them
#pragma unroll
            for (int i = 0; i < Rn; ++i) a[b * Rn + i] = sm[padi_run<E, Vn>(pb, i)];
        }
        team_sync<WS>();
    }

    // Padded shared index of output e after run() (out_index(tt, e) padded).
    __device__ __forceinline__ static int out_padded(int tt, int e) {
        const int b = e / RL, i = e % RL;
        const int v = tt + TT * b;
        if constexpr (NSL % E == 0) return padi_run<E, NSL>(padi<E>(v), i);
        else return padi<E>(v + NSL * i);
    }

    // tw: this length's stage table (TW_SIZE entries, forward exponent).
    // PRED with act = false: an idle team, which only meets the barriers.
    // WS: the teams are warp-contained (see team_sync).
    template <bool PRED = false, bool WS = false>
    __device__ __forceinline__ static void run(cx<T> (&a)[E], int tt, cx<T>* sm,
                                               const cx<T>* __restrict__ tw, bool act = true) {
        stage<R0, 1, 0>(a, tt, tw);
        if constexpr (R1 > 1) {
            exchange<R0, 1, R1, PRED, WS>(a, tt, sm, act);
            stage<R1, R0, TW_OFF1>(a, tt, tw);
            if constexpr (R2 > 1) {
                exchange<R1, R0, R2, PRED, WS>(a, tt, sm, act);
                stage<R2, R0 * R1, TW_OFF2>(a, tt, tw);
            }
        }
    }

    // run() with the stage twiddles already in registers (load_tw).
    template <bool PRED = false, bool WS = false>
    __device__ __forceinline__ static void run_reg(cx<T> (&a)[E], int tt, cx<T>* sm, const Tw& t, bool act = true) {
        stage<R0, 1, 0>(a, tt, nullptr);
        if constexpr (R1 > 1) {
            exchange<R0, 1, R1, PRED, WS>(a, tt, sm, act);
            stage_reg<R1, R0, 0>(a, t);
            if constexpr (R2 > 1) {
                exchange<R1, R0, R2, PRED, WS>(a, tt, sm, act);
                stage_reg<R2, R0 * R1, NW1>(a, t);
            }
        }
    }
};

}  // namespace nufft
