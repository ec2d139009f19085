// dfloat.cuh -- double-word (pairs of FP32) arithmetic for the FP64-accuracy transforms.
//
// GB300's FP64 pipe runs at a small fraction of its FP32 rate, so the fused FP64 passes
// compute in double-word FP32 arithmetic instead: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits (unit roundoff u^2 = 2^-48 ~ 3.6e-15 where u = 2^-24).  The
// building blocks are the error-free transformations of the literature:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2, Theorem B): s + e = a + b exactly, six additions;
//   Fast2Sum (Dekker 1971): the same when |a| >= |b|, three additions;
//   TwoProd with an FMA: p + e = a b exactly, e = fma(a, b, -p).
// Addition is the "sloppy" double-word sum (Dekker 1971; Joldes, Muller, Popescu 2017,
// Algorithm 4): TwoSum of the high parts, the low parts added to its error, Fast2Sum.  Its
// error is a few u^2 (|a| + |b|): relative to the operands, not to a result that cancels,
// which is the normwise bound that FFT error analysis uses.  Multiplication is Dekker's
// product with an FMA (Joldes et al., Algorithm 12 without its last refinement): error a
// few u^2 |a b|.  Every operation uses the _rn intrinsics, which the compiler never
// contracts into FMAs, so the error terms are what the algorithms say they are.
#pragma once

#include <cuda_runtime.h>

namespace nufft {

struct dfloat {
    float hi, lo;
    __host__ __device__ dfloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // the nearest double-word of a double: hi its FP32 rounding, lo the rest rounded
    __host__ __device__ explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    // an int in double-word form: hi its FP32 rounding, lo the (exact) integer remainder
    __host__ __device__ dfloat(int i) : hi((float)i), lo((float)(i - (int)(float)i)) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    dfloat r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    dfloat r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }
// a1 b1 + a2 b2 with one renormalisation: the two high products summed by TwoSum, their
// exact errors (FMA), the TwoSum error and the four cross terms gathered in one word, then
// Fast2Sum.  19 operations against 25 for two products and a sum; the error stays a few
// u^2 (|a1 b1| + |a2 b2|), the normwise bound the FFTs use.
__device__ __forceinline__ dfloat dot2(dfloat a1, dfloat b1, dfloat a2, dfloat b2) {
    const float p1 = __fmul_rn(a1.hi, b1.hi);
    const float p2 = __fmul_rn(a2.hi, b2.hi);
    float s, e;
    two_sum(p1, p2, s, e);
    float t = __fadd_rn(__fmaf_rn(a1.hi, b1.hi, -p1), __fmaf_rn(a2.hi, b2.hi, -p2));
    t = __fadd_rn(t, e);
    t = __fmaf_rn(a1.hi, b1.lo, t);
    t = __fmaf_rn(a1.lo, b1.hi, t);
    t = __fmaf_rn(a2.hi, b2.lo, t);
    t = __fmaf_rn(a2.lo, b2.hi, t);
    dfloat r;
    fast_two_sum(s, t, r.hi, r.lo);
    return r;
}
// Lazy forms for the chains of one in-register DFT: each result is an exact (hi, lo) pair
// but not renormalised (|lo| may grow to a few ulp(hi) over the DFT's log2 R levels, and
// the rounding of the low words stays a few u^2 of the operands); renorm() restores the
// invariant at the DFT's end.  Addition: TwoSum of the high words, the low words added to
// its error (8 operations against 11); dot2_lazy: dot2 without its Fast2Sum (16 against 19).
__device__ __forceinline__ dfloat add_lazy(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return dfloat(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat sub_lazy(dfloat a, dfloat b) { return add_lazy(a, dfloat(-b.hi, -b.lo)); }
__device__ __forceinline__ dfloat dot2_lazy(dfloat a1, dfloat b1, dfloat a2, dfloat b2) {
    const float p1 = __fmul_rn(a1.hi, b1.hi);
    const float p2 = __fmul_rn(a2.hi, b2.hi);
    float s, e;
    two_sum(p1, p2, s, e);
    float t = __fadd_rn(__fmaf_rn(a1.hi, b1.hi, -p1), __fmaf_rn(a2.hi, b2.hi, -p2));
    t = __fadd_rn(t, e);
    t = __fmaf_rn(a1.hi, b1.lo, t);
    t = __fmaf_rn(a1.lo, b1.hi, t);
    t = __fmaf_rn(a2.hi, b2.lo, t);
    t = __fmaf_rn(a2.lo, b2.hi, t);
    return dfloat(s, t);
}
__device__ __forceinline__ dfloat renorm(dfloat a) {
    dfloat r;
    fast_two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}
// the generic code calls fma unqualified: keep the float and double ones visible beside this
using ::fma;
// a b + c, as the product then the sum (each with its own double-word rounding)
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

}  // namespace nufft
