// btrt_dw.cuh -- double-word ("double-float") arithmetic: a value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  GB300's FP64 pipe issues ~1/64 of the FP32 rate, so FP64-class
// accuracy is cheaper on the FP32 pipe this way.
//
// Building blocks (each written from its published definition):
//   TwoSum      (Knuth, TAOCP vol. 2): s = fl(a + b) and the exact error of that sum
//   Fast2Sum    (Dekker 1971): the same when |a| >= |b|, three operations
//   TwoProd     (with an FMA): p = fl(a b), e = fma(a, b, -p) exactly a b - p
//   DW + DW     the "sloppy" double-word sum analysed by Joldes, Muller and Popescu
//               (ACM TOMS 2017): TwoSum of the high parts, the low parts added,
//               renormalised by Fast2Sum; absolute error of order 2^-48 (|x| + |y|)
//   DW x DW     TwoProd of the high parts plus the cross terms (one FMA),
//               renormalised by Fast2Sum, as in the double-word products of the
//               same paper
//   DW / DW     one Newton-corrected quotient of the high parts (used off the hot path)
//   fma(DW)     the product's terms summed with the addend before one renormalisation
// All primitive operations use the _rn intrinsics so that the compiler cannot
// contract a product and a sum into an FMA, which would break the error terms.
#pragma once

#include <cuda_runtime.h>

namespace btrt {

// keep the float/double fma overloads visible next to the double-word one
using ::fma;

struct __align__(8) dw {
    float hi, lo;

    dw() = default;
    __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
    // from a double: the nearest float, then the nearest float of the remainder
    __host__ __device__ constexpr dw(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
    __host__ __device__ constexpr dw(int i) : hi(static_cast<float>(i)), lo(0.0f) {}
    __host__ __device__ explicit operator double() const {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dw(s, e);
}

__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dw two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dw(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }

__device__ __forceinline__ dw operator*(dw x, dw y) {
    const dw p = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

__device__ __forceinline__ dw operator/(dw x, dw y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const dw r = x - y * dw(q1, 0.0f);
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ dw &operator+=(dw &x, dw y) { return x = x + y; }

// a b + c without renormalising the product: TwoProd of the high parts and the
// cross terms, TwoSum of the product's and c's high parts, the remaining terms
// added to its error, one Fast2Sum (16 operations against 19 for DW x DW then
// DW + DW, the same order of error; the double-word sweep measured 6.7 % faster)
__device__ __forceinline__ dw fma(dw a, dw b, dw c) {
    const dw p = two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    const dw s = two_sum(p.hi, c.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(__fadd_rn(p.lo, t), c.lo));
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ bool not_finite(dw v) {
    return (__float_as_int(v.hi) & 0x7f800000) == 0x7f800000;
}

}  // namespace btrt
