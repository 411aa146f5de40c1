// Double-word arithmetic on FP32 pairs (device only).
//
// A double-word value x = h + l holds two FP32 numbers with |l| <= ulp(h)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations of Dekker and Knuth (Fast2Sum, 2Sum, and the exact
// product error fma(a, b, -a*b)) and the double-word algorithms analysed by
// Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
//   add      accurate sum (their Algorithm 6): relative error <= 3u^2
//   add_sl   sloppy sum (Algorithm 5): absolute error about u^2 (|x| + |y|),
//            used where a relative error of 1e-12 of the result suffices
//   mul      double-word product (Algorithm 11): relative error <= 5u^2
//   mul_u    the same before its final Fast2Sum, for operands of a sum
//   mul(x,f) product with an FP32 number (Algorithm 9): <= 2u^2
// with u = 2^-24.  The reciprocal and the reciprocal square root take the
// FP32 hardware approximation (PTX rcp.approx / rsqrt.approx, relative error
// below 2^-22) and one correction of second order in its residual e:
//   1/x       = r (1 + e + e^2 + ...),      e = 1 - x r
//   1/sqrt(x) = y (1 + e/2 + 3e^2/8 + ...), e = 1 - x y^2
// leaving O(e^3) < 2^-60 besides the double-word rounding.
//
// Every FP32 operation is an explicitly rounded intrinsic (__fadd_rn,
// __fmul_rn, __fmaf_rn): the compiler must not fuse a product into a later
// sum, which would break the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace fdu {
namespace dwa {

struct dw {
    float h, l;
};

__device__ __forceinline__ dw dw_make(float h, float l = 0.0f) { return dw{h, l}; }

// s + t = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// s + t = a + b exactly, any order of magnitude
__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    return dw{s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}

__device__ __forceinline__ dw neg(dw x) { return dw{-x.h, -x.l}; }
__device__ __forceinline__ dw dabs(dw x) { return x.h < 0.0f ? neg(x) : x; }

__device__ __forceinline__ dw add(dw x, dw y) {
    const dw s = two_sum(x.h, y.h);
    const dw t = two_sum(x.l, y.l);
    const dw v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ dw sub(dw x, dw y) { return add(x, neg(y)); }
__device__ __forceinline__ dw add_sl(dw x, dw y) {
    const dw s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ dw sub_sl(dw x, dw y) { return add_sl(x, neg(y)); }

__device__ __forceinline__ dw mul(dw x, dw y) {
    const float ch = __fmul_rn(x.h, y.h);
    const float cl1 = __fmaf_rn(x.h, y.h, -ch);
    const float cl2 = __fmaf_rn(x.l, y.h, __fmul_rn(x.h, y.l));
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
// The same product without the final renormalisation (|l| may reach about
// 2 ulp(h)): for operands of a sum, which renormalises.
__device__ __forceinline__ dw mul_u(dw x, dw y) {
    const float ch = __fmul_rn(x.h, y.h);
    const float cl1 = __fmaf_rn(x.h, y.h, -ch);
    return dw{ch, __fadd_rn(cl1, __fmaf_rn(x.l, y.h, __fmul_rn(x.h, y.l)))};
}
__device__ __forceinline__ dw mul(dw x, float y) {
    const float ch = __fmul_rn(x.h, y);
    const float cl1 = __fmaf_rn(x.h, y, -ch);
    return fast_two_sum(ch, __fmaf_rn(x.l, y, cl1));
}
// product with a power of two: exact
__device__ __forceinline__ dw scale(dw x, float p2) { return dw{__fmul_rn(x.h, p2), __fmul_rn(x.l, p2)}; }

__device__ __forceinline__ dw recip(dw x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
    const float p = __fmul_rn(x.h, r);
    const float ep = __fmaf_rn(x.h, r, -p);  // x.h r = p + ep exactly; 1 - p is exact (p near 1)
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), ep), __fmul_rn(x.l, r));
    return fast_two_sum(r, __fmul_rn(r, __fmaf_rn(e, e, e)));
}

__device__ __forceinline__ dw rsqrt(dw x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x.h));
    const float y2 = __fmul_rn(y, y);
    const float y2l = __fmaf_rn(y, y, -y2);  // y^2 = y2 + y2l exactly
    const float p = __fmul_rn(x.h, y2);
    const float ep = __fmaf_rn(x.h, y2, -p);  // x.h y2 = p + ep exactly
    const float e = __fsub_rn(__fsub_rn(1.0f, p), __fadd_rn(ep, __fmaf_rn(x.h, y2l, __fmul_rn(x.l, y2))));
    return fast_two_sum(y, __fmul_rn(__fmul_rn(y, e), __fmaf_rn(0.375f, e, 0.5f)));
}

// Compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005, algorithm Dot2, extended to
// double-word factors): s carries the running FP32 sum, c the sum of the
// exact errors of each product and sum plus the low-word cross terms; the
// result s + c has an absolute error of about u^2 times the sum of |terms|.
struct dot2 {
    float s, c;
};
__device__ __forceinline__ void dot2_add(dot2 &A, dw a, dw x) {
    const float p = __fmul_rn(a.h, x.h);
    const float e1 = __fmaf_rn(a.h, x.h, -p);
    const dw t = two_sum(A.s, p);
    A.s = t.h;
    A.c = __fadd_rn(A.c, __fadd_rn(__fadd_rn(e1, t.l), __fmaf_rn(a.h, x.l, __fmul_rn(a.l, x.h))));
}
__device__ __forceinline__ dw dot2_result(const dot2 &A) { return two_sum(A.s, A.c); }

// FP64 <-> double word by bit manipulation (GB300 runs float <-> double
// conversions on its FP64 pipe)
// double -> double word; magnitudes below 2^-126 flush to zero (the data
// stay far above); the high word keeps the top 24 bits (truncated), the low
// word the next 24 of the remaining 29 (relative error below 2^-47).  The
// pair is not renormalised (|l| < ulp(h) instead of ulp(h)/2): the
// operations that take it renormalise their results.
__device__ __forceinline__ dw d2dw(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e <= 896) return dw_make(0.0f, 0.0f);
    const unsigned sgn = hi & 0x80000000u;
    const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const unsigned m = lo & 0x1fffffffu;  // value m 2^(e - 1075)
    const unsigned lb = __float_as_uint(__uint2float_rn(m));
    const int le = (int)((lb >> 23) & 0xffu) + (e - 1075);
    const float l = (m != 0u && le > 0) ? __uint_as_float(sgn | ((unsigned)le << 23) | (lb & 0x7fffffu)) : 0.0f;
    return dw_make(h, l);  // |l| < ulp(h): the truncated split, not renormalised
}
// float -> double, exact for normal floats (zero and subnormals -> 0)
__device__ __forceinline__ double f2d(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}


}  // namespace dwa
}  // namespace fdu
