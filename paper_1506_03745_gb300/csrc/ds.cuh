// Double-single arithmetic: a number is the unevaluated sum hi + lo of two
// FP32 values with |lo| <= ulp(hi) / 2, about 48 significant bits in the
// FP32 exponent range (magnitudes from about 1e-38 to 1e38; lo loses bits
// below about 1e-31).  Built on the error-free transformations of Knuth
// (two-sum, TAOCP vol. 2, 4.2.2) and Dekker (product error, here by one fused
// multiply-add; Numer. Math. 18, 1971).  The treecode's FP64-class product
// (the outer residual of the refinement) runs in it on the FP32 pipe, which
// GB300 issues 64 times as fast as FP64.  Every operation is written with
// the _rn intrinsics so that the compiler neither fuses nor reorders them.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace pgb {

struct __align__(8) ds {
    float hi, lo;
    ds() = default;
    __host__ __device__ constexpr ds(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ds(int i) : hi((float)i), lo(0.f) {}  // exact for |i| < 2^24
};

// Split of a double constant (folded at compile time for literals).
__host__ __device__ constexpr ds ds_const(double d) {
    return ds((float)d, (float)(d - (double)(float)d));
}

__device__ __forceinline__ ds ds_from_double(double d) {
    const float h = __double2float_rn(d);
    return ds(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double ds_to_double(ds a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ds two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ds(s, e);
}
// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ ds fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ds(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// a + b with error below about 2^-47 (|a| + |b|)
__device__ __forceinline__ ds operator+(ds a, ds b) {
    const ds s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ds operator-(ds a) { return ds(-a.hi, -a.lo); }
__device__ __forceinline__ ds operator-(ds a, ds b) { return a + (-b); }
__device__ __forceinline__ ds& operator+=(ds& a, ds b) {
    a = a + b;
    return a;
}
// a b: the exact product of the high parts by one fused multiply-add, the
// cross terms added to its error (relative error below about 2^-46)
__device__ __forceinline__ ds operator*(ds a, ds b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a b + c in one pass: the product's error term joins the sum (error below
// about 2^-46 (|a b| + |c|)); 15 FP32 operations instead of 18
__device__ __forceinline__ ds ds_fma(ds a, ds b, ds c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const ds s = two_sum(p, c.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
__device__ __forceinline__ ds mul_f(ds a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ bool operator>(ds a, ds b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// 1/sqrt(x), x > 0 (x = 0 gives a non-finite value; callers mask it): the
// SFU estimate y of 1/sqrt(x.hi) (relative error below 2^-22) and one Newton
// step y + (y/2)(1 - x y^2) with the residual 1 - x y^2 formed in
// double-single; the step leaves a relative error of about 1.5 d^2 < 3e-14.
__device__ __forceinline__ ds ds_rsqrt(ds x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x.hi));
    const ds e = ds(1) - mul_f(mul_f(x, y), y);
    return two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e.hi));
}

// 2^t for t < 127 (results below 2^-126 are returned as 0), table-driven
// (Tang's reduction, ACM TOMS 15, 1989): t = m / 64 + f with m = rint(64 t.hi)
// and |f| <= 1/128 (t.hi - m/64 is exact), so 2^t = 2^(m >> 6) 2^(j/64) 2^f
// with j = m & 63.  2^(j/64) comes from a 64-entry double-single table
// computed at compile time from the exponential series; 2^f from its Taylor
// series sum_k (ln 2)^k f^k / k!: the terms k = 3..5 in FP32 (they are below
// 2.7e-8 in all, so FP32 leaves them an error below 2e-15), k = 0..2 by
// Horner steps in double-single; the truncation after k = 5 is below
// 0.0055^6 / 720 < 4e-17.  Then 2^(m >> 6) is applied to both parts (exact).
template <int K>
struct DsCoef {
    static constexpr ds v = ds_const(Exp2Coef<K>::v);
};
// e^x by its series, for the compile-time table (|x| < 1: 30 terms reach
// double rounding)
__host__ __device__ constexpr double exp_series(double x) {
    double s = 1.0, t = 1.0;
    for (int k = 1; k < 30; ++k) {
        t = t * x / k;
        s += t;
    }
    return s;
}
struct Exp2Table {
    ds v[64];
    __host__ __device__ constexpr Exp2Table() : v() {
        for (int j = 0; j < 64; ++j) v[j] = ds_const(exp_series(j * PGB_LN2 / 64.0));
    }
};
__device__ const Exp2Table kExp2Table = Exp2Table();

__device__ __forceinline__ ds ds_exp2(ds t) {
    const float mf = rintf(__fmul_rn(t.hi, 64.f));
    const int m = (int)mf;
    const ds f = two_sum(__fsub_rn(t.hi, __fmul_rn(mf, 0.015625f)), t.lo);
    // tail k = 3..5 in FP32 (Horner), as the coefficient of f^3
    float q = (float)Exp2Coef<5>::v;
    q = __fmaf_rn(q, f.hi, (float)Exp2Coef<4>::v);
    q = __fmaf_rn(q, f.hi, (float)Exp2Coef<3>::v);
    ds p = DsCoef<2>::v + mul_f(f, q);
    p = ds_fma(p, f, DsCoef<1>::v);
    p = ds_fma(p, f, ds(1));
    const float2 tv = __ldg(reinterpret_cast<const float2*>(&kExp2Table.v[m & 63]));
    p = p * ds(tv.x, tv.y);
    const int n = m >> 6;  // floor(m / 64)
    if (n < -126) return ds(0);
    const float sc = __int_as_float((127 + n) << 23);
    return ds(__fmul_rn(p.hi, sc), __fmul_rn(p.lo, sc));
}

// e^x = 2^(x log2 e)
__device__ __forceinline__ ds ds_exp(ds x) {
    constexpr ds log2e = ds_const(1.44269504088896340735992468100189);
    return ds_exp2(x * log2e);
}

}  // namespace pgb
