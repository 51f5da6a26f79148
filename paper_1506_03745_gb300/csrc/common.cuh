// Device helpers shared by the kernels of libpgb (no host state).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pgb_rules.h"

namespace pgb {

#define PGB_FOUR_PI 12.566370614359172953850573533118

// Quadrature rules passed to kernels by value (Section 3.1): far rule (K
// points), fine rule (19 points) and the edge rule of the self integral.
struct Rules {
    int K, Kn, ne;
    double mu[7][3], w[7];
    double mun[37][3], wn[37];  // close-by rule: 19 or 37 points
    double ex[12], ew[12];
};

Rules make_rules(int K, int Kn, int ne);

// Unfused IEEE double arithmetic: the tree decisions (Morton cells, box
// centres, acceptance tests) are evaluated operation by operation so that they
// are reproducible on any IEEE machine.
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ void rigid(const double* P, const double* v, double* out) {
    // out = ((R0 v0 + R1 v1) + R2 v2) + t, each row, no fused products
    for (int a = 0; a < 3; ++a)
        out[a] = dadd(dadd(dadd(dmul(P[3 * a + 0], v[0]), dmul(P[3 * a + 1], v[1])), dmul(P[3 * a + 2], v[2])), P[9 + a]);
}

// FP64 reciprocal square root, for 1e-30 < x < 1e30: the FP32 SFU estimate
// (relative error below 2^-22) refined by NEWTON steps of Newton's iteration
// for 1/y^2 = x, written as y <- y + (y/2)(1 - x y^2).  A step maps a relative
// error d to about 1.5 d^2: one step leaves below 1e-13, two reach FP64
// rounding.  x = 0 gives a non-finite value; callers mask it.
template <int NEWTON>
__device__ __forceinline__ double rsqrt_nr(double x) {
    const float xf = __double2float_rn(x);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    double y = (double)yf;
#pragma unroll
    for (int i = 0; i < NEWTON; ++i) {
        const double e = fma(-(x * y), y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y;
}

// Coefficients (ln 2)^k / k! of the Taylor series of 2^f = e^{f ln 2}.
constexpr double PGB_LN2 = 0.69314718055994530941723212145818;
template <int K>
struct Exp2Coef {
    static constexpr double v = Exp2Coef<K - 1>::v * PGB_LN2 / K;
};
template <>
struct Exp2Coef<0> {
    static constexpr double v = 1.0;
};

// FP64 2^t for -2^30 < t <= 1020.  t = n + f with n = rint(t), found by adding
// and removing 1.5 * 2^52 (the sum rounds to an integer, whose low word is n),
// |f| <= 1/2; 2^f from its Taylor series to degree 11 (remainder below
// 0.347^12 / 12! * sqrt(2) < 1e-14 relative), then n is added to the exponent
// field.  Results below 2^-1020 are returned as 0.
__device__ __forceinline__ double exp2_taylor(double t) {
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    const double s = t + magic;
    const int n = __double2loint(s);
    const double f = t - (s - magic);
    double p = Exp2Coef<11>::v;
    p = fma(p, f, Exp2Coef<10>::v);
    p = fma(p, f, Exp2Coef<9>::v);
    p = fma(p, f, Exp2Coef<8>::v);
    p = fma(p, f, Exp2Coef<7>::v);
    p = fma(p, f, Exp2Coef<6>::v);
    p = fma(p, f, Exp2Coef<5>::v);
    p = fma(p, f, Exp2Coef<4>::v);
    p = fma(p, f, Exp2Coef<3>::v);
    p = fma(p, f, Exp2Coef<2>::v);
    p = fma(p, f, Exp2Coef<1>::v);
    p = fma(p, f, 1.0);
    const int hi = __double2hiint(p) + (int)((unsigned)n << 20);
    const double y = __hiloint2double(hi, __double2loint(p));
    return n < -1020 ? 0.0 : y;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide reduction helpers (blockDim.x multiple of 32, <= 1024).
template <typename T>
__device__ T block_sum(T v, T* sh) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;  // valid in thread 0
}

}  // namespace pgb
