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
    double mun[19][3], wn[19];
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
