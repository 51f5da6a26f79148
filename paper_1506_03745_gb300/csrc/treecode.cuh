// Treecode kernels of the boundary-element matvec (Section 3.2 of the paper),
// templated on the arithmetic type and on the Taylor order P.
//
// Combined potential.  Every row of Eq. 6 / Eq. 7 needs, per target x and per
// kernel G (Laplace 1/r or Yukawa e^{-kappa r}/r, without the 1/4pi), the
// combination U = S_V - S_K of single- and double-layer sums:
//   U(x) = sum_s [ q_s G(x - y_s) - p_s . grad_y G(x - y_s) ],
// with, per quadrature point s of panel j (weight w_s = w_m A_j):
//   q_s = w_s psi_j  (single-layer density),  p_s = w_s phi_j n_j (double layer).
// Near: direct sum.  Far: G(R - d) = sum_k G_k(R) (-d)^k with R = x - c,
// d = y - c, G_k = d^k G / k! (derivatives in R), so
//   U = sum_k G_k(R) M_k,  M_k = sum_s (q_s + p_s . grad_u) u_s^k,  u_s = c - y_s.
// Recurrences for G_k (derived from rho^2 dG/dR_i = -R_i G - kappa R_i H and
// dH/dR_i = -kappa R_i G with H = e^{-kappa rho}), n = |k| >= 1:
//   S1 = sum_a R_a G_{k-e_a},  S2 = sum_a G_{k-2e_a}   (and T1, T2 with H)
//   H_k = -(kappa/n) (S1 + S2)
//   G_k = -[(2n-1) S1 + (n-1) S2 + kappa (T1 + T2)] / (n rho^2)
// Laplace is the same with kappa = 0 (H_0 = 1, H_k = 0).
// Moment shift (upward pass): M_k(c') = sum_{j<=k} C(k,j) (c'-c)^{k-j} M_j(c).
#pragma once
#include "common.cuh"
#include "pgb_internal.cuh"

namespace pgb {

template <typename T>
struct V4;
template <>
struct V4<float> {
    using t = float4;
};
template <>
struct V4<double> {
    using t = dbl4;
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float exp_(float x) { return __expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }

// Neumaier-compensated accumulation s + c += v.
template <typename T>
__device__ __forceinline__ void kadd(T& s, T& c, T v) {
    T t = s + v;
    c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// Multi-indices of total degree <= P: graded, and within a degree kx
// descending then ky descending.
template <int P>
struct MI {
    static constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6;
    int k[T][3];
    int lvl[T];
    int m1[T][3];
    int m2[T][3];
    constexpr MI() : k(), lvl(), m1(), m2() {
        int t = 0;
        for (int n = 0; n <= P; ++n)
            for (int x = n; x >= 0; --x)
                for (int y = n - x; y >= 0; --y) {
                    k[t][0] = x;
                    k[t][1] = y;
                    k[t][2] = n - x - y;
                    lvl[t] = n;
                    ++t;
                }
        for (int i = 0; i < T; ++i)
            for (int a = 0; a < 3; ++a) {
                m1[i][a] = -1;
                m2[i][a] = -1;
                for (int j = 0; j < T; ++j) {
                    bool e1 = true, e2 = true;
                    for (int b = 0; b < 3; ++b) {
                        int d = (a == b) ? 1 : 0;
                        if (k[j][b] != k[i][b] - d) e1 = false;
                        if (k[j][b] != k[i][b] - 2 * d) e2 = false;
                    }
                    if (e1) m1[i][a] = j;
                    if (e2) m2[i][a] = j;
                }
            }
    }
    constexpr int index(int x, int y, int z) const {
        for (int i = 0; i < T; ++i)
            if (k[i][0] == x && k[i][1] == y && k[i][2] == z) return i;
        return -1;
    }
};

// Runtime decode of the multi-index order of MI<P>: index t -> (kx, ky, kz).
__device__ __forceinline__ void decode_mi(int t, int& x, int& y, int& z) {
    int n = 0, cnt = 1;
    while (t >= cnt) {
        t -= cnt;
        ++n;
        cnt = (n + 1) * (n + 2) / 2;
    }
    int xx = n, m = 1;
    while (t >= m) {
        t -= m;
        --xx;
        ++m;
    }
    x = xx;
    y = (n - xx) - t;
    z = n - x - y;
}

struct EvalArgs {
    int64_t n_groups;
    const int32_t *gstart, *gend, *gbody;
    const double* gcenter;
    const int64_t *near_off, *far_off;
    const int32_t *near_l, *far_l;
    const int32_t *nstart, *nend, *nbody;
    const double* ncenter;
    int K;
    double kappa;
    int lap_body[PGB_MAX_BODIES];  // 1 when the body is dielectric
    double* U;                     // 2 per sorted panel
};

// Far-field contraction sum_k G_k(R) M_k for one target (returns Yukawa and,
// when lap, Laplace).
template <typename real, int P>
__device__ __forceinline__ void m2p_eval(real Rx, real Ry, real Rz, real kappa, const real* ML, const real* MY,
                                         bool lap, real& uL, real& uY) {
    constexpr MI<P> mi{};
    constexpr int T = MI<P>::T;
    real R[3] = {Rx, Ry, Rz};
    real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    real ri = rsqrt_(r2);
    real i2 = ri * ri;
    real rho = r2 * ri;
    real G[T], H[T];
    H[0] = exp_(-kappa * rho);
    G[0] = H[0] * ri;
    real accY = G[0] * MY[0];
#pragma unroll
    for (int k = 1; k < T; ++k) {
        const int n = mi.lvl[k];
        real S1 = 0, S2 = 0, T1 = 0, T2 = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mi.m1[k][a] >= 0) {
                S1 += R[a] * G[mi.m1[k][a]];
                T1 += R[a] * H[mi.m1[k][a]];
            }
            if (mi.m2[k][a] >= 0) {
                S2 += G[mi.m2[k][a]];
                T2 += H[mi.m2[k][a]];
            }
        }
        const real inv_n = real(1) / real(n);
        const real c1 = real(2 * n - 1) * inv_n, c2 = real(n - 1) * inv_n;
        real kn = kappa * inv_n;
        H[k] = -kn * (S1 + S2);
        G[k] = -(c1 * S1 + c2 * S2 + kn * (T1 + T2)) * i2;
        accY += G[k] * MY[k];
    }
    uY = accY;
    if (lap) {
        real L[T];
        L[0] = ri;
        real accL = L[0] * ML[0];
#pragma unroll
        for (int k = 1; k < T; ++k) {
            const int n = mi.lvl[k];
            real S1 = 0, S2 = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (mi.m1[k][a] >= 0) S1 += R[a] * L[mi.m1[k][a]];
                if (mi.m2[k][a] >= 0) S2 += L[mi.m2[k][a]];
            }
            const real inv_n = real(1) / real(n);
            const real c1 = real(2 * n - 1) * inv_n, c2 = real(n - 1) * inv_n;
            L[k] = -(c1 * S1 + c2 * S2) * i2;
            accL += L[k] * ML[k];
        }
        uL = accL;
    } else {
        uL = 0;
    }
}

// K-point sums of one tile of source points for one target (relative position
// r0 = target - leaf centre).  With OWN, points of the target's own panel
// (indices [own_lo, own_hi)) are skipped.
template <typename real, bool LAP, bool OWN>
__device__ __forceinline__ void p2p_tile(const typename V4<real>::t* sA, const typename V4<real>::t* sB, int cnt,
                                         int64_t t, int64_t own_lo, int64_t own_hi, real r0x, real r0y, real r0z,
                                         real kappa, real& sumL, real& sumY) {
    using v4 = typename V4<real>::t;
    const real nkl = -kappa;
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
        const v4 A = sA[j], B = sB[j];
        const real dx = r0x - A.x, dy = r0y - A.y, dz = r0z - A.z;
        const real r2 = dx * dx + dy * dy + dz * dz;
        bool keep = r2 > real(0);
        if (OWN) keep = keep && !(t + j >= own_lo && t + j < own_hi);
        const real ri = keep ? rsqrt_(r2) : real(0);
        const real pd = B.x * dx + B.y * dy + B.z * dz;
        const real tt = pd * (ri * ri);
        if (LAP) sumL += ri * (A.w - tt);
        const real r = r2 * ri;
        const real ex = exp_(nkl * r);
        const real gg = kappa * r + real(1);
        sumY += (ex * ri) * (B.w - gg * tt);
    }
}

// One warp per target group: P2P over the near leaves, M2P over the far nodes.
template <typename real, int P>
__global__ void __launch_bounds__(128) k_eval(EvalArgs a, const typename V4<real>::t* __restrict__ src,
                                              const typename V4<real>::t* __restrict__ xrel,
                                              const real* __restrict__ mom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    __shared__ v4 sA[4][32], sB[4][32];
    __shared__ real sM[4][2 * T];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * 4 + w;
    if (g >= a.n_groups) return;
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    const int64_t p = p0 + lane;
    const bool active = p < p1;
    v4 xr = active ? xrel[p] : xrel[p0];
    const double gc0 = a.gcenter[3 * g], gc1 = a.gcenter[3 * g + 1], gc2 = a.gcenter[3 * g + 2];
    const int gb = a.gbody[g];
    const real kappa = (real)a.kappa;
    real UL = 0, cL = 0, UY = 0, cY = 0;
    // ---- near field: direct K-point sums
    for (int64_t e = a.near_off[g]; e < a.near_off[g + 1]; ++e) {
        const int nd = a.near_l[e];
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        const real r0x = xr.x - (real)(a.ncenter[3 * nd] - gc0);
        const real r0y = xr.y - (real)(a.ncenter[3 * nd + 1] - gc1);
        const real r0z = xr.z - (real)(a.ncenter[3 * nd + 2] - gc2);
        const int64_t s0 = (int64_t)a.nstart[nd] * a.K, s1 = (int64_t)a.nend[nd] * a.K;
        // the target's own panel is left to the near-field correction (its
        // centroid node is singular); only a leaf overlapping the group needs the test
        const bool own = (a.nstart[nd] < p1) && (a.nend[nd] > p0);
        const int64_t own_lo = p * a.K, own_hi = own_lo + a.K;
        for (int64_t t = s0; t < s1; t += 32) {
            const int cnt = (int)min((int64_t)32, s1 - t);
            __syncwarp();
            if (lane < cnt) {
                sA[w][lane] = src[2 * (t + lane)];
                sB[w][lane] = src[2 * (t + lane) + 1];
            }
            __syncwarp();
            real sumL = 0, sumY = 0;
            if (own) {
                if (lap) p2p_tile<real, true, true>(sA[w], sB[w], cnt, t, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
                else p2p_tile<real, false, true>(sA[w], sB[w], cnt, t, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
            } else {
                if (lap) p2p_tile<real, true, false>(sA[w], sB[w], cnt, t, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
                else p2p_tile<real, false, false>(sA[w], sB[w], cnt, t, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
            }
            kadd(UL, cL, sumL);
            kadd(UY, cY, sumY);
        }
    }
    // ---- far field: Taylor expansions about node centres
    for (int64_t e = a.far_off[g]; e < a.far_off[g + 1]; ++e) {
        const int nd = a.far_l[e];
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        __syncwarp();
        for (int k = lane; k < 2 * T; k += 32) sM[w][k] = mom[(int64_t)nd * 2 * T + k];
        __syncwarp();
        const real Rx = xr.x - (real)(a.ncenter[3 * nd] - gc0);
        const real Ry = xr.y - (real)(a.ncenter[3 * nd + 1] - gc1);
        const real Rz = xr.z - (real)(a.ncenter[3 * nd + 2] - gc2);
        real uL, uY;
        m2p_eval<real, P>(Rx, Ry, Rz, kappa, sM[w], sM[w] + T, lap, uL, uY);
        kadd(UL, cL, uL);
        kadd(UY, cY, uY);
    }
    if (active) {
        a.U[2 * p] = (double)UL + (double)cL;
        a.U[2 * p + 1] = (double)UY + (double)cY;
    }
}

struct UpArgs {
    int64_t n_leaves;
    const int32_t *leaf_node, *nstart, *nend, *parent, *child, *nchild;
    const double* ncenter;
    int K;
    unsigned int* counter;  // per node, zero between launches
};

// Upward pass in one launch: each block forms the moments of one leaf from its
// points, then the block that completes the last child of a node forms the
// node from its children by the binomial shift, and so on to the root.  No
// block waits on another; the child order of every sum is fixed.
template <typename real, int P>
__global__ void __launch_bounds__(128) k_upward(UpArgs a, const typename V4<real>::t* __restrict__ src,
                                                real* __restrict__ mom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    __shared__ real pw[128][3][P + 1];
    __shared__ real sq[128][5];
    __shared__ real dp[3][P + 1];
    __shared__ short idx3[P + 1][P + 1][P + 1];
    __shared__ int last;
    const int tid = threadIdx.x;
    const int64_t leaf = blockIdx.x;
    if (leaf >= a.n_leaves) return;
    int nd = a.leaf_node[leaf];
    int kx = 0, ky = 0, kz = 0;
    if (tid < T) {
        decode_mi(tid, kx, ky, kz);
        idx3[kx][ky][kz] = (short)tid;
    }
    // ---- P2M at the leaf centre: u = c - y = -(y - c)
    {
        real accL = 0, accY = 0;
        const int64_t s0 = (int64_t)a.nstart[nd] * a.K, s1 = (int64_t)a.nend[nd] * a.K;
        for (int64_t t = s0; t < s1; t += 128) {
            const int cnt = (int)min((int64_t)128, s1 - t);
            __syncthreads();
            if (tid < cnt) {
                const v4 A = src[2 * (t + tid)], B = src[2 * (t + tid) + 1];
                const real u[3] = {-A.x, -A.y, -A.z};
                for (int q = 0; q < 3; ++q) {
                    real v = 1;
                    for (int m = 0; m <= P; ++m) {
                        pw[tid][q][m] = v;
                        v *= u[q];
                    }
                }
                sq[tid][0] = A.w;  // qL
                sq[tid][1] = B.w;  // qY
                sq[tid][2] = B.x;  // p
                sq[tid][3] = B.y;
                sq[tid][4] = B.z;
            }
            __syncthreads();
            if (tid < T) {
                for (int j = 0; j < cnt; ++j) {
                    const real mono = pw[j][0][kx] * pw[j][1][ky] * pw[j][2][kz];
                    real dl = 0;
                    if (kx) dl += sq[j][2] * real(kx) * pw[j][0][kx - 1] * pw[j][1][ky] * pw[j][2][kz];
                    if (ky) dl += sq[j][3] * real(ky) * pw[j][0][kx] * pw[j][1][ky - 1] * pw[j][2][kz];
                    if (kz) dl += sq[j][4] * real(kz) * pw[j][0][kx] * pw[j][1][ky] * pw[j][2][kz - 1];
                    accL += sq[j][0] * mono + dl;
                    accY += sq[j][1] * mono + dl;
                }
            }
        }
        if (tid < T) {
            mom[(int64_t)nd * 2 * T + tid] = accL;
            mom[(int64_t)nd * 2 * T + T + tid] = accY;
        }
    }
    // ---- walk up while this block completed the last child
    while (true) {
        __threadfence();
        __syncthreads();
        const int par = a.parent[nd];
        if (par < 0) break;
        if (tid == 0) {
            unsigned int prev = atomicAdd(&a.counter[par], 1u);
            last = (prev + 1 == (unsigned int)a.nchild[par]);
            if (last) a.counter[par] = 0;  // leave the counter clean for the next launch
        }
        __syncthreads();
        if (!last) break;
        __threadfence();
        nd = par;
        real accL = 0, accY = 0;
        const int fc = a.child[nd], nc = a.nchild[nd];
        for (int ci = 0; ci < nc; ++ci) {
            const int ch = fc + ci;
            __syncthreads();
            if (tid < 3) {
                const real d = (real)(a.ncenter[3 * nd + tid] - a.ncenter[3 * ch + tid]);
                real v = 1;
                for (int m = 0; m <= P; ++m) {
                    dp[tid][m] = v;
                    v *= d;
                }
            }
            __syncthreads();
            if (tid < T) {
                const volatile real* mc = mom + (int64_t)ch * 2 * T;
                real bx = 1;
                for (int jx = 0; jx <= kx; ++jx) {
                    real by = 1;
                    for (int jy = 0; jy <= ky; ++jy) {
                        real bz = 1;
                        for (int jz = 0; jz <= kz; ++jz) {
                            const int j = idx3[jx][jy][jz];
                            const real coef = bx * by * bz * dp[0][kx - jx] * dp[1][ky - jy] * dp[2][kz - jz];
                            accL += coef * mc[j];
                            accY += coef * mc[T + j];
                            bz = bz * real(kz - jz) / real(jz + 1);
                        }
                        by = by * real(ky - jy) / real(jy + 1);
                    }
                    bx = bx * real(kx - jx) / real(jx + 1);
                }
            }
        }
        if (tid < T) {
            mom[(int64_t)nd * 2 * T + tid] = accL;
            mom[(int64_t)nd * 2 * T + T + tid] = accY;
        }
    }
}

}  // namespace pgb
