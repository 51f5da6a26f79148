// Transposed treecode (the adjoint operator A^T of Eq. 6 / Eq. 7).
//
// (A^T lam)_j = sum_i lam_i A_ij.  With the panel integrals of Eq. 9,
//   sum_i s_i V_ij = sum_{nodes y_s of panel j} w_s Phi(y_s),
//   sum_i s_i K_ij = sum_{nodes y_s of panel j} w_s n_j . grad Phi(y_s),
// where Phi(y) = sum_i s_i G(|y - c_i|) is the potential of point sources
// s_i at the collocation points.  So the transposed product is a treecode
// with the centroids as sources and the quadrature nodes as targets that
// evaluates the potential and its normal derivative: P2P directly, and M2P
//   Phi = sum_{|k|<=P} G_k(R) M_k,
//   n . grad Phi = sum_{|m|<=P+1} G_m(R) D_m,  D_m = sum_a n_a m_a M_{m-e_a},
// from dG_k/dR_a = (k_a + 1) G_{k+e_a}, with R = y - c and moments
// M_k = sum_i s_i (c - c_i)^k about the node centre c.
#pragma once
#include "treecode.cuh"

namespace pgb {

struct TArgs {
    int64_t n_groups;
    const int32_t *gstart, *gend, *gbody;
    const int64_t *near_off, *far_off;
    const float4 *near4, *far4;    // FP32 node centre - group centre, node id bits
    const int32_t *near_l, *far_l;
    const int32_t *nstart, *nend, *nbody;
    const double *ncenter, *gcenter;
    int K;
    double kappa;
    int lap_body[PGB_MAX_BODIES];
    double* out;                   // 4 per quadrature node: Phi_L, dPhi_L/dn, Phi_Y, dPhi_Y/dn (no 1/4pi)
};

template <typename real>
__device__ __forceinline__ void t_offset(const TArgs& a, int64_t e, bool far, int64_t g, int& nd, real& ox, real& oy,
                                         real& oz) {
    if (sizeof(real) == sizeof(float)) {
        const float4 q = far ? a.far4[e] : a.near4[e];
        nd = __float_as_int(q.w);
        ox = (real)q.x;
        oy = (real)q.y;
        oz = (real)q.z;
    } else {
        nd = far ? a.far_l[e] : a.near_l[e];
        ox = (real)(a.ncenter[3 * nd] - a.gcenter[3 * g]);
        oy = (real)(a.ncenter[3 * nd + 1] - a.gcenter[3 * g + 1]);
        oz = (real)(a.ncenter[3 * nd + 2] - a.gcenter[3 * g + 2]);
    }
}

// P2P: one block per target group with K warps; warp w owns the group's
// quadrature nodes 32w .. 32w+31 (node q belongs to panel q / K).  Sources:
// centroids of the near leaves, `srcT` = {c - c_leaf, s_L} and {s_Y, -, -, -},
// staged 32 at a time.  The target's own panel is skipped: its self entry is
// carried by the near-field corrections.
template <typename real>
__global__ void __launch_bounds__(224) k_p2p_T(TArgs a, const typename V4<real>::t* __restrict__ ytg,
                                                const typename V4<real>::t* __restrict__ nrm,
                                                const typename V4<real>::t* __restrict__ srcT) {
    using v4 = typename V4<real>::t;
    __shared__ v4 sA[7][32], sB[7][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = blockIdx.x;
    if (g >= a.n_groups) return;
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    if (32 * w >= (p1 - p0) * a.K) return;  // whole warp beyond the group's nodes
    const int64_t q = p0 * a.K + 32 * w + lane;
    const bool active = q < p1 * a.K;
    const v4 y = ytg[active ? q : p0 * a.K];
    const int64_t panel = active ? q / a.K : p0;
    const v4 n = nrm[panel];
    const int gb = a.gbody[g];
    const real kappa = (real)a.kappa;
    const real nkl = -kappa * real(1.4426950408889634);
    real acc[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (int64_t e = a.near_off[g]; e < a.near_off[g + 1]; ++e) {
        int nd;
        real ox, oy, oz;
        t_offset<real>(a, e, false, g, nd, ox, oy, oz);
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        const real rx = y.x - ox, ry = y.y - oy, rz = y.z - oz;
        for (int64_t j0 = a.nstart[nd]; j0 < a.nend[nd]; j0 += 32) {
            const int cnt = (int)min((int64_t)32, (int64_t)a.nend[nd] - j0);
            __syncwarp();
            if (lane < cnt) {
                sA[w][lane] = srcT[2 * (j0 + lane)];
                sB[w][lane] = srcT[2 * (j0 + lane) + 1];
            }
            __syncwarp();
            real t[4] = {0, 0, 0, 0};
            for (int j = 0; j < cnt; ++j) {
                const v4 C = sA[w][j];
                const real sY = sB[w][j].x;
                const real dx = rx - C.x, dy = ry - C.y, dz = rz - C.z;
                const real r2 = dx * dx + dy * dy + dz * dz;
                real ri = rsqrt_fast(r2);
                ri = (r2 > real(0) && (j0 + j) != panel) ? ri : real(0);
                const real ri3 = ri * ri * ri;
                const real nd_ = n.x * dx + n.y * dy + n.z * dz;
                if (lap) {
                    t[0] += C.w * ri;
                    t[1] -= C.w * nd_ * ri3;
                }
                const real r = r2 * ri;
                const real ex = exp2_(nkl * r);
                t[2] += sY * ex * ri;
                t[3] -= sY * (kappa * r + real(1)) * ex * nd_ * ri3;
            }
            for (int k = 0; k < 4; ++k) kadd(acc[k], cmp[k], t[k]);
        }
    }
    if (active)
        for (int k = 0; k < 4; ++k) a.out[4 * q + k] = (double)acc[k] + (double)cmp[k];
}

// Far-field potential and normal derivative for one target: Yukawa always,
// Laplace when lap (see the header comment for the formulas).
template <typename real, int P>
__device__ __forceinline__ void m2p_grad(real Rx, real Ry, real Rz, real nx, real ny, real nz, real kappa,
                                         const real* ML, const real* MY, bool lap, real* res) {
    constexpr MI<P + 1> mi{};
    constexpr int T1 = MI<P + 1>::T;
    constexpr int T0 = MI<P>::T;
    const real R[3] = {Rx, Ry, Rz};
    const real nn[3] = {nx, ny, nz};
    const real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const real ri = rsqrt_fast(r2);
    const real i2 = ri * ri;
    const real rho = r2 * ri;
    real an[P + 2], bn[P + 2], en[P + 2], hn[P + 2];
#pragma unroll
    for (int n = 1; n <= P + 1; ++n) {
        const real inv_n = real(1) / real(n);
        an[n] = -(real(2 * n - 1) * inv_n) * i2;
        bn[n] = -(real(n - 1) * inv_n) * i2;
        hn[n] = -kappa * inv_n;
        en[n] = hn[n] * i2;
    }
    {
        real G[T1], H[T1];
        H[0] = exp_(-kappa * rho);
        G[0] = H[0] * ri;
        real phi = G[0] * MY[0], dphi = 0;
#pragma unroll
        for (int k = 1; k < T1; ++k) {
            const int n = mi.lvl[k];
            real S1 = 0, S2 = 0, T1s = 0, T2s = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (mi.m1[k][a] >= 0) {
                    S1 += R[a] * G[mi.m1[k][a]];
                    T1s += R[a] * H[mi.m1[k][a]];
                }
                if (mi.m2[k][a] >= 0) {
                    S2 += G[mi.m2[k][a]];
                    T2s += H[mi.m2[k][a]];
                }
            }
            if (n < P + 1) H[k] = hn[n] * (S1 + S2);
            G[k] = an[n] * S1 + bn[n] * S2 + en[n] * (T1s + T2s);
            if (k < T0) phi += G[k] * MY[k];
            real D = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (mi.m1[k][a] >= 0) D += nn[a] * real(mi.k[k][a]) * MY[mi.m1[k][a]];
            dphi += G[k] * D;
        }
        res[2] = phi;
        res[3] = dphi;
    }
    if (lap) {
        real L[T1];
        L[0] = ri;
        real phi = L[0] * ML[0], dphi = 0;
#pragma unroll
        for (int k = 1; k < T1; ++k) {
            const int n = mi.lvl[k];
            real S1 = 0, S2 = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (mi.m1[k][a] >= 0) S1 += R[a] * L[mi.m1[k][a]];
                if (mi.m2[k][a] >= 0) S2 += L[mi.m2[k][a]];
            }
            L[k] = an[n] * S1 + bn[n] * S2;
            if (k < T0) phi += L[k] * ML[k];
            real D = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (mi.m1[k][a] >= 0) D += nn[a] * real(mi.k[k][a]) * ML[mi.m1[k][a]];
            dphi += L[k] * D;
        }
        res[0] = phi;
        res[1] = dphi;
    } else {
        res[0] = res[1] = 0;
    }
}

// M2P: one block per target group (K warps, as k_p2p_T); the block loads each
// far node's moments once into shared memory; adds to out.
template <typename real, int P>
__global__ void __launch_bounds__(224, sizeof(real) == 4 ? 2 : 1) k_m2p_T(TArgs a, const typename V4<real>::t* __restrict__ ytg,
                                                const typename V4<real>::t* __restrict__ nrm,
                                                const real* __restrict__ mom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    __shared__ real sM[2 * T];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = blockIdx.x;
    if (g >= a.n_groups) return;
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    const bool warp_on = 32 * w < (p1 - p0) * a.K;
    const int64_t q = p0 * a.K + 32 * w + lane;
    const bool active = warp_on && q < p1 * a.K;
    const v4 y = ytg[active ? q : p0 * a.K];
    const v4 n = nrm[active ? q / a.K : p0];
    const int gb = a.gbody[g];
    const real kappa = (real)a.kappa;
    real acc[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (int64_t e = a.far_off[g]; e < a.far_off[g + 1]; ++e) {
        int nd;
        real ox, oy, oz;
        t_offset<real>(a, e, true, g, nd, ox, oy, oz);
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) sM[k] = mom[(int64_t)nd * 2 * T + k];
        __syncthreads();
        if (!warp_on) continue;
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        real res[4];
        m2p_grad<real, P>(y.x - ox, y.y - oy, y.z - oz, n.x, n.y, n.z, kappa, sM, sM + T, lap, res);
        for (int k = 0; k < 4; ++k) kadd(acc[k], cmp[k], res[k]);
    }
    if (active)
        for (int k = 0; k < 4; ++k) a.out[4 * q + k] += (double)acc[k] + (double)cmp[k];
}

// P2M for point sources at the centroids of each leaf: M_k = sum_i s_i u_i^k,
// u = c_leaf - c_i (one block per leaf, one thread per k).
template <typename real, int P>
__global__ void __launch_bounds__(128) k_p2m_T(UpArgs a, const typename V4<real>::t* __restrict__ srcT,
                                                real* __restrict__ mom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    __shared__ real pw[128][3][P + 1];
    __shared__ real sq[128][2];
    const int tid = threadIdx.x;
    const int64_t leaf = blockIdx.x;
    if (leaf >= a.n_leaves) return;
    const int nd = a.leaf_node[leaf];
    const int64_t s0 = a.nstart[nd], s1 = a.nend[nd];
    for (int k0 = 0; k0 < T; k0 += 128) {
        const int k = k0 + tid;
        int kx = 0, ky = 0, kz = 0;
        if (k < T) decode_mi(k, kx, ky, kz);
        real accL = 0, accY = 0;
        for (int64_t t = s0; t < s1; t += 128) {
            const int cnt = (int)min((int64_t)128, s1 - t);
            __syncthreads();
            if (tid < cnt) {
                const v4 A = srcT[2 * (t + tid)], B = srcT[2 * (t + tid) + 1];
                const real u[3] = {-A.x, -A.y, -A.z};
                for (int c = 0; c < 3; ++c) {
                    real v = 1;
                    for (int m = 0; m <= P; ++m) {
                        pw[tid][c][m] = v;
                        v *= u[c];
                    }
                }
                sq[tid][0] = A.w;
                sq[tid][1] = B.x;
            }
            __syncthreads();
            if (k < T)
                for (int j = 0; j < cnt; ++j) {
                    const real mono = pw[j][0][kx] * pw[j][1][ky] * pw[j][2][kz];
                    accL += sq[j][0] * mono;
                    accY += sq[j][1] * mono;
                }
        }
        if (k < T) {
            mom[(int64_t)nd * 2 * T + k] = accL;
            mom[(int64_t)nd * 2 * T + T + k] = accY;
        }
    }
}

}  // namespace pgb
