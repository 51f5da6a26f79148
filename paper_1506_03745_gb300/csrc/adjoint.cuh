// Transposed treecode (the adjoint operator A^T of Eq. 6 / Eq. 7), built as
// the exact transpose of the forward treecode product, so that
// <A x, lam> = <x, A^T lam> holds to rounding for any theta and P.
//
// (A^T lam)_j = sum_i lam_i A_ij.  With the panel integrals of Eq. 9,
//   sum_i s_i V_ij = sum_{nodes y_s of panel j} w_s Phi(y_s),
//   sum_i s_i K_ij = sum_{nodes y_s of panel j} w_s n_j . grad_y Phi(y_s),
// Phi(y) = sum_i s_i G(x_i - y) over the collocation points x_i, with the
// row weights s_i taken from lam (Laplace: interior rows, Yukawa: the
// others).  The forward product splits every (target group, source node)
// pair into near (P2P) and far (M2P); the transpose keeps the same split:
//  * near: for every forward pair (group g, near leaf b) the point sums run
//    the other way, targets of g to the quadrature nodes of b (k_p2p_T);
//  * far: the forward far field of target i from node b is
//    sum_k G_k(x_i - c_b) M_k(b) with M_k = sum_s (q_s + p_s . grad_u) u_s^k,
//    u_s = c_b - y_s, so its transpose gathers
//      L_k(b) = sum over the pairs (g, b) of sum_{i in g} s_i G_k(x_i - c_b)
//    (k_m2p_T), pushes L down the tree by the binomial shift
//      L_j(child) += sum_{k >= j} C(k, j) (c_b - c_child)^{k - j} L_k(b)
//    (k_l2l_level, the transpose of the moment shift) and evaluates at the
//    leaves Phi(y_s) = sum_k L_k u_s^k and n . grad_y Phi = -sum_k L_k n . grad_u u^k
//    (k_l2p).
#pragma once
#include "treecode.cuh"

namespace pgb {

struct TArgs {
    // the forward target groups and their lists
    int64_t n_groups;
    const int32_t *gstart, *gend, *gbody;
    const double *gcenter, *ncenter;
    const int32_t *nstart, *nend, *nbody, *nchild, *child;
    int K;
    double kappa;
    int lap_body[PGB_MAX_BODIES];
    // far: work items over the forward far lists
    int64_t n_fitems;
    const int64_t *far_off, *fitem_off;
    const int32_t *far_l, *fitem_group;
    const float4* far4;
    int m2p_item;
    // near: per source leaf (node id), the forward near entries that hold it
    const int64_t *tn_off;          // n_nodes + 1
    const int64_t* tn_e;            // forward near entry ids (group order)
    const int32_t* near_group;      // group of each forward near entry
    const float4* near4;            // leaf centre - group centre per forward near entry
    const int32_t* near_l;          // leaf node of each forward near entry
    int64_t n_leaves;
    const int32_t* leaf_node;
    int64_t lvl_begin, lvl_end;     // node range of one level (k_l2l_level)
    double* out;                    // 4 per quadrature node: Phi_L, n.grad Phi_L, Phi_Y, n.grad Phi_Y (no 1/4pi)
};

// Butterfly reduce-scatter of 32 values over the 32 lanes: lane l returns
// the sum over the warp of v[l] (31 exchanges instead of 32 x 5).
template <typename real>
__device__ __forceinline__ real reduce_scatter32(real (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool hi = lane & s;
#pragma unroll
        for (int u = 0; u < s; ++u) {
            const real give = hi ? v[u] : v[u + s];
            const real keep = hi ? v[u + s] : v[u];
            v[u] = keep + __shfl_xor_sync(0xffffffffu, give, s);
        }
    }
    return v[0];
}

// G_k(R) for |k| <= P (Yukawa when yuk, else Laplace), the recurrences of the
// forward M2P (see treecode.cuh), into G[T].
template <typename real, int P, bool YUK>
__device__ __forceinline__ void taylor_coeffs(real Rx, real Ry, real Rz, real kappa, real (&G)[MI<P>::T]) {
    constexpr MI<P> mi{};
    constexpr int T = MI<P>::T;
    const real R[3] = {Rx, Ry, Rz};
    const real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const real ri = rsqrt_(r2);
    const real i2 = ri * ri;
    const real rho = r2 * ri;
    real an[P + 1], bn[P + 1], en[P + 1], hn[P + 1];
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const real inv_n = real(1) / real(n);
        an[n] = -(real(2 * n - 1) * inv_n) * i2;
        bn[n] = -(real(n - 1) * inv_n) * i2;
        hn[n] = -kappa * inv_n;
        en[n] = hn[n] * i2;
    }
    real H[T];
    if (YUK) {
        H[0] = exp_(-kappa * rho);
        G[0] = H[0] * ri;
    } else {
        G[0] = ri;
    }
#pragma unroll
    for (int k = 1; k < T; ++k) {
        const int n = mi.lvl[k];
        real S1 = 0, S2 = 0, T1 = 0, T2 = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mi.m1[k][a] >= 0) {
                S1 += R[a] * G[mi.m1[k][a]];
                if (YUK) T1 += R[a] * H[mi.m1[k][a]];
            }
            if (mi.m2[k][a] >= 0) {
                S2 += G[mi.m2[k][a]];
                if (YUK) T2 += H[mi.m2[k][a]];
            }
        }
        if (YUK) {
            if (n < P) H[k] = hn[n] * (S1 + S2);
            G[k] = an[n] * S1 + bn[n] * S2 + en[n] * (T1 + T2);
        } else {
            G[k] = an[n] * S1 + bn[n] * S2;
        }
    }
}

// sum over the warp's lanes of s * G[k], k < T, added to dst[k] (atomic: the
// forward pairs (g, b) of one node b are spread over blocks).
template <typename real, int T>
__device__ __forceinline__ void gather_coeffs(const real (&G)[T], real s, real* dst) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b0 = 0; b0 < T; b0 += 32) {
        real v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = b0 + u < T ? s * G[b0 + u < T ? b0 + u : 0] : real(0);
        const real sum = reduce_scatter32(v);
        if (b0 + lane < T) atomicAdd(dst + b0 + lane, sum);
    }
}

// Far gather: one block of NW warps per forward M2P work item (up to m2p_item
// far nodes of one target group, as k_m2p); lane = target i with weights
// (s_L, s_Y); per node b the Yukawa (and, for a same-body dielectric pair,
// Laplace) coefficients of the 32 targets are summed and added to Lmom(b)
// (layout as the moments: T Laplace then T Yukawa per node).
template <typename real, int P, int NW>
__global__ void __launch_bounds__(NW * 32) k_m2p_T(TArgs a, const typename V4<real>::t* __restrict__ xrel,
                                                    const double* __restrict__ sT, real* __restrict__ Lmom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t it = blockIdx.x;
    if (it >= a.n_fitems) return;
    const int64_t g = a.fitem_group[it];
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    const int64_t p = p0 + lane;
    const bool active = p < p1;
    const v4 xr = active ? xrel[p] : xrel[p0];
    const real sL = active ? (real)sT[2 * p] : real(0), sY = active ? (real)sT[2 * p + 1] : real(0);
    const double gc0 = a.gcenter[3 * g], gc1 = a.gcenter[3 * g + 1], gc2 = a.gcenter[3 * g + 2];
    const int gb = a.gbody[g];
    const real kappa = (real)a.kappa;
    const int64_t fb = a.far_off[g] + (it - a.fitem_off[g]) * a.m2p_item;
    const int64_t f1 = min(a.far_off[g + 1], fb + a.m2p_item);
    for (int64_t e = fb + w; e < f1; e += NW) {
        int nd;
        real ox, oy, oz;
        if (sizeof(real) == sizeof(float)) {
            const float4 q = a.far4[e];
            nd = __float_as_int(q.w);
            ox = (real)q.x;
            oy = (real)q.y;
            oz = (real)q.z;
        } else {
            nd = a.far_l[e];
            ox = (real)(a.ncenter[3 * nd] - gc0);
            oy = (real)(a.ncenter[3 * nd + 1] - gc1);
            oz = (real)(a.ncenter[3 * nd + 2] - gc2);
        }
        const real Rx = xr.x - ox, Ry = xr.y - oy, Rz = xr.z - oz;
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        real G[T];
        taylor_coeffs<real, P, true>(Rx, Ry, Rz, kappa, G);
        gather_coeffs<real, T>(G, sY, Lmom + (int64_t)nd * 2 * T + T);
        if (lap) {
            taylor_coeffs<real, P, false>(Rx, Ry, Rz, kappa, G);
            gather_coeffs<real, T>(G, sL, Lmom + (int64_t)nd * 2 * T);
        }
    }
}

// Downward shift for every node of one level that has children:
// L_j(child) += sum_{k >= j} C(k, j) (c - c_child)^{k - j} L_k(c), applied as
// three one-axis passes (the transpose of the moment shift of the upward pass, up_m2m).
template <typename real, int P>
__global__ void __launch_bounds__(256) k_l2l_level(TArgs a, real* __restrict__ Lmom) {
    constexpr int T = MI<P>::T;
    __shared__ real bufA[2 * T], bufB[2 * T];
    __shared__ real cd[3][P + 1];
    __shared__ real binom[P + 1][P + 1];
    __shared__ short idx3[P + 1][P + 1][P + 1];
    __shared__ signed char kk[T][3];
    const int tid = threadIdx.x;
    const int64_t nd = a.lvl_begin + blockIdx.x;
    if (nd >= a.lvl_end) return;
    const int nc = a.nchild[nd];
    if (nc == 0) return;
    const int fc = a.child[nd];
    for (int k = tid; k < T; k += blockDim.x) {
        int x, y, z;
        decode_mi(k, x, y, z);
        idx3[x][y][z] = (short)k;
        kk[k][0] = (signed char)x;
        kk[k][1] = (signed char)y;
        kk[k][2] = (signed char)z;
    }
    for (int q = tid; q < (P + 1) * (P + 1); q += blockDim.x) {
        const int n = q / (P + 1), m = q - n * (P + 1);
        binom[n][m] = (real)kBinom[n][m];
    }
    for (int ci = 0; ci < nc; ++ci) {
        const int ch = fc + ci;
        __syncthreads();
        for (int k = tid; k < 2 * T; k += blockDim.x) bufA[k] = Lmom[nd * 2 * T + k];
        if (tid < 3) {
            const real d = (real)(a.ncenter[3 * nd + tid] - a.ncenter[3 * ch + tid]);
            real v = 1;
            for (int m = 0; m <= P; ++m) {
                cd[tid][m] = v;
                v *= d;
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int ax = 0; ax < 3; ++ax) {
            real* src = (ax == 1) ? bufB : bufA;
            real* dst = (ax == 1) ? bufA : bufB;
            for (int k = tid; k < T; k += blockDim.x) {
                const int k0 = kk[k][0], k1 = kk[k][1], k2 = kk[k][2];
                const int ka = kk[k][ax];
                const int top = P - (k0 + k1 + k2 - ka);  // largest index along ax with |.| <= P
                real sL = 0, sY = 0;
                for (int jv = ka; jv <= top; ++jv) {
                    const int jx = ax == 0 ? jv : k0, jy = ax == 1 ? jv : k1, jz = ax == 2 ? jv : k2;
                    const int jj = idx3[jx][jy][jz];
                    const real coef = binom[jv][ka] * cd[ax][jv - ka];
                    sL += coef * src[jj];
                    sY += coef * src[T + jj];
                }
                dst[k] = sL;
                dst[T + k] = sY;
            }
            __syncthreads();
        }
        for (int k = tid; k < 2 * T; k += blockDim.x) Lmom[(int64_t)ch * 2 * T + k] += bufB[k];
    }
}

// Far field at the quadrature nodes of every leaf (one block per leaf):
// Phi = sum_k L_k u^k, n . grad_y Phi = -sum_k L_k n . grad_u u^k, u = c - y,
// added to out (which k_p2p_T has written).
template <typename real, int P>
__global__ void __launch_bounds__(128) k_l2p(TArgs a, const typename V4<real>::t* __restrict__ yrel,
                                             const typename V4<real>::t* __restrict__ nrm,
                                             const real* __restrict__ Lmom) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    __shared__ real sL[2 * T];
    __shared__ signed char kk[T][3];
    const int64_t leaf = blockIdx.x;
    if (leaf >= a.n_leaves) return;
    const int nd = a.leaf_node[leaf];
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        int x, y, z;
        decode_mi(k, x, y, z);
        kk[k][0] = (signed char)x;
        kk[k][1] = (signed char)y;
        kk[k][2] = (signed char)z;
    }
    for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) sL[k] = Lmom[(int64_t)nd * 2 * T + k];
    __syncthreads();
    const int64_t q0 = (int64_t)a.nstart[nd] * a.K, q1 = (int64_t)a.nend[nd] * a.K;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const v4 A = yrel[q];
        const v4 n = nrm[q / a.K];
        const real u[3] = {-A.x, -A.y, -A.z};
        real pw[3][P + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pw[c][0] = 1;
#pragma unroll
            for (int m = 1; m <= P; ++m) pw[c][m] = pw[c][m - 1] * u[c];
        }
        real vL = 0, dL = 0, vY = 0, dY = 0;
        for (int k = 0; k < T; ++k) {
            const int x = kk[k][0], y = kk[k][1], z = kk[k][2];
            const real px = pw[0][x], py = pw[1][y], pz = pw[2][z];
            const real mono = px * py * pz;
            real dn = 0;  // n . grad_u u^k
            if (x) dn += n.x * real(x) * pw[0][x - 1] * py * pz;
            if (y) dn += n.y * real(y) * px * pw[1][y - 1] * pz;
            if (z) dn += n.z * real(z) * px * py * pw[2][z - 1];
            vL += sL[k] * mono;
            dL += sL[k] * dn;
            vY += sL[T + k] * mono;
            dY += sL[T + k] * dn;
        }
        a.out[4 * q] += (double)vL;
        a.out[4 * q + 1] -= (double)dL;
        a.out[4 * q + 2] += (double)vY;
        a.out[4 * q + 3] -= (double)dY;
    }
}

// Near field, transposed: one block per source leaf b; for every forward near
// entry (g, b) the 32 targets of g (offsets from the leaf centre, weights,
// panel) are staged in shared memory and every thread sums them at its
// quadrature node(s) of b, skipping the target's own panel (as the forward
// P2P does).  Writes out (4 per node, no 1/4pi).
template <typename real>
__global__ void __launch_bounds__(256) k_p2p_T(TArgs a, const typename V4<real>::t* __restrict__ xrel,
                                                const double* __restrict__ sT,
                                                const typename V4<real>::t* __restrict__ yrel,
                                                const typename V4<real>::t* __restrict__ nrm) {
    using v4 = typename V4<real>::t;
    __shared__ v4 sX[32];       // target - leaf centre, s_L
    __shared__ real sYw[32];    // s_Y
    __shared__ int sPan[32];    // target panel (-1: none)
    const int64_t leaf = blockIdx.x;
    if (leaf >= a.n_leaves) return;
    const int nd = a.leaf_node[leaf];
    const int nb = a.nbody[nd];
    const real kappa = (real)a.kappa;
    const real nkl = -kappa * real(1.4426950408889634);
    const int64_t q0 = (int64_t)a.nstart[nd] * a.K, q1 = (int64_t)a.nend[nd] * a.K;
    for (int64_t qb = q0; qb < q1; qb += blockDim.x) {  // chunks of the leaf's nodes
        const int64_t q = qb + threadIdx.x;
        const bool on = q < q1;
        const v4 A = yrel[on ? q : q0];
        const v4 n = nrm[(on ? q : q0) / a.K];
        const int64_t panel = (on ? q : q0) / a.K;
        real acc[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
        for (int64_t t = a.tn_off[nd]; t < a.tn_off[nd + 1]; ++t) {
            const int64_t e = a.tn_e[t];
            const int64_t g = a.near_group[e];
            const int64_t p0 = a.gstart[g], p1 = a.gend[g];
            const int gb = a.gbody[g];
            const bool lap = (nb == gb) && a.lap_body[gb];
            __syncthreads();
            if (threadIdx.x < 32) {
                const int64_t p = p0 + threadIdx.x;
                real ox, oy, oz;
                if (sizeof(real) == sizeof(float)) {
                    const float4 o = a.near4[e];
                    ox = (real)o.x;
                    oy = (real)o.y;
                    oz = (real)o.z;
                } else {
                    ox = (real)(a.ncenter[3 * nd] - a.gcenter[3 * g]);
                    oy = (real)(a.ncenter[3 * nd + 1] - a.gcenter[3 * g + 1]);
                    oz = (real)(a.ncenter[3 * nd + 2] - a.gcenter[3 * g + 2]);
                }
                v4 X = v4();
                real sy = 0;
                int pan = -1;
                if (p < p1) {
                    const v4 xr = xrel[p];
                    X.x = xr.x - ox;  // target relative to the leaf centre, as the forward r0
                    X.y = xr.y - oy;
                    X.z = xr.z - oz;
                    X.w = (real)sT[2 * p];
                    sy = (real)sT[2 * p + 1];
                    pan = (int)p;
                }
                sX[threadIdx.x] = X;
                sYw[threadIdx.x] = sy;
                sPan[threadIdx.x] = pan;
            }
            __syncthreads();
            if (!on) continue;
            real t0 = 0, t1 = 0, t2 = 0, t3 = 0;
            for (int i = 0; i < 32; ++i) {
                const v4 X = sX[i];
                if (sPan[i] < 0) continue;
                const real dx = X.x - A.x, dy = X.y - A.y, dz = X.z - A.z;  // x_i - y_s
                const real r2 = dx * dx + dy * dy + dz * dz;
                real ri = rsqrt_fast(r2);
                ri = (r2 > real(0) && sPan[i] != panel) ? ri : real(0);
                const real ri3 = ri * ri * ri;
                const real pd = n.x * dx + n.y * dy + n.z * dz;  // n_j . (x_i - y_s)
                if (lap) {
                    t0 += X.w * ri;
                    t1 += X.w * pd * ri3;
                }
                const real r = r2 * ri;
                const real ex = exp2_(nkl * r);
                t2 += sYw[i] * ex * ri;
                t3 += sYw[i] * (kappa * r + real(1)) * ex * pd * ri3;
            }
            kadd(acc[0], cmp[0], t0);
            kadd(acc[1], cmp[1], t1);
            kadd(acc[2], cmp[2], t2);
            kadd(acc[3], cmp[3], t3);
        }
        if (on)
            for (int k = 0; k < 4; ++k) a.out[4 * q + k] = (double)acc[k] + (double)cmp[k];
    }
}

}  // namespace pgb
