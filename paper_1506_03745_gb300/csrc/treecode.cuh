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
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "ds.cuh"
#include "pgb_internal.cuh"

namespace pgb {

struct __align__(16) ds4 {
    ds x, y, z, w;
};

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
template <>
struct V4<ds> {
    using t = ds4;
};

// Storage type of the kernels' inputs per arithmetic type: the
// double-single kernels read the FP64 product's data (source terms, target
// offsets, moments) and convert as they stage it.
template <typename C>
struct Store {
    using S = C;
};
template <>
struct Store<ds> {
    using S = double;
};
template <typename C>
__device__ __forceinline__ C to_c(typename Store<C>::S v) {
    return v;
}
template <>
__device__ __forceinline__ ds to_c<ds>(double v) {
    return ds_from_double(v);
}
template <typename C>
__device__ __forceinline__ typename V4<C>::t cvt4(const typename V4<typename Store<C>::S>::t& v) {
    return v;
}
template <>
__device__ __forceinline__ ds4 cvt4<ds>(const dbl4& v) {
    return ds4{ds_from_double(v.x), ds_from_double(v.y), ds_from_double(v.z), ds_from_double(v.w)};
}
__device__ __forceinline__ double to_dbl(float v) { return (double)v; }
__device__ __forceinline__ double to_dbl(double v) { return v; }
__device__ __forceinline__ double to_dbl(ds v) { return ds_to_double(v); }
// a double literal in the arithmetic type (split at compile time for ds)
template <typename C>
__device__ __forceinline__ C lit(double d) {
    return (C)d;
}
template <>
__device__ __forceinline__ ds lit<ds>(double d) {
    return ds_const(d);
}
// 1/n in the arithmetic type (n a compile-time constant after unrolling)
template <typename C>
__device__ __forceinline__ C inv_int(int n) {
    return C(1) / C(n);
}
template <>
__device__ __forceinline__ ds inv_int<ds>(int n) {
    return ds_const(1.0 / n);
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float exp_(float x) { return __expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
// 2^x (the P2P loop folds log2(e) into its constant) and 1/sqrt(x) of the
// P2P loop.  FP32: the SFU's approximate forms (relative error about 2^-22),
// one instruction each.  FP64: exp2_taylor and one Newton step on the SFU
// estimate (relative errors below 1e-14 and 1e-13), about a third of the FP64
// operations of the library's correctly rounded forms on a part whose FP64
// rate is 1/64 of its FP32 rate.
__device__ __forceinline__ float exp2_(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double exp2_(double x) { return exp2_taylor(x); }
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsqrt_fast(double x) { return rsqrt_nr<1>(x); }
__device__ __forceinline__ ds rsqrt_(ds x) { return ds_rsqrt(x); }
__device__ __forceinline__ ds rsqrt_fast(ds x) { return ds_rsqrt(x); }
__device__ __forceinline__ ds exp_(ds x) { return ds_exp(x); }
__device__ __forceinline__ ds exp2_(ds x) { return ds_exp2(x); }

// Neumaier-compensated accumulation s + c += v.
template <typename T>
__device__ __forceinline__ void kadd(T& s, T& c, T v) {
    T t = s + v;
    c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}
// double-single sums carry their own error term (c stays 0)
__device__ __forceinline__ void kadd(ds& s, ds&, ds v) { s = s + v; }

// c + a b: as written for FP32 / FP64 (the compiler contracts it), one fused
// double-single operation for ds
template <typename T>
__device__ __forceinline__ T madd(T a, T b, T c) {
    return c + a * b;
}
__device__ __forceinline__ ds madd(ds a, ds b, ds c) { return ds_fma(a, b, c); }
template <typename T>
constexpr bool is_ds = false;
template <>
constexpr bool is_ds<ds> = true;

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

// the run-time body mask of a product (all bodies without one)
__device__ __forceinline__ unsigned long long body_mask(const unsigned long long* m) { return m ? *m : ~0ull; }

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
    int src_active[PGB_MAX_BODIES];  // 0: the body's densities are all zero (skip)
    int all_active;                // every body active (the plain product): no per-node test
    unsigned long long tgt_mask;   // bit b: the rows of body b are used (other groups' items are skipped)
    int64_t g_lo, g_hi;            // only the groups g_lo <= g < g_hi (a rank's rows of a sharded product)
    // device copy of a further body mask, read at run time (a replayed
    // lockstep iteration: bit b clear = body b's rows and sources left out);
    // nullptr: none.  With it all_active is 0.
    const unsigned long long* bmask = nullptr;
    const float4* near4;           // per near entry: leaf centre - group centre, node id bits
    const float4* far4;            // per far entry: node centre - group centre, node id bits
    const int64_t* tile_off;       // per group: its P2P tiles [tile_off[g], tile_off[g+1])
    const float4* tile_d;          // per tile: leaf centre - group centre (FP32), first point (int bits)
    const int4* tile_m;            // per tile: leaf node, point count, flags (1 Laplace, 2 own panel), body
    // work items (a group's tiles / far entries in runs of p2p_item / m2p_item)
    int64_t n_pitems, n_fitems;
    const int64_t *pitem_off, *fitem_off;  // per group
    const int32_t *pitem_group, *fitem_group;
    int p2p_item, m2p_item;
    double *Up, *Uf;               // per item: 32 Laplace then 32 Yukawa partial sums (one per lane)
    // persistent launch: a grid smaller than the item count whose blocks take
    // items from these counters (zero before the launch); nullptr: one item per block
    unsigned long long *p2p_work, *m2p_work;
    int persist_blocks;            // grid of a persistent launch
};

// Item loop of a block: one item per block, or (persistent launch) items
// taken from a counter until none is left.  The barrier also keeps a block
// from reusing its shared memory while a warp still reads the last item.
__device__ __forceinline__ int64_t next_item(unsigned long long* work, int64_t cur, int64_t* slot) {
    if (!work) return cur < 0 ? (int64_t)blockIdx.x : INT64_MAX;
    __syncthreads();
    if (threadIdx.x == 0) *slot = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    return *slot;
}

// 16-byte vector of the arithmetic type (4 floats, 2 doubles, 2 double-singles),
// for loads of consecutive coefficients from shared memory.
template <typename real>
struct alignas(16) Vec16 {
    static constexpr int N = 16 / sizeof(real);
    real v[N];
};

// Far field of one node at R = target - node centre from its coefficients in
// the evaluation order (a = 0..P, b = 0..P-a, c = 0..P-a-b for S^(a,b,c)),
// S = R / r^2 and x = kappa r (the tables of farfield.cu):
//   U_Y = (e^{-x} / r) sum_p g_p(x) sum_{a+b+c=p} cY_abc S^(a,b,c),
//   U_L = (1 / r) sum_abc cL_abc S^(a,b,c),
// g_0 = 1, g_1 = -(1 + x), g_p = x^2 g_{p-2} - (2p - 1) g_{p-1}.  The monomials
// are formed in nested order, one product each, and summed per degree, so
// that a term costs one product and one multiply-add per kernel.
// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1, so
// that array indices formed from I are constants whatever the trip count
// (a plain unrolled loop nest is left partly rolled by the compiler at the
// higher orders, which moves the per-degree sums to local memory).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}
// index of S^(a,b,0) in the evaluation order of order P
__host__ __device__ constexpr int eval_index(int P, int a, int b) {
    int o = 0;
    for (int q = 0; q < a; ++q) o += (P - q + 1) * (P - q + 2) / 2;
    for (int q = 0; q < b; ++q) o += P - a - q + 1;
    return o;
}

template <typename real, int P, bool LAP>
__device__ __forceinline__ void far_eval(real Rx, real Ry, real Rz, real kappa, const real* __restrict__ cL,
                                         const real* __restrict__ cY, real& uL, real& uY) {
    using V = Vec16<real>;
    constexpr int VN = V::N;
    real r2;
    if constexpr (is_ds<real>) r2 = madd(Rx, Rx, madd(Ry, Ry, Rz * Rz));
    else r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const real ri = rsqrt_(r2);
    const real i2 = ri * ri;
    const real sx = Rx * i2, sy = Ry * i2, sz = Rz * i2;
    real acc[P + 1];
#pragma unroll
    for (int p = 0; p <= P; ++p) acc[p] = real(0);
    real aL = real(0);
    V qy, ql;
    real xa = real(1);
    if constexpr (is_ds<real> && P > 8) {
        // double-single above order 8: loops the compiler unrolls as it sees
        // fit (the full unroll of these long double-single bodies takes the
        // compiler minutes); the FP64-class residual product runs a few times
        // per solve
        int idx = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            real xy = xa;
#pragma unroll
            for (int b = 0; b <= P - a; ++b) {
                real t = xy;
#pragma unroll
                for (int c = 0; c <= P - a - b; ++c) {
                    if (idx % VN == 0) {
                        qy = *reinterpret_cast<const V*>(cY + idx);
                        if (LAP) ql = *reinterpret_cast<const V*>(cL + idx);
                    }
                    acc[a + b + c] = madd(qy.v[idx % VN], t, acc[a + b + c]);
                    if (LAP) aL = madd(ql.v[idx % VN], t, aL);
                    ++idx;
                    if (c < P - a - b) t = t * sz;
                }
                if (b < P - a) xy = xy * sy;
            }
            if (a < P) xa = xa * sx;
        }
    } else {
    static_for<0, P + 1>([&](auto A) {
        constexpr int a = decltype(A)::value;
        real xy = xa;
        static_for<0, P - a + 1>([&](auto Bc) {
            constexpr int b = decltype(Bc)::value;
            constexpr int i0 = eval_index(P, a, b);
            real t = xy;
            static_for<0, P - a - b + 1>([&](auto Cc) {
                constexpr int c = decltype(Cc)::value;
                constexpr int idx = i0 + c;
                if constexpr (idx % VN == 0) {
                    qy = *reinterpret_cast<const V*>(cY + idx);
                    if constexpr (LAP) ql = *reinterpret_cast<const V*>(cL + idx);
                }
                acc[a + b + c] = madd(qy.v[idx % VN], t, acc[a + b + c]);
                if constexpr (LAP) aL = madd(ql.v[idx % VN], t, aL);
                if constexpr (c < P - a - b) t = t * sz;
            });
            if constexpr (b < P - a) xy = xy * sy;
        });
        if constexpr (a < P) xa = xa * sx;
    });
    }
    const real r = r2 * ri;
    const real x = kappa * r;
    const real x2 = x * x;
    real u = acc[0];
    real gm2 = real(1), gm1 = -(x + real(1));
    if (P >= 1) u = madd(gm1, acc[P >= 1 ? 1 : 0], u);
#pragma unroll
    for (int p = 2; p <= P; ++p) {
        const real g = madd(x2, gm2, -(real(2 * p - 1) * gm1));
        u = madd(g, acc[p], u);
        gm2 = gm1;
        gm1 = g;
    }
    uY = (exp_(-x) * ri) * u;
    uL = LAP ? aL * ri : real(0);
}

// K-point sums of one tile of source points for one target (relative position
// r0 = target - leaf centre).  With OWN, points of the target's own panel
// (indices [own_lo, own_hi)) are skipped.
template <typename real, bool LAP, bool OWN>
__device__ __forceinline__ void p2p_tile(const typename V4<real>::t* sA, const typename V4<real>::t* sB, int cnt,
                                         int64_t t, int64_t own_lo, int64_t own_hi, real r0x, real r0y, real r0z,
                                         real kappa, real& sumL, real& sumY) {
    using v4 = typename V4<real>::t;
    const real nkl = -kappa * lit<real>(1.4426950408889634);  // -kappa log2(e)
    real sL2 = 0, sY2 = 0;  // second accumulator pair: two independent chains
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
        const v4 A = sA[j], B = sB[j];
        const real dx = r0x - A.x, dy = r0y - A.y, dz = r0z - A.z;
        real r2;
        if constexpr (is_ds<real>) r2 = madd(dx, dx, madd(dy, dy, dz * dz));
        else r2 = dx * dx + dy * dy + dz * dz;
        // a quadrature node of another panel never coincides with a target
        // centroid on a valid (non-overlapping) mesh; only the target's own
        // panel, in the leaf that holds the group, needs the exclusion
        real ri = rsqrt_fast(r2);
        if (OWN) ri = (r2 > real(0) && !(t + j >= own_lo && t + j < own_hi)) ? ri : real(0);
        real pd;
        if constexpr (is_ds<real>) pd = madd(B.x, dx, madd(B.y, dy, B.z * dz));
        else pd = B.x * dx + B.y * dy + B.z * dz;
        const real tt = pd * (ri * ri);
        const real r = r2 * ri;
        const real ex = exp2_(nkl * r);
        if constexpr (is_ds<real>) {
            const ds yw = madd(-madd(kappa, r, ds(1)), tt, B.w);  // B.w - (kappa r + 1) tt
            if (j & 1) {
                if (LAP) sL2 = madd(ri, A.w - tt, sL2);
                sY2 = madd(ex * ri, yw, sY2);
            } else {
                if (LAP) sumL = madd(ri, A.w - tt, sumL);
                sumY = madd(ex * ri, yw, sumY);
            }
        } else {
            const real gg = kappa * r + real(1);
            if (j & 1) {
                if (LAP) sL2 += ri * (A.w - tt);
                sY2 += (ex * ri) * (B.w - gg * tt);
            } else {
                if (LAP) sumL += ri * (A.w - tt);
                sumY += (ex * ri) * (B.w - gg * tt);
            }
        }
    }
    sumL += sL2;
    sumY += sY2;
}

// One block of NW warps per target group (32 targets, one per lane): the
// warps share out the near leaves (P2P) and far nodes (M2P) of the group's
// lists round robin, and their partial sums are combined in warp order.
template <typename real>
__device__ __forceinline__ void entry_offset(const EvalArgs& a, int64_t e, bool is_far, double gc0, double gc1,
                                             double gc2, int& nd, real& ox, real& oy, real& oz);
template <>
__device__ __forceinline__ void entry_offset<float>(const EvalArgs& a, int64_t e, bool is_far, double, double, double,
                                                    int& nd, float& ox, float& oy, float& oz) {
    const float4 q = is_far ? a.far4[e] : a.near4[e];
    nd = __float_as_int(q.w);
    ox = q.x;
    oy = q.y;
    oz = q.z;
}
template <>
__device__ __forceinline__ void entry_offset<double>(const EvalArgs& a, int64_t e, bool is_far, double gc0, double gc1,
                                                     double gc2, int& nd, double& ox, double& oy, double& oz) {
    nd = is_far ? a.far_l[e] : a.near_l[e];
    ox = a.ncenter[3 * nd] - gc0;
    oy = a.ncenter[3 * nd + 1] - gc1;
    oz = a.ncenter[3 * nd + 2] - gc2;
}

// Partial sums of the NW warps of a block combined in warp order (each warp
// carries a compensated pair per kernel) and stored per lane for the item.
template <typename real, int NW>
__device__ __forceinline__ void store_item(real (*red)[4][32], int w, int lane, real UL, real cL, real UY, real cY,
                                           double* out) {
    red[w][0][lane] = UL;
    red[w][1][lane] = cL;
    red[w][2][lane] = UY;
    red[w][3][lane] = cY;
    __syncthreads();
    if (w == 0) {
        real sL = 0, eL = 0, sY = 0, eY = 0;
        for (int k = 0; k < NW; ++k) {
            kadd(sL, eL, red[k][0][lane]);
            kadd(sL, eL, red[k][1][lane]);
            kadd(sY, eY, red[k][2][lane]);
            kadd(sY, eY, red[k][3][lane]);
        }
        out[lane] = to_dbl(sL) + to_dbl(eL);
        out[32 + lane] = to_dbl(sY) + to_dbl(eY);
    }
}

// P2P: one block of NW warps per work item, i.e. up to p2p_item source tiles
// (up to 32 quadrature points of one near leaf each) of one target group (32
// targets, one per lane); the tiles are dealt round robin to the warps, the
// next tile prefetched into registers.  The item's partial sums go to Up.
// The source terms come in the arithmetic type (for double-single, split
// once per product by k_src_to_ds); the targets in the storage type.
template <typename real, int NW>
__global__ void __launch_bounds__(NW * 32) k_p2p(EvalArgs a, const typename V4<real>::t* __restrict__ src,
                                                 const typename V4<typename Store<real>::S>::t* __restrict__ xrel) {
    using S = typename Store<real>::S;  // storage type of the inputs
    using v4 = typename V4<real>::t;
    using s4 = typename V4<S>::t;
    __shared__ v4 sA[NW][32], sB[NW][32];
    __shared__ real red[NW][4][32];
    __shared__ int64_t s_item;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long dm = body_mask(a.bmask);
    for (int64_t it = next_item(a.p2p_work, -1, &s_item); it < a.n_pitems; it = next_item(a.p2p_work, it, &s_item)) {
    const int64_t g = a.pitem_group[it];
    if (!(((a.tgt_mask & dm) >> a.gbody[g]) & 1ull) || g < a.g_lo || g >= a.g_hi) continue;  // rows not used (block-uniform)
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    const int64_t p = p0 + lane;
    const bool active = p < p1;
    const s4 xr = active ? xrel[p] : xrel[p0];
    const double gc0 = a.gcenter[3 * g], gc1 = a.gcenter[3 * g + 1], gc2 = a.gcenter[3 * g + 2];
    const real kappa = to_c<real>((S)a.kappa);
    const int64_t own_lo = p * a.K, own_hi = own_lo + a.K;
    real UL = 0, cL = 0, UY = 0, cY = 0;
    const int64_t tb = a.tile_off[g] + (it - a.pitem_off[g]) * a.p2p_item;
    const int64_t t1 = min(a.tile_off[g + 1], tb + a.p2p_item);
    int64_t t = tb + w;
    v4 pa = v4(), pb = v4();
    int4 m = make_int4(0, 0, 0, 0);
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < t1) {
        d = a.tile_d[t];
        m = a.tile_m[t];
        if (lane < m.y) {
            const int64_t q = (int64_t)__float_as_int(d.w) + lane;
            pa = src[2 * q];
            pb = src[2 * q + 1];
        }
    }
    while (t < t1) {
        const int cnt = m.y, flags = m.z | (a.src_active[m.w] && ((dm >> m.w) & 1ull) ? 0 : 4);
        const int64_t first = (int64_t)__float_as_int(d.w);
        // target relative to the leaf centre: FP32 from the tile's offset,
        // else formed in FP64 (and split for double-single)
        real r0x, r0y, r0z;
        if constexpr (sizeof(real) == sizeof(float)) {
            r0x = xr.x - (real)d.x;
            r0y = xr.y - (real)d.y;
            r0z = xr.z - (real)d.z;
        } else {
            const int nd = m.x;
            const S ox = (S)(a.ncenter[3 * nd] - gc0);
            const S oy = (S)(a.ncenter[3 * nd + 1] - gc1);
            const S oz = (S)(a.ncenter[3 * nd + 2] - gc2);
            r0x = to_c<real>(xr.x - ox);
            r0y = to_c<real>(xr.y - oy);
            r0z = to_c<real>(xr.z - oz);
        }
        __syncwarp();
        if (lane < cnt) {
            sA[w][lane] = pa;
            sB[w][lane] = pb;
        }
        __syncwarp();
        t += NW;
        if (t < t1) {  // prefetch this warp's next tile
            d = a.tile_d[t];
            m = a.tile_m[t];
            if (lane < m.y) {
                const int64_t q = (int64_t)__float_as_int(d.w) + lane;
                pa = src[2 * q];
                pb = src[2 * q + 1];
            }
        }
        real sumL = 0, sumY = 0;
        if (flags & 4) {
            // source body without density in this product (imposed-boundary terms)
        } else if (flags & 2) {
            if (flags & 1) p2p_tile<real, true, true>(sA[w], sB[w], cnt, first, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
            else p2p_tile<real, false, true>(sA[w], sB[w], cnt, first, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
        } else {
            if (flags & 1) p2p_tile<real, true, false>(sA[w], sB[w], cnt, first, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
            else p2p_tile<real, false, false>(sA[w], sB[w], cnt, first, own_lo, own_hi, r0x, r0y, r0z, kappa, sumL, sumY);
        }
        kadd(UL, cL, sumL);
        kadd(UY, cY, sumY);
    }
    store_item<real, NW>(red, w, lane, UL, cL, UY, cY, a.Up + 64 * it);
    }
}

// M2P: one block of NW warps per work item, i.e. up to m2p_item far entries of
// one target group; the nodes go round robin to the warps with the next
// node's far-field coefficients (k_far_coef) prefetched.  The item's partial
// sums go to Uf.
template <typename real, int P, int NW>
__global__ void __launch_bounds__(NW * 32) k_m2p(EvalArgs a,
                                                 const typename V4<typename Store<real>::S>::t* __restrict__ xrel,
                                                 const real* __restrict__ far) {
    using S = typename Store<real>::S;  // storage type of the inputs
    using s4 = typename V4<S>::t;
    constexpr int TP = n_terms_pad(P);
    // orders up to 8: the next node's coefficients are prefetched into
    // registers (MW words per lane) while the current one is evaluated;
    // above, they are loaded into shared memory when needed
    constexpr bool BIG = P > 8;
    constexpr int MW = BIG ? 1 : (2 * TP + 31) / 32;
    __shared__ __align__(16) real sM[NW][2 * TP];
    __shared__ real red[NW][4][32];
    __shared__ int64_t s_item;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long dm = body_mask(a.bmask);
    for (int64_t it = next_item(a.m2p_work, -1, &s_item); it < a.n_fitems; it = next_item(a.m2p_work, it, &s_item)) {
    const int64_t g = a.fitem_group[it];
    if (!(((a.tgt_mask & dm) >> a.gbody[g]) & 1ull) || g < a.g_lo || g >= a.g_hi) continue;  // rows not used (block-uniform)
    const int64_t p0 = a.gstart[g], p1 = a.gend[g];
    const int64_t p = p0 + lane;
    const bool active = p < p1;
    const s4 xr = active ? xrel[p] : xrel[p0];
    const double gc0 = a.gcenter[3 * g], gc1 = a.gcenter[3 * g + 1], gc2 = a.gcenter[3 * g + 2];
    const int gb = a.gbody[g];
    const real kappa = to_c<real>((S)a.kappa);
    real UL = 0, cL = 0, UY = 0, cY = 0;
    const int64_t fb = a.far_off[g] + (it - a.fitem_off[g]) * a.m2p_item;
    const int64_t f1 = min(a.far_off[g + 1], fb + a.m2p_item);
    auto seek = [&](int64_t ee) -> int64_t {  // next active entry of this warp
        if (a.all_active) return ee;
        while (ee < f1) {
            int nn;
            S qx, qy, qz;
            entry_offset<S>(a, ee, true, gc0, gc1, gc2, nn, qx, qy, qz);
            if (a.src_active[a.nbody[nn]] && ((dm >> a.nbody[nn]) & 1ull)) return ee;
            ee += NW;
        }
        return ee;
    };
    real pm[MW];
    int nd = -1;
    S ox = 0, oy = 0, oz = 0;
    int64_t e = seek(fb + w);
    if (e < f1) {
        entry_offset<S>(a, e, true, gc0, gc1, gc2, nd, ox, oy, oz);
        if constexpr (!BIG) {
#pragma unroll
            for (int q = 0; q < MW; ++q) {
                const int k = lane + 32 * q;
                pm[q] = k < 2 * TP ? far[(int64_t)nd * 2 * TP + k] : real(0);
            }
        }
    }
    while (e < f1) {
        __syncwarp();
        if constexpr (BIG) {
            for (int k = lane; k < 2 * TP; k += 32) sM[w][k] = far[(int64_t)nd * 2 * TP + k];
        } else {
#pragma unroll
            for (int q = 0; q < MW; ++q) {
                const int k = lane + 32 * q;
                if (k < 2 * TP) sM[w][k] = pm[q];
            }
        }
        __syncwarp();
        const bool lap = (a.nbody[nd] == gb) && a.lap_body[gb];
        const real Rx = to_c<real>(xr.x - ox), Ry = to_c<real>(xr.y - oy), Rz = to_c<real>(xr.z - oz);
        e = seek(e + NW);
        if (e < f1) {  // the next node (its coefficients prefetched up to order 8)
            entry_offset<S>(a, e, true, gc0, gc1, gc2, nd, ox, oy, oz);
            if constexpr (!BIG) {
#pragma unroll
                for (int q = 0; q < MW; ++q) {
                    const int k = lane + 32 * q;
                    pm[q] = k < 2 * TP ? far[(int64_t)nd * 2 * TP + k] : real(0);
                }
            }
        }
        real uL, uY;
        if (lap) far_eval<real, P, true>(Rx, Ry, Rz, kappa, sM[w], sM[w] + TP, uL, uY);
        else far_eval<real, P, false>(Rx, Ry, Rz, kappa, sM[w], sM[w] + TP, uL, uY);
        kadd(UL, cL, uL);
        kadd(UY, cY, uY);
    }
    store_item<real, NW>(red, w, lane, UL, cL, UY, cY, a.Uf + 64 * it);
    }
}

struct UpArgs {
    int64_t n_leaves;
    const int32_t *leaf_node, *nstart, *nend, *child, *nchild, *nbody;
    int src_active[PGB_MAX_BODIES];
    const unsigned long long* bmask = nullptr;  // as EvalArgs::bmask
    const double* ncenter;
    int K;
    int64_t lvl_begin, lvl_end;  // node ids of one level (unused by k_upward)
    int p2m_grid;                // > 0: P2M over at most this many blocks (leaves strided)
    int64_t n_nodes;             // k_far_coef: every node
    const void* far_tab;         // its table (farfield.cu) in the arithmetic type
    void* far;                   // its output: 2 * n_terms_pad(P) coefficients per node
    const int32_t* parent;       // k_upward: parent of every node (-1 at a body's root)
    int* arrive;                 // k_upward: per node, children finished (zero between launches)
};
// a source body of the upward pass is used (its densities are not all zero
// and the run-time mask keeps it)
__device__ __forceinline__ bool body_on(const UpArgs& a, int b) {
    return a.src_active[b] && (!a.bmask || ((*a.bmask >> b) & 1ull));
}


// C(n, m) for n, m <= 15 (0 for m > n), by Pascal's rule at compile time
struct BinomTable {
    double v[16][16];
    __host__ __device__ constexpr BinomTable() : v() {
        for (int n = 0; n < 16; ++n) {
            v[n][0] = 1.0;
            for (int m = 1; m <= n; ++m) v[n][m] = v[n - 1][m - 1] + (m < n ? v[n - 1][m] : 0.0);
        }
    }
};
__device__ const BinomTable kBinomTable = BinomTable();

__device__ __constant__ const int kBinom[9][9] = {
    {1, 0, 0, 0, 0, 0, 0, 0, 0},      {1, 1, 0, 0, 0, 0, 0, 0, 0},      {1, 2, 1, 0, 0, 0, 0, 0, 0},
    {1, 3, 3, 1, 0, 0, 0, 0, 0},      {1, 4, 6, 4, 1, 0, 0, 0, 0},      {1, 5, 10, 10, 5, 1, 0, 0, 0},
    {1, 6, 15, 20, 15, 6, 1, 0, 0},   {1, 7, 21, 35, 35, 21, 7, 1, 0}, {1, 8, 28, 56, 70, 56, 28, 8, 1}};

// Degree a + b + c of the evaluation-order index j (a, then b, then c).
__device__ __forceinline__ int eval_degree(int j, int P) {
    int a = 0;
    for (;; ++a) {
        const int n = (P - a + 1) * (P - a + 2) / 2;
        if (j < n) break;
        j -= n;
    }
    int b = 0;
    for (;; ++b) {
        const int n = P - a - b + 1;
        if (j < n) break;
        j -= n;
    }
    return a + b + j;
}

// Nonzero entries of one output row of the far-field tables: a Yukawa
// output of degree p takes the moments of degrees p, p + 2, ..., P, a Laplace
// output those of degree p.
__host__ __device__ constexpr int far_row_nnz(int p, int P) {
    int n = (p + 1) * (p + 2) / 2;  // Laplace
    for (int q = p; q <= P; q += 2) n += (q + 1) * (q + 2) / 2;
    return n;
}
// Packed table size, and the offset of the first row of degree p (rows in
// the graded order of the moments).
__host__ __device__ constexpr int far_pack_offset(int p, int P) {
    int o = 0;
    for (int q = 0; q < p; ++q) o += (q + 1) * (q + 2) / 2 * far_row_nnz(q, P);
    return o;
}

// Far-field coefficients of every node of an active body from its moments
// (farfield.cu).  The table comes packed: per output row in the graded order,
// its Yukawa entries over the moments of degrees p, p + 2, ... then its
// Laplace entries over degree p (far_pack_offset, far_row_nnz); it is staged
// in shared memory once per block.  The block then takes nodes in turn: the
// node's moments go to shared memory, each thread forms outputs (its row of
// the packed table against the moments) and writes them in the evaluation
// order of far_eval.  Output per node: Laplace then Yukawa, each padded with
// zeros.
template <typename real, int P>
__global__ void __launch_bounds__(128) k_far_coef(UpArgs a, const real* __restrict__ mom) {
    constexpr int T = MI<P>::T;
    constexpr int TP = n_terms_pad(P);
    constexpr int NNZ = far_pack_offset(P + 1, P);
    extern __shared__ __align__(16) unsigned char far_smem[];
    real* tab = reinterpret_cast<real*>(far_smem);
    real* sm = tab + ((NNZ + 3) & ~3);
    const real* __restrict__ gtab = (const real*)a.far_tab;
    for (int k = threadIdx.x; k < NNZ; k += blockDim.x) tab[k] = gtab[k];
    real* __restrict__ far = (real*)a.far;
    for (int64_t nd = blockIdx.x; nd < a.n_nodes; nd += gridDim.x) {
        if (!body_on(a, a.nbody[nd])) continue;  // block-uniform
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) sm[k] = mom[nd * 2 * T + k];
        for (int k = T + threadIdx.x; k < TP; k += blockDim.x) {  // padding
            far[nd * 2 * TP + k] = real(0);
            far[nd * 2 * TP + TP + k] = real(0);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < T; j += blockDim.x) {
            int x, y, z;
            decode_mi(j, x, y, z);
            const int p = x + y + z;
            const int g0 = p * (p + 1) * (p + 2) / 6;  // first graded index of degree p
            const real* row = tab + far_pack_offset(p, P) + (j - g0) * far_row_nnz(p, P);
            real aY = 0, aL = 0;
            int e = 0;
            for (int q = p; q <= P; q += 2) {
                const int k0 = q * (q + 1) * (q + 2) / 6, k1 = k0 + (q + 1) * (q + 2) / 2;
                for (int k = k0; k < k1; ++k) aY += row[e++] * sm[T + k];
            }
            for (int k = g0; k < g0 + (p + 1) * (p + 2) / 2; ++k) aL += row[e++] * sm[k];
            // evaluation-order index of (x, y, z): a = x, b = y, c = z
            int ev = 0;
            for (int aa = 0; aa < x; ++aa) ev += (P - aa + 1) * (P - aa + 2) / 2;
            ev += y * (P - x + 1) - y * (y - 1) / 2 + z;
            far[nd * 2 * TP + ev] = aL;
            far[nd * 2 * TP + TP + ev] = aY;
        }
    }
}

template <typename real, int P>
constexpr size_t far_coef_smem() {
    return sizeof(real) * (((far_pack_offset(P + 1, P) + 3) & ~3) + 2 * MI<P>::T);
}

// Orders above 8, where the packed table no longer fits shared memory: the
// table is read from global memory (L2-resident) and each of its entries
// serves NB nodes, whose moments the block stages in shared memory; a
// thread forms output rows j (sums in the order of k_far_coef) for all NB
// nodes.  Inactive nodes in a block get no output.
template <typename real, int P, int NB>
__global__ void __launch_bounds__(128) k_far_big(UpArgs a, const real* __restrict__ mom) {
    constexpr int T = MI<P>::T;
    constexpr int TP = n_terms_pad(P);
    extern __shared__ __align__(16) unsigned char far_smem[];
    real(*sm)[2 * T] = reinterpret_cast<real(*)[2 * T]>(far_smem);
    const real* __restrict__ tab = (const real*)a.far_tab;
    real* __restrict__ far = (real*)a.far;
    for (int64_t n0 = (int64_t)blockIdx.x * NB; n0 < a.n_nodes; n0 += (int64_t)gridDim.x * NB) {
        const int nn = (int)min((int64_t)NB, a.n_nodes - n0);
        bool act[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) act[i] = i < nn && body_on(a, a.nbody[n0 + i]);
        __syncthreads();
        for (int q = threadIdx.x; q < NB * 2 * T; q += blockDim.x) {
            const int i = q / (2 * T), k = q - i * 2 * T;
            sm[i][k] = act[i] ? mom[(n0 + i) * 2 * T + k] : real(0);
        }
        if constexpr (TP > T) {
            for (int q = threadIdx.x; q < NB * (TP - T); q += blockDim.x) {  // padding
                const int i = q / (TP - T), k = T + q - i * (TP - T);
                if (act[i]) {
                    far[(n0 + i) * 2 * TP + k] = real(0);
                    far[(n0 + i) * 2 * TP + TP + k] = real(0);
                }
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < T; j += blockDim.x) {
            int x, y, z;
            decode_mi(j, x, y, z);
            const int p = x + y + z;
            const int g0 = p * (p + 1) * (p + 2) / 6;
            const real* row = tab + far_pack_offset(p, P) + (int64_t)(j - g0) * far_row_nnz(p, P);
            real aY[NB], aL[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) aY[i] = aL[i] = real(0);
            int e = 0;
            for (int q = p; q <= P; q += 2) {
                const int k0 = q * (q + 1) * (q + 2) / 6, k1 = k0 + (q + 1) * (q + 2) / 2;
                for (int k = k0; k < k1; ++k) {
                    const real t = row[e++];
#pragma unroll
                    for (int i = 0; i < NB; ++i) aY[i] += t * sm[i][T + k];
                }
            }
            for (int k = g0; k < g0 + (p + 1) * (p + 2) / 2; ++k) {
                const real t = row[e++];
#pragma unroll
                for (int i = 0; i < NB; ++i) aL[i] += t * sm[i][k];
            }
            int ev = 0;
            for (int aa = 0; aa < x; ++aa) ev += (P - aa + 1) * (P - aa + 2) / 2;
            ev += y * (P - x + 1) - y * (y - 1) / 2 + z;
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (act[i]) {
                    far[(n0 + i) * 2 * TP + ev] = aL[i];
                    far[(n0 + i) * 2 * TP + TP + ev] = aY[i];
                }
        }
    }
}

// FP32 far-field coefficients: one block per (node, table), one thread per
// output j of the evaluation order (blockDim = n_terms_pad(P) rounded up to
// 32), E[j] = sum_k M[k] tab[k][j] over the table transposed and padded
// (tab[k][j], rows of far_tr(P) columns, Yukawa then Laplace, zeros off the
// degree pattern): the warp's 32 threads read consecutive entries of a row
// (L1-resident after first use) against the node's moments broadcast from
// shared memory.  The problem is small (nodes x 2 T outputs), so the work is
// spread over as many warps as it has outputs to hide the load latency.
__host__ __device__ constexpr int far_tr(int P) { return (n_terms_pad(P) + 31) & ~31; }
template <int P>
__global__ void __launch_bounds__(256) k_far_f32(UpArgs a, const float* __restrict__ mom) {
    constexpr int T = MI<P>::T;
    constexpr int TP = n_terms_pad(P);
    constexpr int TR = far_tr(P);
    __shared__ float m[T];
    const int64_t nd = blockIdx.x;
    const int t = blockIdx.y;  // 0: Yukawa (moments T .. 2T-1), 1: Laplace
    if (!body_on(a, a.nbody[nd])) return;  // block-uniform
    for (int k = threadIdx.x; k < T; k += blockDim.x) m[k] = mom[nd * 2 * T + (t == 0 ? T : 0) + k];
    __syncthreads();
    const int j = threadIdx.x;
    const float* __restrict__ tab = (const float*)a.far_tab + (size_t)t * T * TR + j;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 8
    for (int k = 0; k + 1 < T; k += 2) {
        acc0 += m[k] * __ldg(tab + (size_t)k * TR);
        acc1 += m[k + 1] * __ldg(tab + (size_t)(k + 1) * TR);
    }
    if (T & 1) acc0 += m[T - 1] * __ldg(tab + (size_t)(T - 1) * TR);
    if (j < TP) ((float*)a.far)[nd * 2 * TP + (t == 0 ? TP : 0) + j] = acc0 + acc1;
}

// ---------------------------------------------------------------- fused upward pass
// The upward pass in one launch: each block takes leaves (P2M), and a node's
// moment shift runs in the block whose child finished last (a counter per
// node; the last of nchild increments goes on up, the others stop), so the
// tree is climbed without a launch or a barrier per level and no block waits
// for another.  Writers fence before their increment; the climbing block
// fences after it and reads the children's moments from L2 (ld.global.cg).
// The far-field coefficients follow in k_far_coef.
// children shifted at once by the moment shift: all eight while their two
// buffers take at most 64 KB, else half as many per halving
__host__ __device__ constexpr int up_child_batch(int bytes, int T) {
    int cb = 8;
    while (cb > 1 && 2 * cb * 2 * T * bytes > 64 * 1024) cb /= 2;
    return cb;
}
template <typename real, int P>
struct UpShared {
    static constexpr int T = MI<P>::T;
    static constexpr int TD = P * (P + 1) * (P + 2) / 6 > 0 ? P * (P + 1) * (P + 2) / 6 : 1;
    static constexpr int CB = up_child_batch((int)sizeof(real), T);
    struct P2M {
        real pw[128][3][P + 1];
        real sq[128][5];
        real sd[3][TD];
    };
    struct M2M {
        real bufA[CB][2 * T], bufB[CB][2 * T];
        real cd[CB][3][P + 1];
    };
    union {
        P2M p;
        M2M m;
    } u;
    real binom[P + 1][P + 1];
    short idx3[P + 1][P + 1][P + 1];
    signed char kk[T][3];
    int next;
};

template <typename real>
__device__ __forceinline__ real ld_cg(const real* p) {
    return __ldcg(p);
}
__device__ __forceinline__ ds ld_cg(const ds* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return ds(v.x, v.y);
}
// a double in the arithmetic type
template <typename real>
__device__ __forceinline__ real from_dbl(double v) {
    return (real)v;
}
template <>
__device__ __forceinline__ ds from_dbl<ds>(double v) {
    return ds_from_double(v);
}

// P2M of node nd (a leaf) into mom[nd]: the moments about its centre,
// u = c - y, one thread per multi-index k (two when T > 128).  The
// double-layer part is split off:
//   M_k = sum_s q_s u^k + sum_a k_a D_a[k - e_a],  D_a[k'] = sum_s p_{s,a} u^{k'},
// so each (point, k) costs one monomial (two products of cached powers) and
// five multiply-adds; the D_a (|k'| <= P - 1) meet the q sums in shared memory.
template <typename real, int P>
__device__ __forceinline__ void up_p2m(const UpArgs& a, int nd, const typename V4<real>::t* __restrict__ src,
                                       real* __restrict__ mom, UpShared<real, P>& sh) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    constexpr int H = (T + 127) / 128;  // multi-indices per thread
    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)a.nstart[nd] * a.K, s1 = (int64_t)a.nend[nd] * a.K;
    int kx[H], ky[H], kz[H];
    bool on[H], low[H];
    real qL[H], qY[H], dx[H], dy[H], dz[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int k = tid + 128 * h;
        on[h] = k < T;
        kx[h] = ky[h] = kz[h] = 0;
        if (on[h]) {
            kx[h] = sh.kk[k][0];
            ky[h] = sh.kk[k][1];
            kz[h] = sh.kk[k][2];
        }
        low[h] = on[h] && kx[h] + ky[h] + kz[h] < P;
        qL[h] = qY[h] = dx[h] = dy[h] = dz[h] = real(0);
    }
    for (int64_t t = s0; t < s1; t += 128) {
        const int cnt = (int)min((int64_t)128, s1 - t);
        __syncthreads();
        if (tid < cnt) {
            const v4 A = src[2 * (t + tid)], B = src[2 * (t + tid) + 1];
            const real u[3] = {-A.x, -A.y, -A.z};
            for (int q = 0; q < 3; ++q) {
                real v = 1;
                for (int m = 0; m <= P; ++m) {
                    sh.u.p.pw[tid][q][m] = v;
                    v = v * u[q];
                }
            }
            sh.u.p.sq[tid][0] = A.w;
            sh.u.p.sq[tid][1] = B.w;
            sh.u.p.sq[tid][2] = B.x;
            sh.u.p.sq[tid][3] = B.y;
            sh.u.p.sq[tid][4] = B.z;
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (!on[h]) continue;
            for (int j = 0; j < cnt; ++j) {
                const real mono = sh.u.p.pw[j][0][kx[h]] * sh.u.p.pw[j][1][ky[h]] * sh.u.p.pw[j][2][kz[h]];
                qL[h] += sh.u.p.sq[j][0] * mono;
                qY[h] += sh.u.p.sq[j][1] * mono;
                if (low[h]) {
                    dx[h] += sh.u.p.sq[j][2] * mono;
                    dy[h] += sh.u.p.sq[j][3] * mono;
                    dz[h] += sh.u.p.sq[j][4] * mono;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < H; ++h)
        if (low[h]) {
            const int k = tid + 128 * h;
            sh.u.p.sd[0][k] = dx[h];
            sh.u.p.sd[1][k] = dy[h];
            sh.u.p.sd[2][k] = dz[h];
        }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < H; ++h) {
        if (!on[h]) continue;
        const int k = tid + 128 * h;
        real dl = 0;
        if (kx[h]) dl += real(kx[h]) * sh.u.p.sd[0][sh.idx3[kx[h] - 1][ky[h]][kz[h]]];
        if (ky[h]) dl += real(ky[h]) * sh.u.p.sd[1][sh.idx3[kx[h]][ky[h] - 1][kz[h]]];
        if (kz[h]) dl += real(kz[h]) * sh.u.p.sd[2][sh.idx3[kx[h]][ky[h]][kz[h] - 1]];
        mom[(int64_t)nd * 2 * T + k] = qL[h] + dl;
        mom[(int64_t)nd * 2 * T + T + k] = qY[h] + dl;
    }
}

// Moment shift of node nd from its (at most eight) children,
// M_k(c) = sum_{j<=k} C(k,j) (c - c_child)^{k-j} M_j(c_child): the shift is
// separable, so it is applied as three one-axis passes x, y, z, each output
// summing at most P+1 terms; CB children are shifted at once, and the results
// summed in child order.  The children's moments are read from L2.
template <typename real, int P>
__device__ __forceinline__ void up_m2m(const UpArgs& a, int nd, real* __restrict__ mom, UpShared<real, P>& sh) {
    constexpr int T = MI<P>::T;
    constexpr int CB = UpShared<real, P>::CB;
    constexpr int HO = (2 * T + 127) / 128;  // outputs per thread
    const int tid = threadIdx.x;
    const int nc = a.nchild[nd];
    const int fc = a.child[nd];
    real acc[HO];
#pragma unroll
    for (int h = 0; h < HO; ++h) acc[h] = real(0);
    for (int c0 = 0; c0 < nc; c0 += CB) {
        const int nb = min(CB, nc - c0);
        __syncthreads();
        for (int q = tid; q < nb * 2 * T; q += blockDim.x) {
            const int ci = q / (2 * T), k = q - ci * 2 * T;
            sh.u.m.bufA[ci][k] = ld_cg(mom + (int64_t)(fc + c0 + ci) * 2 * T + k);
        }
        if (tid < 3 * nb) {
            const int ci = tid / 3, ax = tid - 3 * ci;
            const real d = from_dbl<real>(a.ncenter[3 * nd + ax] - a.ncenter[3 * (fc + c0 + ci) + ax]);
            real v = 1;
            for (int m = 0; m <= P; ++m) {
                sh.u.m.cd[ci][ax][m] = v;
                v = v * d;
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int ax = 0; ax < 3; ++ax) {
            real(*srcb)[2 * T] = (ax == 1) ? sh.u.m.bufB : sh.u.m.bufA;
            real(*dstb)[2 * T] = (ax == 1) ? sh.u.m.bufA : sh.u.m.bufB;
            for (int it = tid; it < nb * T; it += blockDim.x) {
                const int ci = it / T, k = it - ci * T;
                const int k0 = sh.kk[k][0], k1 = sh.kk[k][1], k2 = sh.kk[k][2];
                const int ka = sh.kk[k][ax];
                real sL = 0, sY = 0;
                for (int j = 0; j <= ka; ++j) {
                    const int jx = ax == 0 ? j : k0, jy = ax == 1 ? j : k1, jz = ax == 2 ? j : k2;
                    const int jj = sh.idx3[jx][jy][jz];
                    const real coef = sh.binom[ka][j] * sh.u.m.cd[ci][ax][ka - j];
                    sL += coef * srcb[ci][jj];
                    sY += coef * srcb[ci][T + jj];
                }
                dstb[ci][k] = sL;
                dstb[ci][T + k] = sY;
            }
            __syncthreads();
        }
#pragma unroll
        for (int h = 0; h < HO; ++h) {
            const int k = tid + 128 * h;
            if (k < 2 * T)
                for (int ci = 0; ci < nb; ++ci) acc[h] += sh.u.m.bufB[ci][k];
        }
    }
#pragma unroll
    for (int h = 0; h < HO; ++h) {
        const int k = tid + 128 * h;
        if (k < 2 * T) mom[(int64_t)nd * 2 * T + k] = acc[h];
    }
}

template <typename real, int P>
__global__ void __launch_bounds__(128) k_upward(UpArgs a, const typename V4<real>::t* __restrict__ src,
                                                real* __restrict__ mom) {
    constexpr int T = MI<P>::T;
    extern __shared__ __align__(16) unsigned char up_smem[];
    UpShared<real, P>& sh = *reinterpret_cast<UpShared<real, P>*>(up_smem);
    const int tid = threadIdx.x;
    for (int k = tid; k < T; k += blockDim.x) {
        int x, y, z;
        decode_mi(k, x, y, z);
        sh.idx3[x][y][z] = (short)k;
        sh.kk[k][0] = (signed char)x;
        sh.kk[k][1] = (signed char)y;
        sh.kk[k][2] = (signed char)z;
    }
    for (int q = tid; q < (P + 1) * (P + 1); q += blockDim.x) {
        const int n = q / (P + 1), m = q - n * (P + 1);
        sh.binom[n][m] = from_dbl<real>(kBinomTable.v[n][m]);
    }
    __syncthreads();
    for (int64_t leaf = blockIdx.x; leaf < a.n_leaves; leaf += gridDim.x) {
        int nd = a.leaf_node[leaf];
        if (!body_on(a, a.nbody[nd])) continue;  // block-uniform
        up_p2m<real, P>(a, nd, src, mom, sh);
        for (;;) {
            // publish nd's moments, then count it at its parent
            __syncthreads();
            __threadfence();
            if (tid == 0) {
                const int par = a.parent[nd];
                int go = -1;
                if (par >= 0 && atomicAdd(a.arrive + par, 1) == a.nchild[par] - 1) go = par;
                sh.next = go;
            }
            __syncthreads();
            const int par = sh.next;
            if (par < 0) break;
            __threadfence();
            up_m2m<real, P>(a, par, mom, sh);
            if (tid == 0) a.arrive[par] = 0;  // every child has arrived: ready for the next launch
            nd = par;
        }
    }
}

// M2P warps per block: 8 (FP32) or 4 (8-byte types, for their registers),
// halved while the per-warp coefficient slices exceed 40 KB of shared memory
template <typename real, int P>
constexpr int m2p_warps() {
    int nw = sizeof(real) == 8 ? 4 : 8;
    while (nw > 1 && (size_t)nw * 2 * n_terms_pad(P) * sizeof(real) > 40 * 1024) nw /= 2;
    return nw;
}

// Nodes per block of k_far_big: 8 in FP32, 4 in the 8-byte types (shared memory).
template <typename real>
constexpr int far_big_nb() { return sizeof(real) == sizeof(float) ? 8 : 4; }

// The upward pass of one product: P2M and the moment shifts in one launch
// (k_upward), then the far-field coefficients (orders up to 8: k_far_f32 in
// FP32, k_far_coef with the packed table in shared memory otherwise; above:
// k_far_big for every type).
template <typename real, int P>
void launch_upward(const UpArgs& up, const void* src, void* mom, cudaStream_t s) {
    using v4 = typename V4<real>::t;
    if (up.n_leaves <= 0) return;
    constexpr size_t up_smem = sizeof(UpShared<real, P>);
    static bool up_attr = false;  // per instantiation
    if (!up_attr) {
        PGB_CUDA(cudaFuncSetAttribute(k_upward<real, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_smem));
        up_attr = true;
    }
    const int64_t grid = up.p2m_grid > 0 ? std::min<int64_t>(up.n_leaves, up.p2m_grid) : up.n_leaves;
    k_upward<real, P><<<(unsigned)grid, 128, up_smem, s>>>(up, (const v4*)src, (real*)mom);
    if (up.n_nodes <= 0) return;
    int dev = 0, n_sm = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    PGB_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    if constexpr (P > 8) {
        constexpr int NB = far_big_nb<real>();
        constexpr size_t smem = sizeof(real) * NB * 2 * MI<P>::T;
        static bool attr = false;
        if (!attr) {
            PGB_CUDA(cudaFuncSetAttribute(k_far_big<real, P, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr = true;
        }
        int64_t gf = (up.n_nodes + NB - 1) / NB;
        if (up.p2m_grid > 0) gf = std::min<int64_t>(gf, up.p2m_grid);
        k_far_big<real, P, NB><<<(unsigned)std::max<int64_t>(gf, 1), 128, smem, s>>>(up, (const real*)mom);
    } else if constexpr (sizeof(real) == sizeof(float)) {
        // FP32: a block per (node, table), a thread per output
        k_far_f32<P><<<dim3((unsigned)up.n_nodes, 2), far_tr(P), 0, s>>>(up, (const float*)mom);
    } else {
        // a few blocks per SM, each with the packed table in shared memory,
        // taking the nodes in turn
        constexpr size_t smem = far_coef_smem<real, P>();
        static bool attr = false;
        if (!attr) {
            PGB_CUDA(cudaFuncSetAttribute(k_far_coef<real, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr = true;
        }
        int64_t gf = std::min<int64_t>(up.n_nodes, 4 * (int64_t)n_sm);
        if (up.p2m_grid > 0) gf = std::min<int64_t>(gf, up.p2m_grid);
        k_far_coef<real, P><<<(unsigned)std::max<int64_t>(gf, 1), 128, smem, s>>>(up, (const real*)mom);
    }
}

}  // namespace pgb
