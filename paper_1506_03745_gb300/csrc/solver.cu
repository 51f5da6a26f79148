// Right-hand side and GMRES (Section 3.2 of the paper): FP64 Arnoldi with
// classical Gram-Schmidt applied twice, Givens rotations on the device, the
// restarted iteration driven from the host; optional FP32 inner solves with
// FP64 residual refinement.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "pgb_internal.cuh"

namespace pgb {

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// Coulomb rows (first line of Eq. 5, with its 1/eps_in kept -- reading of
// Eq. 6/7): (1/eps_in) sum_k q_k / (4 pi |c_i - r_k|) over the body's charges.
// With nested interfaces the outer row of a body inside another (a cavity in
// a molecule) takes the enclosing body's charges the same way (added to the
// row, which may hold imposed terms already).
__global__ void k_coulomb_rows(Geo g, BodyDev bd, const double* qxyz, const double* qv, const int64_t* qoff,
                               const double* eps_in, double* b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int bi = g.pbody[i];
    if (bd.kind[bi] != PGB_DIELECTRIC) return;
    const double x = g.c[3 * i], y = g.c[3 * i + 1], z = g.c[3 * i + 2];
    const int64_t loc = g.perm[i] - bd.pan_off[bi];
    const int64_t N = bd.pan_off[bi + 1] - bd.pan_off[bi];
    for (int side = 0; side < 2; ++side) {
        const int src = side == 0 ? bi : bd.parent[bi];
        if (src < 0) continue;
        double s = 0;
        for (int64_t k = qoff[src]; k < qoff[src + 1]; ++k) {
            double dx = x - qxyz[3 * k], dy = y - qxyz[3 * k + 1], dz = z - qxyz[3 * k + 2];
            s += qv[k] * rsqrt_nr<2>(dx * dx + dy * dy + dz * dz);  // FP64 rounding (common.cuh)
        }
        if (side == 0) b[bd.unk_off[bi] + loc] = s / (PGB_FOUR_PI * eps_in[bi]);
        else b[bd.unk_off[bi] + N + loc] += s / (PGB_FOUR_PI * eps_in[src]);
    }
}

// b = 0 except the Coulomb rows of the molecules.
void coulomb_rows(pgb_ctx* c, double* b) {
    cudaStream_t s = c->stream;
    PGB_CUDA(cudaMemsetAsync(b, 0, 8 * c->n_unk, s));
    std::vector<int64_t> qoff(c->bodies.size() + 1, 0);
    std::vector<double> eps(c->bodies.size());
    for (size_t i = 0; i < c->bodies.size(); ++i) {
        qoff[i] = c->bodies[i].q_off;
        eps[i] = c->bodies[i].eps_in;
    }
    qoff.back() = c->n_q;
    DBuf<int64_t> dq;
    DBuf<double> de;
    dq.resize(qoff.size());
    de.resize(eps.size());
    PGB_CUDA(cudaMemcpyAsync(dq.p, qoff.data(), 8 * qoff.size(), cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(de.p, eps.data(), 8 * eps.size(), cudaMemcpyHostToDevice, s));
    k_coulomb_rows<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), c->d_qxyz, c->d_qval, dq, de, b);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    PGB_LAUNCHED(c, 1);
}

__global__ void k_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n);

// bc: the Coulomb rows already formed (coulomb_rows), added to the imposed
// terms instead of being computed again (the imposed terms of a molecule's
// interior rows are zero: Laplace couples a body only to itself).
void build_rhs(pgb_ctx* c, double* b, int precision, const double* bc) {
    cudaStream_t s = c->stream;
    StageTimer tm(c, PGB_STAGE_RHS);
    PGB_CUDA(cudaMemsetAsync(b, 0, 8 * c->n_unk, s));
    bool any_known = false;
    for (auto& bd : c->bodies) any_known |= bd.kind != PGB_DIELECTRIC;
    if (any_known) apply_operator(c, nullptr, b, precision, true);
    if (bc) {
        k_axpby<<<nblk(c->n_unk, 256), 256, 0, s>>>(1.0, b, 1.0, bc, b, c->n_unk);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
        return;
    }
    std::vector<int64_t> qoff(c->bodies.size() + 1, 0);
    std::vector<double> eps(c->bodies.size());
    for (size_t i = 0; i < c->bodies.size(); ++i) {
        qoff[i] = c->bodies[i].q_off;
        eps[i] = c->bodies[i].eps_in;
    }
    qoff.back() = c->n_q;
    DBuf<int64_t> dq;
    DBuf<double> de;
    dq.resize(qoff.size());
    de.resize(eps.size());
    PGB_CUDA(cudaMemcpyAsync(dq.p, qoff.data(), 8 * qoff.size(), cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(de.p, eps.data(), 8 * eps.size(), cudaMemcpyHostToDevice, s));
    k_coulomb_rows<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), c->d_qxyz, c->d_qval, dq, de, b);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 2);
    PGB_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- BLAS-1/2
#define DOT_BLOCKS 304
#define DOT_THREADS 256

// partial[i * nb + blk] = sum over this block's rows of V_i . w, i < m.
// Each warp reduces its rows by shuffles and the warps' sums meet in shared
// memory, so the m products cost one block barrier in total.
__global__ void k_multi_dot(const double* __restrict__ V, int64_t ld, int m, const double* __restrict__ w, int64_t n,
                            double* partial) {
    extern __shared__ double shd[];  // m x (warps)
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int i = 0; i < m; ++i) {
        const double* v = V + i * ld;
        double s = 0;
        for (int64_t r = r0; r < n; r += stride) s += v[r] * w[r];
        s = warp_sum(s);
        if (lane == 0) shd[i * nw + wi] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s = 0;
        for (int k = 0; k < nw; ++k) s += shd[i * nw + k];
        partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
}

// out[i] = (accumulate ? out[i] : 0) + sum_b partial[i*nb + b]   (one block per i)
__global__ void k_reduce_partials(const double* partial, int nb, double* out, int accumulate, int sqrt_out) {
    __shared__ double sh[32];
    int i = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)i * nb + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        if (sqrt_out) s = sqrt(s);
        out[i] = accumulate ? out[i] + s : s;
    }
}

// w -= sum_i h[i] V_i   (sign = -1)  or  x += sum_i h[i] V_i (sign = +1)
__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ld, int m, const double* __restrict__ h, double sign,
                             double* __restrict__ w, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += h[i] * V[i * ld + r];
        w[r] += sign * s;
    }
}

// v = w / *nrm
__global__ void k_scale_by(const double* w, const double* nrm, double* v, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double a = *nrm;
    const double inv = a > 0 ? 1.0 / a : 0.0;
    if (r < n) v[r] = w[r] * inv;
}

__global__ void k_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = a * x[r] + b * y[r];
}

// y = H(0:k,0:k)^{-1} g(0:k) (upper triangular)
__global__ void k_backsolve(const double* H, int ld, const double* g, int k, double* y) {
    if (threadIdx.x || blockIdx.x) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= H[(int64_t)j * ld + i] * y[j];
        y[i] = H[(int64_t)i * ld + i] != 0 ? s / H[(int64_t)i * ld + i] : 0.0;
    }
}

__global__ void k_init_g(double* g, int m1, const double* beta) {
    int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < m1) g[i] = (i == 0) ? *beta : 0.0;
}

// ---------------------------------------------------------------- Arnoldi step in four launches
// The CGS2 step of column j without grid-wide barriers: every block keeps the
// same rows r = blockIdx.x * blockDim.x + threadIdx.x + k * stride in every
// launch, so w and v_{j+1} are only ever touched by their owner; the only
// data crossing blocks are the per-block partial sums, which each block of
// the next launch reduces for itself (in the same fixed order everywhere).
//   k_arn_dot:    part[i][b] = (V_i . w) over block b's rows
//   k_arn_update: c_i = sum_b part[i][b]; w -= sum_i c_i V_i; (pass 1) the
//                 partials of the second pass, (pass 2) of |w|^2
//   k_arn_finish: |w|, v_{j+1} = w / |w|, Givens step (block 0)
#define ARN_BLOCKS_PER_SM 1
#define ARN_THREADS 256

struct ArnArgs {
    double* V;      // basis, column i at V + i * ld
    int64_t ld, n;
    int j;          // the new column's index (m = j + 1 coefficients)
    double* w;      // A v_j on entry
    double* h;      // column j of H
    double* hc;     // second-pass coefficients
    double* part;   // nb * (m + 1) partial sums, row i at part + i * nb
    double* part2;  // second buffer (the next launch's partials)
    double *cs, *sn, *g;
    double* out;    // out[0] = |g_{j+1}|, out[1] = h_{j+1,j}
    // Independent problems of a block-diagonal system, one per blockIdx.y:
    // problem p owns rows poff[p] .. poff[p + 1] (poff == nullptr: one
    // problem, rows 0 .. n) and its own H, rotations and partial sums at
    // p * sH (h), p * sV (hc, cs, sn, g), p * sP (part, part2) and 2 p (out);
    // act[p] == 0 leaves problem p untouched (act == nullptr: all active).
    const int64_t* poff;
    const int* act;
    int64_t sH, sV, sP;
    // jdev != nullptr: the column index is read from device memory (an
    // Arnoldi step replayed from a graph), j above is ignored and column j
    // of H is at Hb + j * ldH
    const int* jdev;
    double* Hb;
    int64_t ldH;
};
__device__ __forceinline__ int arn_j(const ArnArgs& a) { return a.jdev ? *a.jdev : a.j; }

// The slice of ArnArgs that block (., p) works on; false when p is inactive.
struct ArnView {
    double *h, *hc, *part, *part2, *cs, *sn, *g, *out;
    int64_t lo, hi;
};
__device__ __forceinline__ bool arn_view(const ArnArgs& a, int j, ArnView& v) {
    const int p = blockIdx.y;
    if (a.act && !a.act[p]) return false;
    v.lo = a.poff ? a.poff[p] : 0;
    v.hi = a.poff ? a.poff[p + 1] : a.n;
    v.h = (a.jdev ? a.Hb + (int64_t)j * a.ldH : a.h) + p * a.sH;
    v.hc = a.hc + p * a.sV;
    v.cs = a.cs + p * a.sV;
    v.sn = a.sn + p * a.sV;
    v.g = a.g + p * a.sV;
    v.part = a.part + p * a.sP;
    v.part2 = a.part2 + p * a.sP;
    v.out = a.out + 2 * p;
    return true;
}

// Sums of eight values over the 32 lanes of a warp by a butterfly
// reduce-scatter: each exchange halves the values a lane keeps, so a lane
// does 9 additions instead of 40 (FP64 additions are scarce on this part).
// Returns the full sum of value k = 4 b4 + 2 b3 + b2 (b_i: bit i of the lane)
// in every lane; *k_out receives k.
__device__ __forceinline__ double warp_sum8(const double (&t)[8], int* k_out) {
    const int lane = threadIdx.x & 31;
    double u[4], v[2], x;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double give = h4 ? t[k] : t[k + 4];
        const double keep = h4 ? t[k + 4] : t[k];
        u[k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double give = h3 ? u[k] : u[k + 2];
        const double keep = h3 ? u[k + 2] : u[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    {
        const double give = h2 ? v[0] : v[1];
        const double keep = h2 ? v[1] : v[0];
        x = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    *k_out = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
    return x;
}

// Block partials of V_i . w (i < m) over this block's rows of its problem,
// eight vectors at a time.
__device__ __forceinline__ void arn_block_dots(const ArnArgs& a, const ArnView& v, int m, double* part, double* shd) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nb = gridDim.x;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int64_t r0 = v.lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int i0 = 0; i0 < m; i0 += 8) {
        double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t r = r0; r < v.hi; r += stride) {
            const double wr = a.w[r];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u < m) t[u] += a.V[(i0 + u) * a.ld + r] * wr;
        }
        int k;
        const double sum = warp_sum8(t, &k);
        if ((lane & 3) == 0 && i0 + k < m) shd[(i0 + k) * nw + wi] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = 0;
        for (int k = 0; k < nw; ++k) t += shd[i * nw + k];
        part[(int64_t)i * nb + blockIdx.x] = t;
    }
}

// c_i = sum_b part[i][b] for i < m into shared memory (one warp per i, lanes
// over b in a fixed order, then a fixed shuffle tree).
__device__ __forceinline__ void arn_reduce(const double* part, int m, double* coef) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nb = gridDim.x;
    for (int i = wi; i < m; i += nw) {
        double t = 0;
        for (unsigned b = lane; b < nb; b += 32) t += part[(int64_t)i * nb + b];
        t = warp_sum(t);
        if (lane == 0) coef[i] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(ARN_THREADS) k_arn_dot(ArnArgs a) {
    extern __shared__ double shd[];
    const int j = arn_j(a);
    ArnView v;
    if (!arn_view(a, j, v)) return;
    arn_block_dots(a, v, j + 1, v.part, shd);
}

// pass 0: coefficients into h; pass 1: into hc and h += hc.  Then w -= sum
// c_i V_i on this block's rows and the partials of the next step (pass 0:
// the second-pass dots; pass 1: |w|^2 in part2[b]).
__global__ void __launch_bounds__(ARN_THREADS) k_arn_update(ArnArgs a, int pass) {
    extern __shared__ double shd[];  // m coefficients, then the dot scratch
    const int j = arn_j(a);
    ArnView v;
    if (!arn_view(a, j, v)) return;
    const int m = j + 1;
    double* coef = shd;
    double* scratch = shd + ((m + 31) & ~31);
    arn_reduce(pass ? v.part2 : v.part, m, coef);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            if (pass) {
                v.hc[i] = coef[i];
                v.h[i] += coef[i];
            } else {
                v.h[i] = coef[i];
            }
        }
    const unsigned nb = gridDim.x;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int64_t r0 = v.lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double sq = 0;
    for (int64_t r = r0; r < v.hi; r += stride) {
        double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i0 = 0; i0 < m; i0 += 8)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u < m) t[u] += coef[i0 + u] * a.V[(i0 + u) * a.ld + r];
        const double wr = a.w[r] - (((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7])));
        a.w[r] = wr;
        sq += wr * wr;
    }
    if (pass == 0) {
        __syncthreads();
        arn_block_dots(a, v, m, v.part2, scratch);
    } else {
        sq = block_sum(sq, scratch);
        if (threadIdx.x == 0) v.part[blockIdx.x] = sq;
    }
}

__global__ void __launch_bounds__(ARN_THREADS) k_arn_finish(ArnArgs a) {
    extern __shared__ double shd[];
    const int j = arn_j(a);
    ArnView v;
    if (!arn_view(a, j, v)) return;
    const unsigned nb = gridDim.x;
    double t = 0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x) t += v.part[b];
    t = block_sum(t, shd);
    if (threadIdx.x == 0) shd[32] = sqrt(t);
    __syncthreads();
    const double nrm = shd[32];
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;  // one division per block, not per row
    const int64_t stride = (int64_t)nb * blockDim.x;
    double* vn = a.V + (int64_t)(j + 1) * a.ld;
    for (int64_t r = v.lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < v.hi; r += stride)
        vn[r] = a.w[r] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // Givens step on column j of H (column-major, ld = m + 1): the previous
        // rotations, then the new one, applied to g; out[0] = |g_{j+1}|, out[1] = h_{j+1,j}
        double* h = v.h;
        h[j + 1] = nrm;
        for (int i = 0; i < j; ++i) {
            const double x = v.cs[i] * h[i] + v.sn[i] * h[i + 1];
            const double y = -v.sn[i] * h[i] + v.cs[i] * h[i + 1];
            h[i] = x;
            h[i + 1] = y;
        }
        v.out[1] = h[j + 1];
        const double p = h[j], q = h[j + 1];
        const double r = hypot(p, q);
        const double c = r > 0 ? p / r : 1.0, sv = r > 0 ? q / r : 0.0;
        v.cs[j] = c;
        v.sn[j] = sv;
        h[j] = r;
        h[j + 1] = 0;
        v.g[j + 1] = -sv * v.g[j];
        v.g[j] = c * v.g[j];
        v.out[0] = fabs(v.g[j + 1]);
    }
}

// The four launches of one Arnoldi step; with sg, for the problems of a
// block-diagonal system (sg->nbp blocks per problem).
void arnoldi_step(pgb_ctx* c, int j, double* w, double* h, double* hc, double* cs, double* sn, double* g,
                  double* out, const ArnSeg* sg, const int* jdev, int mcap) {
    if (c->arn_blocks == 0) {
        int dev = 0, sms = 0;
        PGB_CUDA(cudaGetDevice(&dev));
        PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        c->arn_blocks = ARN_BLOCKS_PER_SM * sms;
    }
    const int B = sg ? sg->B : 1;
    // with jdev the column is only known on the device: sizes for the largest (mcap)
    const int nb = sg ? sg->nbp : c->arn_blocks, m = jdev ? mcap : j + 1, warps = ARN_THREADS / 32;
    c->d_red.resize(std::max<size_t>(c->d_red.n, (size_t)2 * nb * (m + 1) * B));
    ArnArgs a;
    a.V = c->d_V;
    a.ld = c->n_unk;
    a.n = c->n_unk;
    a.j = j;
    a.w = w;
    a.h = h;
    a.hc = hc;
    a.part = c->d_red;
    a.part2 = c->d_red.p + (size_t)nb * (m + 1) * B;
    a.cs = cs;
    a.sn = sn;
    a.g = g;
    a.out = out;
    a.poff = sg ? sg->poff : nullptr;
    a.act = sg ? sg->act : nullptr;
    a.sH = sg ? sg->sH : 0;
    a.sV = sg ? sg->sV : 0;
    a.sP = (int64_t)nb * (m + 1);
    a.jdev = jdev;
    a.Hb = h;
    a.ldH = (int64_t)mcap + 1;
    const size_t dots = 8 * (size_t)std::max(32, m * warps);
    const size_t upd = 8 * (size_t)((m + 31) & ~31) + dots;
    if (upd > 48 * 1024)
        PGB_CUDA(cudaFuncSetAttribute(k_arn_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd));
    cudaStream_t s = c->stream;
    const dim3 grid(nb, B);
    k_arn_dot<<<grid, ARN_THREADS, dots, s>>>(a);
    k_arn_update<<<grid, ARN_THREADS, upd, s>>>(a, 0);
    k_arn_update<<<grid, ARN_THREADS, upd, s>>>(a, 1);
    k_arn_finish<<<grid, ARN_THREADS, 8 * 64, s>>>(a);
    PGB_CUDA(cudaGetLastError());
}

// Block-diagonal preconditioner from the self terms (no equation of the
// paper: an addition to its GMRES).  The self entry of panel i holds
// a = V_L,ii and V_Y,ii (K_ii = 0 on a flat panel), so its own unknowns enter
// its own rows as
//   molecule (phi, dphi):  [[1/2, -a], [1/2, r b]],  r = eps_in/eps_out, b = V_Y,ii
//   imposed potential (dphi2):  b;   imposed charge (phi2):  1/2.
// pc[i] holds the inverse block (m00, m01, m10, m11).
__global__ void k_precond_build(Geo g, BodyDev bd, const int64_t* __restrict__ coff, const int32_t* __restrict__ cj,
                                const dbl4* __restrict__ cval, dbl4* __restrict__ pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    dbl4 d{0, 0, 0, 0};
    bool found = false;
    for (int64_t e = coff[i]; e < coff[i + 1]; ++e)
        if (cj[e] == i) {
            d = cval[e];
            found = true;
        }
    const int b = g.pbody[i];
    const int kind = bd.kind[b];
    dbl4 m{1, 0, 0, 1};
    if (found) {
        if (kind == PGB_DIELECTRIC) {
            const double a = d.x, rb = bd.eps_ratio[b] * d.z;
            const double det = 0.5 * (a + rb);
            if (det > 0) m = dbl4{rb / det, a / det, -0.5 / det, 0.5 / det};
        } else if (kind == PGB_SET_POTENTIAL) {
            if (d.z > 0) m = dbl4{1.0 / d.z, 0, 0, 0};
        } else {
            m = dbl4{2.0, 0, 0, 0};
        }
    }
    pc[i] = m;
}

// z = M^{-1} v (or M^{-T} v), add: z += instead of z =; vectors in the caller's layout.
__global__ void k_precond_apply(Geo g, BodyDev bd, const dbl4* __restrict__ pc, const double* __restrict__ v,
                                double* __restrict__ z, int transpose, int add) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    const dbl4 m = pc[i];
    if (bd.kind[b] == PGB_DIELECTRIC) {
        const double v1 = v[o + loc], v2 = v[o + N + loc];
        const double m01 = transpose ? m.z : m.y, m10 = transpose ? m.y : m.z;
        const double z1 = m.x * v1 + m01 * v2, z2 = m10 * v1 + m.w * v2;
        z[o + loc] = add ? z[o + loc] + z1 : z1;
        z[o + N + loc] = add ? z[o + N + loc] + z2 : z2;
    } else {
        const double z1 = m.x * v[o + loc];
        z[o + loc] = add ? z[o + loc] + z1 : z1;
    }
}

void precond_prepare(pgb_ctx* c) {
    c->pc_ready = false;
    if (!c->p.precond) return;
    c->d_pc.resize(c->n_pan);
    c->d_pz.resize(c->n_unk);
    k_precond_build<<<nblk(c->n_pan, 128), 128, 0, c->stream>>>(geo(c), body_dev(c), c->d_corr_off, c->d_corr_j,
                                                                c->d_corr_val, c->d_pc);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 1);
    c->pc_ready = true;
}

void precond_apply(pgb_ctx* c, const double* v, double* z, bool transpose, bool add) {
    k_precond_apply<<<nblk(c->n_pan, 128), 128, 0, c->stream>>>(geo(c), body_dev(c), c->d_pc, v, z,
                                                                transpose ? 1 : 0, add ? 1 : 0);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 1);
}

struct Krylov {
    pgb_ctx* c;
    int64_t n;
    int m;
    cudaStream_t s;

    void norm(const double* w, double* out) {
        k_multi_dot<<<DOT_BLOCKS, DOT_THREADS, 8 * (DOT_THREADS / 32), s>>>(w, n, 1, w, n, c->d_red);
        k_reduce_partials<<<1, 256, 0, s>>>(c->d_red, DOT_BLOCKS, out, 0, 1);
    }
    double host_read(const double* d) {
        PGB_CUDA(cudaMemcpyAsync(c->h_pinned, d, 8, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        return c->h_pinned[0];
    }
};

// ---------------------------------------------------------------- replayed iterations
// The column the next replayed product reads: dst = V_j, j from the device.
__global__ void k_gm_select(const double* __restrict__ V, int64_t n, const int* __restrict__ jdev,
                            double* __restrict__ dst) {
    const int64_t j = *jdev;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        dst[r] = V[j * n + r];
}
// After the Arnoldi step of column j: keep the estimate, advance j and set the
// graph's loop condition (go on while the estimate is above the tolerance,
// no breakdown and columns remain): ctl = {tol, column limit, estimate}.
__global__ void k_gm_check(const double* __restrict__ out, int* jdev, double* ctl, cudaGraphConditionalHandle h) {
    const int j = *jdev;
    const double est = out[0], hnext = out[1];
    *jdev = j + 1;
    ctl[2] = est;
    const bool more = est > ctl[0] && hnext > 0 && (double)(j + 1) < ctl[1];
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Restarted GMRES on A x = b from the given x; precision of the operator
// `prec`; stops when the (estimated) residual <= abs_tol or after max_it
// iterations.  Returns iterations done; *matvecs counts operator uses.
// Graph of the GMRES iterations after the first column of a cycle: a
// device-side while loop whose body takes column j (k_gm_select), applies the
// (preconditioned) operator, makes the Arnoldi step of column j and tests the
// estimate (k_gm_check).  Captured from the launches the host loop makes,
// with the context's work sent to its own capture stream; rebuilt when the
// tree, a parameter or a buffer it holds changes (gmres_op also drops it at
// the start of every call).
template <class ApplyPc>
static void gm_graph_ready(pgb_ctx* c, int prec, bool pc, int m, double* w, double* hcol, double* cs, double* sn,
                           double* g, double* out2, ApplyPc apply_pc) {
    auto& gg = c->gm_graph;
    const int64_t n = c->n_unk;
    if (gg.exec && gg.tree_gen == c->tree_gen && gg.prec == prec && gg.m == m && gg.pc == (int)pc &&
        gg.V == c->d_V.p && gg.w == w && gg.H == c->d_H.p && gg.g == g && gg.n == n && gg.P == c->p.P &&
        gg.theta == c->p.theta)
        return;
    if (gg.exec) {
        PGB_CUDA(cudaGraphExecDestroy(gg.exec));
        gg.exec = nullptr;
    }
    if (!c->gm_stream) PGB_CUDA(cudaStreamCreateWithFlags(&c->gm_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    PGB_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    PGB_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    PGB_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t saved = c->stream;
    const bool saved_timing = c->timing;
    const int64_t l0 = c->launches;
    c->stream = c->gm_stream;
    c->timing = false;
    c->capturing = true;
    std::string why;
    PGB_CUDA(cudaStreamBeginCaptureToGraph(c->gm_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        k_gm_select<<<nblk(n, 256), 256, 0, c->gm_stream>>>(c->d_V, n, c->d_gmi, c->d_xsel);
        apply_pc(c->d_xsel.p, w);
        arnoldi_step(c, 0, w, c->d_H, hcol, cs, sn, g, out2, nullptr, c->d_gmi, m);
        k_gm_check<<<1, 1, 0, c->gm_stream>>>(out2, c->d_gmi, c->d_gmd, h);
        PGB_LAUNCHED(c, 6);
    } catch (const Error& e) {
        why = e.msg;
    }
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->gm_stream, &captured);
    c->stream = saved;
    c->timing = saved_timing;
    c->capturing = false;
    gg.body_launches = c->launches - l0;
    c->launches = l0;
    if (!why.empty() || le != cudaSuccess || ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        fail(PGB_ECUDA, "GMRES iteration graph capture: " +
                            (why.empty() ? std::string(cudaGetErrorString(le != cudaSuccess ? le : ce)) : why));
    }
    const cudaError_t ie = cudaGraphInstantiate(&gg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) gg.exec = nullptr;
    PGB_CUDA(ie);
    gg.tree_gen = c->tree_gen;
    gg.prec = prec;
    gg.m = m;
    gg.pc = (int)pc;
    gg.V = c->d_V.p;
    gg.w = w;
    gg.H = c->d_H.p;
    gg.g = g;
    gg.n = n;
    gg.P = c->p.P;
    gg.theta = c->p.theta;
}

int gmres_op(pgb_ctx* c, int prec, bool transpose, const double* b, double* x, double abs_tol, int max_it,
             int restart, int* matvecs, double* est_out, bool x_zero, GmresSpec* spec) {
    const bool pc = c->p.precond && c->pc_ready;
    auto apply = [&](const double* in, double* out) {
        if (transpose) apply_transpose(c, in, out, prec);
        else apply_operator(c, in, out, prec, false);
    };
    // right preconditioning: the Krylov space is built on A M^{-1}, the
    // residual b - A x (and so the stopping test) is the unpreconditioned one
    auto apply_pc = [&](const double* in, double* out) {
        if (!pc) return apply(in, out);
        precond_apply(c, in, c->d_pz, transpose, false);
        apply(c->d_pz, out);
    };
    const int64_t n = c->n_unk;
    const int m = restart;
    cudaStream_t s = c->stream;
    Krylov K{c, n, m, s};
    c->d_V.resize((size_t)(m + 1) * n);
    c->d_H.resize((size_t)(m + 1) * m);
    c->d_red.resize((size_t)DOT_BLOCKS * (m + 1));
    c->d_gv.resize(3 * (m + 1) + 8);
    c->d_wk.resize(n);
    c->d_small.resize(2 * (m + 1) + 8);
    double* cs = c->d_gv.p;
    double* sn = cs + (m + 1);
    double* g = sn + (m + 1);
    double* hcol = c->d_small.p;       // m+1 (current H column tail workspace)
    double* yv = hcol + (m + 1);       // m+1
    DBuf<double> misc;
    misc.resize(8);
    // iterations replayed from a graph (not with the overlap's fork, which
    // the host decides, nor for the transposed operator)
    const bool graph = c->p.graphs >= 2 && !spec && !transpose && m >= 2;
    if (graph) {
        // The graph holds the launches of this call's operator (kernel
        // arguments, buffer addresses, grid sizes), which other calls may
        // change (parameters, trees, buffers): it is captured afresh for
        // each call, on its first replay, and kept for its restart cycles.
        if (c->gm_graph.exec) {
            PGB_CUDA(cudaGraphExecDestroy(c->gm_graph.exec));
            c->gm_graph.exec = nullptr;
        }
        // everything the replayed body touches is sized here, outside the capture
        c->d_gmi.resize(1);
        c->d_gmd.resize(3);
        c->d_xsel.resize(n);
        if (pc) c->d_pz.resize(n);
        reserve_product(c, prec);
        if (c->arn_blocks == 0) {
            int dev = 0, sms = 0;
            PGB_CUDA(cudaGetDevice(&dev));
            PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            c->arn_blocks = ARN_BLOCKS_PER_SM * sms;
        }
        c->d_red.resize(std::max<size_t>(c->d_red.n, (size_t)2 * c->arn_blocks * (m + 1)));
    }
    int it = 0;
    double est = INFINITY;
    while (it < max_it) {
        // r = b - A x (x = 0 on entry needs no product)
        if (x_zero) {
            PGB_CUDA(cudaMemcpyAsync(c->d_wk.p, b, 8 * n, cudaMemcpyDeviceToDevice, s));
            x_zero = false;
        } else {
            apply(x, c->d_wk);
            ++*matvecs;
            k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, b, -1.0, c->d_wk, c->d_wk, n);
        }
        K.norm(c->d_wk, misc.p);
        PGB_LAUNCHED(c, 3);
        double beta = K.host_read(misc.p);
        est = beta;
        if (beta <= abs_tol || beta == 0) break;
        k_scale_by<<<nblk(n, 256), 256, 0, s>>>(c->d_wk, misc.p, c->d_V, n);
        k_init_g<<<1, 256, 0, s>>>(g, m + 1, misc.p);
        int j = 0;
        for (; j < m && it < max_it; ++j, ++it) {
            double* vj = c->d_V.p + (size_t)j * n;
            double* w = c->d_wk.p;
            apply_pc(vj, w);
            ++*matvecs;
            double* h = c->d_H.p + (size_t)j * (m + 1);
            {
                StageTimer tm(c, PGB_STAGE_KRYLOV);
                arnoldi_step(c, j, w, h, hcol, cs, sn, g, misc.p + 2, nullptr);
                PGB_LAUNCHED(c, 4);
            }
            PGB_CUDA(cudaMemcpyAsync(c->h_pinned, misc.p + 2, 16, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            est = c->h_pinned[0];
            double hnext = c->h_pinned[1];
            if (est <= abs_tol || !(hnext > 0)) {
                ++j;
                ++it;
                break;
            }
            if (graph && j == 0 && j + 1 < m && it + 1 < max_it) {
                // columns 1 .. from the graph: the first column sized every
                // buffer the body touches
                const int jmax = (int)std::min<int64_t>(m, (int64_t)j + 1 + (max_it - it - 1));
                gm_graph_ready(c, prec, pc, m, w, hcol, cs, sn, g, misc.p + 2, apply_pc);
                c->h_pinned[4] = abs_tol;
                c->h_pinned[5] = (double)jmax;
                int* hj = reinterpret_cast<int*>(c->h_pinned + 6);
                hj[0] = 1;
                PGB_CUDA(cudaMemcpyAsync(c->d_gmi.p, hj, sizeof(int), cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaMemcpyAsync(c->d_gmd.p, c->h_pinned + 4, 16, cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaGraphLaunch(c->gm_graph.exec, s));
                PGB_CUDA(cudaMemcpyAsync(hj, c->d_gmi.p, sizeof(int), cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaMemcpyAsync(c->h_pinned + 5, c->d_gmd.p + 2, 8, cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaStreamSynchronize(s));
                const int done = hj[0] - 1;  // columns the graph made
                est = c->h_pinned[5];
                c->launches += done * c->gm_graph.body_launches;
                c->graph_kernels += done * c->gm_graph.body_launches;
                ++c->graph_launches;
                *matvecs += done;
                it += 1 + done;
                j += 1 + done;
                break;
            }
            if (spec && !spec->forked && est <= spec->abs_thresh) {
                // xs = x + M^{-1} V y with the j + 1 columns so far
                k_backsolve<<<1, 1, 0, s>>>(c->d_H, m + 1, g, j + 1, yv);
                PGB_CUDA(cudaMemcpyAsync(spec->xs, x, 8 * n, cudaMemcpyDeviceToDevice, s));
                if (pc) {
                    PGB_CUDA(cudaMemsetAsync(c->d_pz.p, 0, 8 * n, s));
                    k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(c->d_V, n, j + 1, yv, 1.0, c->d_pz, n);
                    precond_apply(c, c->d_pz, spec->xs, transpose, true);
                } else {
                    k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(c->d_V, n, j + 1, yv, 1.0, spec->xs, n);
                }
                PGB_CUDA(cudaGetLastError());
                PGB_LAUNCHED(c, 2);
                spec->forked = true;
                spec->fork(c, spec->xs, spec->user);
            }
        }
        k_backsolve<<<1, 1, 0, s>>>(c->d_H, m + 1, g, j, yv);
        if (pc) {  // x += M^{-1} V y
            PGB_CUDA(cudaMemsetAsync(c->d_pz.p, 0, 8 * n, s));
            k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(c->d_V, n, j, yv, 1.0, c->d_pz, n);
            precond_apply(c, c->d_pz, x, transpose, true);
        } else {
            k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(c->d_V, n, j, yv, 1.0, x, n);
        }
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 2);
        if (est <= abs_tol) break;
    }
    if (est_out) *est_out = est;
    return it;
}

static int gmres(pgb_ctx* c, int prec, const double* b, double* x, double abs_tol, int max_it, int restart,
                 int* matvecs, double* est_out, bool x_zero) {
    return gmres_op(c, prec, false, b, x, abs_tol, max_it, restart, matvecs, est_out, x_zero);
}

double vec_dot(pgb_ctx* c, const double* a, const double* b) {
    PGB_LAUNCHED(c, 2);
    Krylov K{c, c->n_unk, 0, c->stream};
    DBuf<double> t;
    t.resize(1);
    c->d_red.resize(std::max<size_t>(c->d_red.n, DOT_BLOCKS));
    k_multi_dot<<<DOT_BLOCKS, DOT_THREADS, 8 * (DOT_THREADS / 32), c->stream>>>(a, c->n_unk, 1, b, c->n_unk,
                                                                                   c->d_red);
    k_reduce_partials<<<1, 256, 0, c->stream>>>(c->d_red, DOT_BLOCKS, t, 0, 0);
    return K.host_read(t);
}

static double vec_norm(pgb_ctx* c, const double* v) {
    PGB_LAUNCHED(c, 2);
    Krylov K{c, c->n_unk, 0, c->stream};
    DBuf<double> t;
    t.resize(1);
    c->d_red.resize(std::max<size_t>(c->d_red.n, DOT_BLOCKS));
    K.norm(v, t);
    return K.host_read(t);
}

// For the duration of a refinement with overlap: the context's work goes to
// its highest-priority stream (ordered after the caller's stream at entry,
// and the caller's stream after it at exit), and allocations follow.
struct StreamSwap {
    pgb_ctx* c;
    cudaStream_t user = nullptr;
    AllocScope* scope = nullptr;
    StreamSwap(pgb_ctx* ctx, bool on) : c(ctx) {
        if (!on) return;
        if (!c->hp_stream) {
            int least = 0, greatest = 0;
            PGB_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            PGB_CUDA(cudaStreamCreateWithPriority(&c->hp_stream, cudaStreamNonBlocking, greatest));
            PGB_CUDA(cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, least));
            PGB_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
            PGB_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        }
        user = c->stream;
        PGB_CUDA(cudaEventRecord(c->ev_fork, user));
        PGB_CUDA(cudaStreamWaitEvent(c->hp_stream, c->ev_fork, 0));
        c->stream = c->hp_stream;
        scope = new AllocScope(c->hp_stream);
    }
    ~StreamSwap() {
        if (!scope) return;
        delete scope;
        c->stream = user;
        // the caller's stream continues after everything of the solve
        cudaEventRecord(c->ev_join, c->hp_stream);
        cudaStreamWaitEvent(user, c->ev_join, 0);
    }
};

// Side-stream FP64 product of the refinement (overlap): x* = x_outer +
// (inner iterate); its FP64 product r64 = A64(x* + imposed) runs on the
// side stream, P2P and M2P launched persistently with one block per SM so
// that the FP32 kernels of the continuing inner iterations keep the rest of
// each SM (the FP64 kernels are bound by the FP64 pipe, which the FP32
// kernels do not use).  The buffers it touches are sized on the main stream
// before the fork.
struct OverlapArgs {
    const double* x_outer;
};

static void overlap_fork(pgb_ctx* c, const double* xs, void* user) {
    const OverlapArgs* oa = (const OverlapArgs*)user;
    const int64_t n = c->n_unk;
    cudaStream_t s = c->stream;
    double* xfull = c->d_xspec.p;  // overwrite x* in place: x_outer + inner iterate
    k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, oa->x_outer, 1.0, xs, xfull, n);
    c->d_r64.resize(n);
    reserve_product(c, PGB_FP64);
    int dev = 0, sms = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PGB_CUDA(cudaEventRecord(c->ev_fork, s));
    PGB_CUDA(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    c->stream = c->side_stream;
    c->persist_blocks = sms;
    try {
        apply_full(c, xfull, c->d_r64, c->p.residual ? PGB_FP64_DS : PGB_FP64);
    } catch (...) {
        c->stream = s;
        c->persist_blocks = 0;
        throw;
    }
    c->stream = s;
    c->persist_blocks = 0;
    PGB_CUDA(cudaEventRecord(c->ev_join, c->side_stream));
}

int solve(pgb_ctx* c, int mode, double tol, int max_iter, int restart, double* x, pgb_solve_stats* st) {
    const int64_t n = c->n_unk;
    cudaStream_t s = c->stream;
    c->d_b.resize(n);
    c->d_r.resize(n);
    c->d_xs.resize(n);
    c->d_red.resize((size_t)DOT_BLOCKS * (restart + 1));
    if (mode != PGB_FP64 && mode != PGB_FP32_REFINE && mode != PGB_FP32)
        fail(PGB_EINVAL, "mode must be PGB_FP64, PGB_FP32_REFINE or PGB_FP32");
    const int rhs_prec = mode == PGB_FP64 ? PGB_FP64 : PGB_FP32;
    if (mode == PGB_FP32_REFINE) {  // the outer residual's Coulomb rows, also the inner right-hand side's
        c->d_bc.resize(n);
        coulomb_rows(c, c->d_bc);
        build_rhs(c, c->d_b, rhs_prec, c->d_bc);
    } else {
        build_rhs(c, c->d_b, rhs_prec);
    }
    precond_prepare(c);
    pgb_solve_stats z{};
    int known_mv = 0;
    for (auto& b : c->bodies)
        if (b.kind != PGB_DIELECTRIC) {
            known_mv = 1;  // imposed-boundary terms of the right-hand side
            break;
        }
    z.matvecs = known_mv;
    z.matvecs_fp64 = rhs_prec == PGB_FP64 ? known_mv : 0;
    const double bnorm = vec_norm(c, c->d_b);
    PGB_CUDA(cudaMemsetAsync(x, 0, 8 * n, s));
    if (bnorm == 0) {
        z.outer_steps = 0;
        z.rel_residual = 0;
        if (st) *st = z;
        return PGB_OK;
    }
    double rel = 1.0;
    if (mode == PGB_FP64) {
        int mv = 0;
        z.iterations = gmres(c, PGB_FP64, c->d_b, x, tol * bnorm, max_iter, restart, &mv, nullptr, true);
        z.matvecs += mv;
        z.matvecs_fp64 += mv;
        z.outer_steps = 1;
        apply_operator(c, x, c->d_r, PGB_FP64, false);
        ++z.matvecs;
        ++z.matvecs_fp64;
        k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_b, -1.0, c->d_r, c->d_r, n);
        rel = vec_norm(c, c->d_r) / bnorm;
    } else if (mode == PGB_FP32_REFINE) {
        // Inner FP32 solves take the right-hand side from the FP32 operator;
        // the outer residual is FP64 throughout: r = b_Coulomb - A64(x + imposed
        // densities), one FP64 product per outer step.
        // With overlap the iterations run on a highest-priority stream and the
        // FP64 product on a lowest-priority one, so that the block scheduler
        // serves the FP32 chain first and the FP64 work fills the rest.
        StreamSwap swap(c, c->p.overlap != 0);
        s = c->stream;
        PGB_CUDA(cudaMemcpyAsync(c->d_r.p, c->d_b.p, 8 * n, cudaMemcpyDeviceToDevice, s));
        double rn = bnorm;
        while (rel > tol && z.iterations < max_iter && z.outer_steps < 50) {
            // aim each inner FP32 solve at the final tolerance (the FP32
            // operator itself is accurate to ~1e-7), so that one FP64 residual
            // usually confirms convergence
            double inner = std::max(0.5 * tol * bnorm / rn, 1e-7);
            PGB_CUDA(cudaMemsetAsync(c->d_xs.p, 0, 8 * n, s));
            // Overlap: once the inner estimate reaches eps* of its right-hand
            // side, the FP64 product of that iterate starts on a side stream
            // while the FP32 iterations go on (see overlap_fork).
            const double eps_star = std::min(1e-2, 1e4 * tol);
            GmresSpec spec;
            OverlapArgs oa{x};
            const bool overlap = c->p.overlap && eps_star > 10 * inner;
            if (overlap) {
                c->d_xspec.resize(2 * n);
                spec.abs_thresh = eps_star * rn;
                spec.xs = c->d_xspec;
                spec.fork = overlap_fork;
                spec.user = &oa;
            }
            int mv = 0;
            int it = gmres_op(c, PGB_FP32, false, c->d_r, c->d_xs, inner * rn, max_iter - z.iterations, restart, &mv,
                              nullptr, true, overlap ? &spec : nullptr);
            z.iterations += it;
            z.matvecs += mv;
            ++z.outer_steps;
            k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, x, 1.0, c->d_xs, x, n);
            if (spec.forked) {
                // r = b - A64(x* + imposed) - A32(x - x*): the FP32 term is of
                // size ~eps* |b| and carries the FP32 operator's relative error
                // (~1e-6), i.e. ~1e-8 |b|, far below the tolerance
                double* dlt = c->d_xspec.p + n;  // x (updated above) - x*
                k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, x, -1.0, c->d_xspec, dlt, n);
                apply_operator(c, dlt, c->d_r, PGB_FP32, false);
                PGB_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
                k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_bc, -1.0, c->d_r64, c->d_wk, n);
                k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_wk, -1.0, c->d_r, c->d_r, n);
                z.matvecs += 2;
                ++z.matvecs_fp64;
            } else {
                apply_full(c, x, c->d_r, c->p.residual ? PGB_FP64_DS : PGB_FP64);
                ++z.matvecs;
                ++z.matvecs_fp64;
                k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_bc, -1.0, c->d_r, c->d_r, n);
            }
            double rn_new = vec_norm(c, c->d_r);
            rel = rn_new / bnorm;
            if (it == 0 || !(rn_new < rn)) {  // no progress: stop
                rn = rn_new;
                break;
            }
            rn = rn_new;
        }
    } else {
        // FP32 operator throughout, FP64 Arnoldi/Givens; the reported residual
        // uses the same FP32 operator
        int mv = 0;
        z.iterations = gmres(c, PGB_FP32, c->d_b, x, tol * bnorm, max_iter, restart, &mv, nullptr, true);
        z.matvecs += mv;
        z.outer_steps = 1;
        apply_operator(c, x, c->d_r, PGB_FP32, false);
        ++z.matvecs;
        k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_b, -1.0, c->d_r, c->d_r, n);
        rel = vec_norm(c, c->d_r) / bnorm;
    }
    PGB_CUDA(cudaGetLastError());
    z.rel_residual = rel;
    if (st) *st = z;
    return rel <= tol ? PGB_OK : PGB_ENOCONV;
}

}  // namespace pgb
