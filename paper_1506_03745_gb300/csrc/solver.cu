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
__global__ void k_coulomb_rows(Geo g, BodyDev bd, const double* qxyz, const double* qv, const int64_t* qoff,
                               const double* eps_in, double* b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int bi = g.pbody[i];
    if (bd.kind[bi] != PGB_DIELECTRIC) return;
    const double x = g.c[3 * i], y = g.c[3 * i + 1], z = g.c[3 * i + 2];
    double s = 0;
    for (int64_t k = qoff[bi]; k < qoff[bi + 1]; ++k) {
        double dx = x - qxyz[3 * k], dy = y - qxyz[3 * k + 1], dz = z - qxyz[3 * k + 2];
        s += qv[k] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    const int64_t loc = g.perm[i] - bd.pan_off[bi];
    b[bd.unk_off[bi] + loc] = s / (PGB_FOUR_PI * eps_in[bi]);
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

void build_rhs(pgb_ctx* c, double* b, int precision) {
    cudaStream_t s = c->stream;
    StageTimer tm(c, PGB_STAGE_RHS);
    PGB_CUDA(cudaMemsetAsync(b, 0, 8 * c->n_unk, s));
    bool any_known = false;
    for (auto& bd : c->bodies) any_known |= bd.kind != PGB_DIELECTRIC;
    if (any_known) apply_operator(c, nullptr, b, precision, true);
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
    if (r < n) v[r] = a > 0 ? w[r] / a : 0.0;
}

__global__ void k_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = a * x[r] + b * y[r];
}

// Givens step on column j of H (column-major, ld = m+1): apply the previous
// rotations, form the new one, rotate g; out[0] = |g_{j+1}|, out[1] = h_{j+1,j}.
__global__ void k_givens(double* H, int ld, double* cs, double* sn, double* g, int j, double* out) {
    if (threadIdx.x || blockIdx.x) return;
    double* h = H + (int64_t)j * ld;
    for (int i = 0; i < j; ++i) {
        double a = cs[i] * h[i] + sn[i] * h[i + 1];
        double b = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = a;
        h[i + 1] = b;
    }
    out[1] = h[j + 1];
    double a = h[j], b = h[j + 1];
    double r = hypot(a, b);
    double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = s;
    h[j] = r;
    h[j + 1] = 0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    out[0] = fabs(g[j + 1]);
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

// ---------------------------------------------------------------- fused Arnoldi step
// One cooperative launch per GMRES iteration does the whole CGS2 step of
// column j: two passes of (V_i . w for i <= j; w -= sum_i h_i V_i), the norm,
// v_{j+1} = w / |w| and the Givens update, with a grid barrier between the
// phases that exchange data between blocks.  Every thread keeps the same rows
// in every phase, so w and v_{j+1} need no barrier; values written by other
// blocks are read with ld.global.cg (L2, never a stale L1 line).
struct GridBar {
    unsigned count, gen;
    int err, pad;
};

#define PGB_BARRIER_NS 1000000000ull  // 1 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch: the arrival counter only grows
// (a release add per block), and barrier k of a launch waits (acquire loads)
// until it reaches target = base + (k + 1) * blocks, so no reset and no extra
// round trip are needed.  The wait is bounded (1 s of the global timer): on
// time-out the barrier records err and every block falls through.
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned target) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(&b->count, 1u);
        volatile int* verr = &b->err;
        const unsigned long long t0 = globaltimer_ns();
        for (long long it = 1;; ++it) {
            if ((int)(ld_acquire(&b->count) - target) >= 0) break;
            if (*verr) break;
            if ((it & 255) == 0 && (globaltimer_ns() - t0 > PGB_BARRIER_NS || it > (1ll << 26))) {
                atomicExch(&b->err, 1);
                break;
            }
        }
    }
    __syncthreads();
    return *(volatile int*)&b->err == 0;
}

struct ArnoldiArgs {
    double* V;      // basis, column i at V + i * ld
    int64_t ld, n;
    int j;          // the new column's index
    double* w;      // A v_j on entry; destroyed
    double* h;      // column j of H (m + 1 entries)
    double* hc;     // second-pass coefficients (j + 1)
    double* part;   // nb * (j + 1) block partial sums
    double *cs, *sn, *g;
    double* out;    // out[0] = |g_{j+1}|, out[1] = h_{j+1,j}, out[2] = 1 on a barrier time-out
    GridBar* bar;
    unsigned bar_base;  // arrival count before this launch (5 barriers per launch)
};

__global__ void __launch_bounds__(512) k_arnoldi(ArnoldiArgs a) {
    extern __shared__ double shd[];  // max(32, m * warps) doubles
    const int m = a.j + 1;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nb = gridDim.x;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = true;
    for (int pass = 0; pass < 2 && ok; ++pass) {
        double* coef = pass ? a.hc : a.h;
        for (int i0 = 0; i0 < m; i0 += 8) {  // block partials of V_i . w, eight vectors at a time
            double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t r = r0; r < a.n; r += stride) {
                const double wr = a.w[r];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < m) t[u] += a.V[(i0 + u) * a.ld + r] * wr;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = warp_sum(t[u]);
            if (lane == 0)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < m) shd[(i0 + u) * nw + wi] = t[u];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            double t = 0;
            for (int k = 0; k < nw; ++k) t += shd[i * nw + k];
            a.part[(int64_t)i * nb + blockIdx.x] = t;
        }
        if (!(ok = grid_sync(a.bar, a.bar_base + (2 * pass + 1) * nb))) break;
        for (int i = blockIdx.x; i < m; i += nb) {  // block i sums coefficient i
            double t = 0;
            for (unsigned b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(a.part + (int64_t)i * nb + b);
            t = block_sum(t, shd);
            if (threadIdx.x == 0) coef[i] = t;
        }
        if (!(ok = grid_sync(a.bar, a.bar_base + (2 * pass + 2) * nb))) break;
        for (int i = threadIdx.x; i < m; i += blockDim.x) shd[i] = __ldcg(coef + i);
        __syncthreads();
        for (int64_t r = r0; r < a.n; r += stride) {
            double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i0 = 0; i0 < m; i0 += 8)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < m) t[u] += shd[i0 + u] * a.V[(i0 + u) * a.ld + r];
            a.w[r] -= ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
        }
        __syncthreads();
    }
    double nrm = 0;
    if (ok) {
        if (blockIdx.x == 0)  // H column: first pass + correction (read after the barrier)
            for (int i = threadIdx.x; i < m; i += blockDim.x) a.h[i] = __ldcg(a.h + i) + __ldcg(a.hc + i);
        double t = 0;
        for (int64_t r = r0; r < a.n; r += stride) t += a.w[r] * a.w[r];
        t = block_sum(t, shd);
        if (threadIdx.x == 0) a.part[blockIdx.x] = t;
        ok = grid_sync(a.bar, a.bar_base + 5 * nb);
    }
    if (ok) {
        double t = 0;  // every block forms the norm (nb values)
        for (unsigned b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(a.part + b);
        t = block_sum(t, shd);
        if (threadIdx.x == 0) shd[0] = sqrt(t);
        __syncthreads();
        nrm = shd[0];
        double* vn = a.V + (int64_t)(a.j + 1) * a.ld;
        for (int64_t r = r0; r < a.n; r += stride) vn[r] = nrm > 0 ? a.w[r] / nrm : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ok) {  // Givens step on column j (as k_givens)
            double* h = a.h;
            h[a.j + 1] = nrm;
            for (int i = 0; i < a.j; ++i) {
                const double x = a.cs[i] * h[i] + a.sn[i] * h[i + 1];
                const double y = -a.sn[i] * h[i] + a.cs[i] * h[i + 1];
                h[i] = x;
                h[i + 1] = y;
            }
            a.out[1] = h[a.j + 1];
            const double p = h[a.j], q = h[a.j + 1];
            const double r = hypot(p, q);
            const double c = r > 0 ? p / r : 1.0, sv = r > 0 ? q / r : 0.0;
            a.cs[a.j] = c;
            a.sn[a.j] = sv;
            h[a.j] = r;
            h[a.j + 1] = 0;
            a.g[a.j + 1] = -sv * a.g[a.j];
            a.g[a.j] = c * a.g[a.j];
            a.out[0] = fabs(a.g[a.j + 1]);
        }
        a.out[2] = ok ? 0.0 : 1.0;
    }
}

// One block waits at a barrier sized for `expected` blocks: with expected > 1
// nothing ever completes it, so the bounded wait must give up and say so.
__global__ void k_barrier_probe(GridBar* b, unsigned expected, int* timed_out) {
    const bool ok = grid_sync(b, expected);
    if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

int barrier_probe(int expected, int* timed_out) {
    DBuf<unsigned> bar;
    DBuf<int> flag;
    bar.resize(4);
    flag.resize(1);
    PGB_CUDA(cudaMemset(bar.p, 0, 16));
    k_barrier_probe<<<1, 32>>>((GridBar*)bar.p, (unsigned)expected, flag.p);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaMemcpy(timed_out, flag.p, 4, cudaMemcpyDeviceToHost));
    return PGB_OK;
}

// Launches the fused Arnoldi step (false: cooperative launch unavailable;
// the caller takes the multi-kernel path).
static bool arnoldi_fused(pgb_ctx* c, int j, double* w, double* h, double* hc, double* cs, double* sn, double* g,
                          double* out) {
    if (c->coop_blocks < 0) return false;
    const int threads = 512, warps = threads / 32;  // one block per SM
    if (c->coop_blocks == 0) {
        int dev = 0, coop = 0, sms = 0, occ = 0;
        PGB_CUDA(cudaGetDevice(&dev));
        PGB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t smem_max = 8 * (size_t)257 * warps;  // restart <= 256
        PGB_CUDA(cudaFuncSetAttribute(k_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi, threads, smem_max));
        if (!coop || occ < 1) {
            c->coop_blocks = -1;
            return false;
        }
        c->coop_blocks = sms;
        c->d_bar.resize(4);
        PGB_CUDA(cudaMemsetAsync(c->d_bar.p, 0, 16, c->stream));
        c->bar_base = 0;
    }
    const int nb = c->coop_blocks;
    c->d_red.resize(std::max<size_t>(c->d_red.n, (size_t)nb * (j + 2)));
    ArnoldiArgs a;
    a.V = c->d_V;
    a.ld = c->n_unk;
    a.n = c->n_unk;
    a.j = j;
    a.w = w;
    a.h = h;
    a.hc = hc;
    a.part = c->d_red;
    a.cs = cs;
    a.sn = sn;
    a.g = g;
    a.out = out;
    a.bar = (GridBar*)c->d_bar.p;
    a.bar_base = c->bar_base;
    c->bar_base += 5u * (unsigned)nb;
    void* args[] = {&a};
    const size_t smem = 8 * (size_t)std::max(32, (j + 1) * warps);
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_arnoldi, nb, threads, args, smem, c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        c->coop_blocks = -1;
        return false;
    }
    return true;
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

static void precond_apply(pgb_ctx* c, const double* v, double* z, bool transpose, bool add) {
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

// Restarted GMRES on A x = b from the given x; precision of the operator
// `prec`; stops when the (estimated) residual <= abs_tol or after max_it
// iterations.  Returns iterations done; *matvecs counts operator uses.
int gmres_op(pgb_ctx* c, int prec, bool transpose, const double* b, double* x, double abs_tol, int max_it,
             int restart, int* matvecs, double* est_out, bool x_zero) {
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
            bool fused = false;
            {
                StageTimer tm(c, PGB_STAGE_KRYLOV);
                fused = arnoldi_fused(c, j, w, h, hcol, cs, sn, g, misc.p + 2);
                if (fused) PGB_LAUNCHED(c, 1);
            }
            if (!fused) {
                StageTimer tm(c, PGB_STAGE_KRYLOV);
                for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
                    k_multi_dot<<<DOT_BLOCKS, DOT_THREADS, 8 * (DOT_THREADS / 32) * (j + 1), s>>>(c->d_V, n, j + 1, w, n,
                                                                                            c->d_red);
                    k_reduce_partials<<<j + 1, 256, 0, s>>>(c->d_red, DOT_BLOCKS, pass ? hcol : h, 0, 0);
                    k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(c->d_V, n, j + 1, pass ? hcol : h, -1.0, w, n);
                    if (pass) k_axpby<<<1, 256, 0, s>>>(1.0, h, 1.0, hcol, h, j + 1);
                }
                K.norm(w, h + j + 1);
                k_scale_by<<<nblk(n, 256), 256, 0, s>>>(w, h + j + 1, c->d_V.p + (size_t)(j + 1) * n, n);
                k_givens<<<1, 1, 0, s>>>(c->d_H, m + 1, cs, sn, g, j, misc.p + 2);
                PGB_CUDA(cudaGetLastError());
                PGB_LAUNCHED(c, 12);
            }
            PGB_CUDA(cudaMemcpyAsync(c->h_pinned, misc.p + 2, fused ? 24 : 16, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            if (fused && c->h_pinned[2] != 0) {
                PGB_CUDA(cudaMemsetAsync(c->d_bar.p, 0, 16, s));
                c->bar_base = 0;
                fail(PGB_ETIMEOUT, "Arnoldi grid barrier timed out");
            }
            est = c->h_pinned[0];
            double hnext = c->h_pinned[1];
            if (est <= abs_tol || !(hnext > 0)) {
                ++j;
                ++it;
                break;
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
    build_rhs(c, c->d_b, rhs_prec);
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
        c->d_bc.resize(n);
        coulomb_rows(c, c->d_bc);
        PGB_CUDA(cudaMemcpyAsync(c->d_r.p, c->d_b.p, 8 * n, cudaMemcpyDeviceToDevice, s));
        double rn = bnorm;
        while (rel > tol && z.iterations < max_iter && z.outer_steps < 50) {
            // aim each inner FP32 solve at the final tolerance (the FP32
            // operator itself is accurate to ~1e-7), so that one FP64 residual
            // usually confirms convergence
            double inner = std::max(0.5 * tol * bnorm / rn, 1e-7);
            PGB_CUDA(cudaMemsetAsync(c->d_xs.p, 0, 8 * n, s));
            int mv = 0;
            int it = gmres(c, PGB_FP32, c->d_r, c->d_xs, inner * rn, max_iter - z.iterations, restart, &mv, nullptr, true);
            z.iterations += it;
            z.matvecs += mv;
            ++z.outer_steps;
            k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, x, 1.0, c->d_xs, x, n);
            apply_full(c, x, c->d_r, PGB_FP64);
            ++z.matvecs;
            ++z.matvecs_fp64;
            k_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_bc, -1.0, c->d_r, c->d_r, n);
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
