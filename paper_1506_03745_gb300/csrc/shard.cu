// A single solve sharded over ranks (one process per GPU): contiguous ranges
// of target groups in Morton order per rank.  Every rank holds the whole
// geometry, tree and near field (the upward pass is computed redundantly);
// a product on rank r computes the rows of its groups from the full density
// vector, which the ranks assemble by one allgather per product; GMRES keeps
// each rank's rows of the Krylov vectors and sums the dot products of the
// Arnoldi steps by allreduce (Section 3.2's GMRES and treecode product,
// split by target rows).  The collectives are the caller's (a callback), so
// the library works with any transport: torch.distributed over NCCL between
// GPUs, or gloo between CPU ranks.
//
// Sharded order of the unknowns: sorted panel by sorted panel (body-major
// Morton order), each panel's rows together (phi then dphi/dn for a
// molecule, u for a surface).  A contiguous range of target groups is then a
// contiguous range of rows.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "pgb_internal.cuh"

namespace pgb {

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// caller order <-> sharded order (full vectors)
__global__ void k_to_sharded(Geo g, BodyDev bd, const double* __restrict__ xc, double* __restrict__ xs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    if (bd.kind[b] == PGB_DIELECTRIC) {
        const int64_t s = o + 2 * (i - bd.pan_off[b]);
        xs[s] = xc[o + loc];
        xs[s + 1] = xc[o + N + loc];
    } else {
        xs[o + (i - bd.pan_off[b])] = xc[o + loc];
    }
}
__global__ void k_from_sharded(Geo g, BodyDev bd, const double* __restrict__ xs, double* __restrict__ xc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    if (bd.kind[b] == PGB_DIELECTRIC) {
        const int64_t s = o + 2 * (i - bd.pan_off[b]);
        xc[o + loc] = xs[s];
        xc[o + N + loc] = xs[s + 1];
    } else {
        xc[o + loc] = xs[o + (i - bd.pan_off[b])];
    }
}

// Local Krylov arithmetic over a rank's rows (n rows, columns of stride ld):
// dots[i] = V_i . w for i < m, by per-block partial sums reduced in a fixed
// order (k_sh_sum), so that every rank sums its rows the same way.
#define SH_BLOCKS 64
#define SH_THREADS 256
__global__ void __launch_bounds__(SH_THREADS) k_sh_dots(const double* __restrict__ V, int64_t ld, int m,
                                                        const double* __restrict__ w, int64_t n,
                                                        double* __restrict__ part) {
    __shared__ double sh[32];
    for (int i = 0; i < m; ++i) {
        double t = 0;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
            t += V[(int64_t)i * ld + r] * w[r];
        t = block_sum(t, sh);
        if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = t;
    }
}
__global__ void k_sh_sum(const double* __restrict__ part, int nb, int m, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double t = 0;
    for (int b = 0; b < nb; ++b) t += part[(int64_t)i * nb + b];
    out[i] = t;
}
// w -= sum_i h_i V_i (i < m)
__global__ void k_sh_update(const double* __restrict__ V, int64_t ld, int m, const double* __restrict__ h,
                            double* __restrict__ w, int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double t = 0;
    for (int i = 0; i < m; ++i) t += h[i] * V[(int64_t)i * ld + r];
    w[r] -= t;
}
__global__ void k_sh_scale(const double* __restrict__ w, double s, double* __restrict__ v, int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) v[r] = w[r] * s;
}
__global__ void k_sh_axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                           double* __restrict__ out, int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = a * x[r] + b * y[r];
}

// Balanced contiguous split of ng groups of the given work over world ranks:
// bounds[r] .. bounds[r + 1] are rank r's groups; each boundary is placed
// where the running work first reaches r / world of the total (every rank
// gets at least one group when ng >= world).
void shard_partition(const double* work, int64_t ng, int world, int64_t* bounds) {
    double tot = 0;
    for (int64_t g = 0; g < ng; ++g) tot += work[g];
    bounds[0] = 0;
    double run = 0;
    int64_t g = 0;
    for (int r = 1; r < world; ++r) {
        const double goal = tot * r / world;
        while (g < ng && run + work[g] <= goal) run += work[g++];
        int64_t b = std::max<int64_t>(g, bounds[r - 1] + (ng >= world ? 1 : 0));
        b = std::min<int64_t>(b, ng - (ng >= world ? (world - r) : 0));
        while (g < b) run += work[g++];
        bounds[r] = b;
    }
    bounds[world] = ng;
}

// Work of each target group (P2P tiles and far entries, weighted by their
// operation counts: a tile of 32 points for 32 targets against a far node
// for 32 targets, about 3 : 1 at P = 6) and the rank's group and row range.
static void shard_ranges(pgb_ctx* c, int world, std::vector<int64_t>& gb, std::vector<int64_t>& rb) {
    const int64_t ng = c->n_groups;
    std::vector<int64_t> toff(ng + 1), foff(ng + 1);
    std::vector<int32_t> gs(ng);
    cudaStream_t s = c->stream;
    PGB_CUDA(cudaMemcpyAsync(toff.data(), c->d_tile_off.p, 8 * (ng + 1), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(foff.data(), c->d_far_off.p, 8 * (ng + 1), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(gs.data(), c->d_group_start.p, 4 * ng, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    std::vector<double> work(ng);
    for (int64_t g = 0; g < ng; ++g) work[g] = 3.0 * (toff[g + 1] - toff[g]) + (foff[g + 1] - foff[g]) + 1.0;
    gb.assign(world + 1, 0);
    shard_partition(work.data(), ng, world, gb.data());
    // sharded row of the first panel of a group: the body's unknown offset
    // plus its panels before it times the rows per panel
    auto row_of_panel = [&](int64_t p) -> int64_t {
        if (p >= c->n_pan) return c->n_unk;
        int64_t off = 0;
        for (const auto& bd : c->bodies) {
            if (p < bd.pan_off + bd.N) return off + (p - bd.pan_off) * (bd.kind == PGB_DIELECTRIC ? 2 : 1);
            off += bd.kind == PGB_DIELECTRIC ? 2 * bd.N : bd.N;
        }
        return c->n_unk;
    };
    rb.assign(world + 1, 0);
    for (int r = 0; r <= world; ++r) rb[r] = gb[r] < ng ? row_of_panel(gs[gb[r]]) : c->n_unk;
}

// A rank's rows of the product: xs (full, sharded order) -> ys (its rows).
static void shard_product(pgb_ctx* c, const std::vector<int64_t>& gb, const std::vector<int64_t>& rb, int rank,
                          const double* xs, double* ys, int prec) {
    const int64_t n = c->n_unk;
    cudaStream_t s = c->stream;
    c->d_xtmp.resize(n);
    c->d_ytmp.resize(n);
    Geo g = geo(c);
    BodyDev bd = body_dev(c);
    k_from_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, xs, c->d_xtmp);
    PGB_LAUNCHED(c, 1);
    c->shard_g[0] = gb[rank];
    c->shard_g[1] = gb[rank + 1];
    try {
        apply_mode(c, c->d_xtmp, c->d_ytmp, prec, 0, nullptr);
    } catch (...) {
        c->shard_g[0] = c->shard_g[1] = -1;
        throw;
    }
    c->shard_g[0] = c->shard_g[1] = -1;
    // the whole vector to sharded order, then the rank's rows
    c->d_shard_tmp.resize(n);
    k_to_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, c->d_ytmp, c->d_shard_tmp);
    PGB_CUDA(cudaMemcpyAsync(ys, c->d_shard_tmp.p + rb[rank], 8 * (rb[rank + 1] - rb[rank]), cudaMemcpyDeviceToDevice,
                             s));
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 1);
}

struct ShardRun {
    pgb_ctx* c;
    int rank, world;
    std::vector<int64_t> gb, rb;
    double *xs, *red;  // exchange buffers (caller's)
    pgb_collective_fn coll;
    void* user;
    int64_t nl() const { return rb[rank + 1] - rb[rank]; }
    void sync() { PGB_CUDA(cudaStreamSynchronize(c->stream)); }
    // xs[own rows] = v (local), then every rank's rows into xs
    void gather(const double* v) {
        PGB_CUDA(cudaMemcpyAsync(xs + rb[rank], v, 8 * nl(), cudaMemcpyDeviceToDevice, c->stream));
        sync();
        if (coll(user, PGB_COLL_ALLGATHER, c->n_unk) != 0) fail(PGB_ECOLL, "allgather callback failed");
    }
    // red[0 .. m) summed over the ranks; returned on the host
    std::vector<double> allreduce(int m) {
        sync();
        if (coll(user, PGB_COLL_ALLREDUCE, m) != 0) fail(PGB_ECOLL, "allreduce callback failed");
        std::vector<double> h(m);
        PGB_CUDA(cudaMemcpy(h.data(), red, 8 * m, cudaMemcpyDeviceToHost));
        return h;
    }
    void local_dots(const double* V, int64_t ld, int m, const double* w) {
        c->d_shard_part.resize((size_t)SH_BLOCKS * std::max(m, 1));
        k_sh_dots<<<SH_BLOCKS, SH_THREADS, 0, c->stream>>>(V, ld, m, w, nl(), c->d_shard_part);
        k_sh_sum<<<nblk(m, 64), 64, 0, c->stream>>>(c->d_shard_part, SH_BLOCKS, m, red);
        PGB_LAUNCHED(c, 2);
    }
    double norm(const double* w) {
        local_dots(w, 0, 1, w);
        return sqrt(allreduce(1)[0]);
    }
};

// Restarted GMRES (CGS2) on the rank's rows: A x = b (local rows of b and x,
// operator of precision prec); returns the iterations; stops when the
// residual estimate <= abs_tol.
static int shard_gmres(ShardRun& S, int prec, const double* b, double* x, double abs_tol, int max_it, int m,
                       int* matvecs, double* est_out) {
    pgb_ctx* c = S.c;
    const int64_t nl = S.nl();
    cudaStream_t s = c->stream;
    c->d_shard_V.resize((size_t)(m + 1) * std::max<int64_t>(nl, 1));
    c->d_shard_w.resize(std::max<int64_t>(nl, 1));
    c->d_shard_h.resize(m + 1);
    double* V = c->d_shard_V;
    double* w = c->d_shard_w;
    double* hd = c->d_shard_h;
    const int64_t ld = std::max<int64_t>(nl, 1);
    int it = 0;
    double est = INFINITY;
    while (it < max_it) {
        // r = b - A x
        S.gather(x);
        shard_product(c, S.gb, S.rb, S.rank, S.xs, w, prec);
        ++*matvecs;
        k_sh_axpby<<<nblk(nl, 256), 256, 0, s>>>(1.0, b, -1.0, w, w, nl);
        const double beta = S.norm(w);
        est = beta;
        if (beta <= abs_tol || beta == 0) break;
        k_sh_scale<<<nblk(nl, 256), 256, 0, s>>>(w, 1.0 / beta, V, nl);
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m && it < max_it; ++j, ++it) {
            S.gather(V + (size_t)j * ld);
            shard_product(c, S.gb, S.rb, S.rank, S.xs, w, prec);
            ++*matvecs;
            double* h = H.data() + (size_t)j * (m + 1);
            for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
                S.local_dots(V, ld, j + 1, w);
                const std::vector<double> hp = S.allreduce(j + 1);
                PGB_CUDA(cudaMemcpyAsync(hd, hp.data(), 8 * (j + 1), cudaMemcpyHostToDevice, s));
                k_sh_update<<<nblk(nl, 256), 256, 0, s>>>(V, ld, j + 1, hd, w, nl);
                PGB_LAUNCHED(c, 1);
                for (int i = 0; i <= j; ++i) h[i] += hp[i];
            }
            const double nrm = S.norm(w);
            h[j + 1] = nrm;
            if (nrm > 0) k_sh_scale<<<nblk(nl, 256), 256, 0, s>>>(w, 1.0 / nrm, V + (size_t)(j + 1) * ld, nl);
            // Givens on the (replicated) Hessenberg column
            for (int i = 0; i < j; ++i) {
                const double a = cs[i] * h[i] + sn[i] * h[i + 1];
                const double bb = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = a;
                h[i + 1] = bb;
            }
            const double r = hypot(h[j], h[j + 1]);
            cs[j] = r > 0 ? h[j] / r : 1.0;
            sn[j] = r > 0 ? h[j + 1] / r : 0.0;
            h[j] = r;
            h[j + 1] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            est = fabs(g[j + 1]);
            if (est <= abs_tol || !(nrm > 0)) {
                ++j;
                ++it;
                break;
            }
        }
        // x += V y, y from the triangular system H y = g (host; replicated)
        std::vector<double> y(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k < j; ++k) t -= H[(size_t)k * (m + 1) + i] * y[k];
            y[i] = t / H[(size_t)i * (m + 1) + i];
        }
        if (j > 0) {
            // x += V y as x -= (-y) V with the update kernel
            for (int i = 0; i < j; ++i) y[i] = -y[i];
            PGB_CUDA(cudaMemcpyAsync(hd, y.data(), 8 * j, cudaMemcpyHostToDevice, s));
            k_sh_update<<<nblk(nl, 256), 256, 0, s>>>(V, ld, j, hd, x, nl);
            PGB_CUDA(cudaStreamSynchronize(s));  // y lives on the host stack
        }
        if (est <= abs_tol) break;
    }
    if (est_out) *est_out = est;
    return it;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_shard_partition(const double* work, int64_t n_groups, int32_t world, int64_t* bounds) {
    if (!work || !bounds || n_groups < 0 || world < 1) return PGB_EINVAL;
    for (int64_t g = 0; g < n_groups; ++g)
        if (!(work[g] >= 0) || !isfinite(work[g])) return PGB_EINVAL;
    shard_partition(work, n_groups, world, bounds);
    return PGB_OK;
}

int pgb_shard_rows(pgb_ctx* c, int32_t world, int64_t* row_begin) {
    if (!c || !row_begin || world < 1) return PGB_EINVAL;
    try {
        AllocScope scope(c->stream);
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        std::vector<int64_t> gb, rb;
        shard_ranges(c, world, gb, rb);
        for (int r = 0; r <= world; ++r) row_begin[r] = rb[r];
        return PGB_OK;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.code;
    }
}

int pgb_to_sharded(pgb_ctx* c, const double* x, double* xs, int32_t inverse) {
    if (!c || !x || !xs) return PGB_EINVAL;
    try {
        AllocScope scope(c->stream);
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        if (inverse) k_from_sharded<<<nblk(c->n_pan, 128), 128, 0, c->stream>>>(geo(c), body_dev(c), x, xs);
        else k_to_sharded<<<nblk(c->n_pan, 128), 128, 0, c->stream>>>(geo(c), body_dev(c), x, xs);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
        return PGB_OK;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.code;
    }
}

int pgb_matvec_shard(pgb_ctx* c, int32_t rank, int32_t world, const double* xs, double* ys, int32_t precision) {
    if (!c || !xs || !ys || world < 1 || rank < 0 || rank >= world) return PGB_EINVAL;
    try {
        AllocScope scope(c->stream);
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        if (precision != PGB_FP32 && precision != PGB_FP64 && precision != PGB_FP64_DS)
            fail(PGB_EINVAL, "precision must be PGB_FP32, PGB_FP64 or PGB_FP64_DS");
        if (nested(c)) fail(PGB_EINVAL, "sharded products do not take nested interfaces");
        std::vector<int64_t> gb, rb;
        shard_ranges(c, world, gb, rb);
        shard_product(c, gb, rb, rank, xs, ys, precision);
        return PGB_OK;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.code;
    }
}

int pgb_solve_shard(pgb_ctx* c, int32_t rank, int32_t world, double* xs, double* red, pgb_collective_fn coll,
                    void* user, int32_t mode, double tol, int32_t max_iter, int32_t restart, double* x_out,
                    pgb_solve_stats* st) {
    if (!c || !xs || !red || !coll || !x_out || world < 1 || rank < 0 || rank >= world) return PGB_EINVAL;
    try {
        AllocScope scope(c->stream);
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        if (mode != PGB_FP64 && mode != PGB_FP32_REFINE) fail(PGB_EINVAL, "mode must be PGB_FP64 or PGB_FP32_REFINE");
        if (!(tol > 0) || max_iter < 1 || restart < 1 || restart > 256) fail(PGB_EINVAL, "bad tol, max_iter or restart");
        if (nested(c)) fail(PGB_EINVAL, "sharded solves do not take nested interfaces");
        ShardRun S{c, rank, world, {}, {}, xs, red, coll, user};
        shard_ranges(c, world, S.gb, S.rb);
        const int64_t n = c->n_unk, nl = S.nl();
        cudaStream_t s = c->stream;
        // right-hand side (every rank forms it whole; its rows are kept) and
        // the Coulomb rows of the refinement's outer residual
        c->d_b.resize(n);
        c->d_bc.resize(n);
        c->d_shard_tmp.resize(n);
        coulomb_rows(c, c->d_bc);
        build_rhs(c, c->d_b, mode == PGB_FP64 ? PGB_FP64 : PGB_FP32, c->d_bc);
        c->d_shard_b.resize(std::max<int64_t>(nl, 1));
        c->d_shard_bc.resize(std::max<int64_t>(nl, 1));
        c->d_shard_x.resize(std::max<int64_t>(nl, 1));
        c->d_shard_r.resize(std::max<int64_t>(nl, 1));
        c->d_shard_d.resize(std::max<int64_t>(nl, 1));
        k_to_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), c->d_b, c->d_shard_tmp);
        PGB_CUDA(cudaMemcpyAsync(c->d_shard_b.p, c->d_shard_tmp.p + S.rb[rank], 8 * nl, cudaMemcpyDeviceToDevice, s));
        k_to_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), c->d_bc, c->d_shard_tmp);
        PGB_CUDA(cudaMemcpyAsync(c->d_shard_bc.p, c->d_shard_tmp.p + S.rb[rank], 8 * nl, cudaMemcpyDeviceToDevice,
                                 s));
        PGB_CUDA(cudaMemsetAsync(c->d_shard_x.p, 0, 8 * std::max<int64_t>(nl, 1), s));
        PGB_LAUNCHED(c, 2);
        pgb_solve_stats z{};
        const double bnorm = S.norm(c->d_shard_b);
        double rel = 0;
        if (bnorm > 0) {
            if (mode == PGB_FP64) {
                int mv = 0;
                z.iterations = shard_gmres(S, PGB_FP64, c->d_shard_b, c->d_shard_x, tol * bnorm, max_iter, restart,
                                           &mv, nullptr);
                z.matvecs = z.matvecs_fp64 = mv + 1;
                z.outer_steps = 1;
                S.gather(c->d_shard_x);
                shard_product(c, S.gb, S.rb, rank, xs, c->d_shard_r, PGB_FP64);
                k_sh_axpby<<<nblk(nl, 256), 256, 0, s>>>(1.0, c->d_shard_b, -1.0, c->d_shard_r, c->d_shard_r, nl);
                rel = S.norm(c->d_shard_r) / bnorm;
            } else {
                // refinement: inner FP32 solves, outer residual b_Coulomb -
                // A64(x + imposed) in the FP64-class product
                PGB_CUDA(cudaMemcpyAsync(c->d_shard_r.p, c->d_shard_b.p, 8 * nl, cudaMemcpyDeviceToDevice, s));
                double rn = bnorm;
                rel = 1.0;
                while (rel > tol && z.iterations < max_iter && z.outer_steps < 50) {
                    const double inner = std::max(0.5 * tol * bnorm / rn, 1e-7);
                    PGB_CUDA(cudaMemsetAsync(c->d_shard_d.p, 0, 8 * std::max<int64_t>(nl, 1), s));
                    int mv = 0;
                    const int it = shard_gmres(S, PGB_FP32, c->d_shard_r, c->d_shard_d, inner * rn,
                                               max_iter - z.iterations, restart, &mv, nullptr);
                    z.iterations += it;
                    z.matvecs += mv;
                    ++z.outer_steps;
                    k_sh_axpby<<<nblk(nl, 256), 256, 0, s>>>(1.0, c->d_shard_x, 1.0, c->d_shard_d, c->d_shard_x, nl);
                    // r = b_Coulomb - A64(x + imposed): the whole product (mode 2)
                    S.gather(c->d_shard_x);
                    k_from_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), xs, c->d_xtmp);
                    c->shard_g[0] = S.gb[rank];
                    c->shard_g[1] = S.gb[rank + 1];
                    try {
                        apply_full(c, c->d_xtmp, c->d_ytmp, c->p.residual ? PGB_FP64_DS : PGB_FP64);
                    } catch (...) {
                        c->shard_g[0] = c->shard_g[1] = -1;
                        throw;
                    }
                    c->shard_g[0] = c->shard_g[1] = -1;
                    k_to_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), c->d_ytmp, c->d_shard_tmp);
                    k_sh_axpby<<<nblk(nl, 256), 256, 0, s>>>(1.0, c->d_shard_bc, -1.0, c->d_shard_tmp.p + S.rb[rank],
                                                             c->d_shard_r, nl);
                    PGB_LAUNCHED(c, 4);
                    ++z.matvecs;
                    ++z.matvecs_fp64;
                    const double rn_new = S.norm(c->d_shard_r);
                    rel = rn_new / bnorm;
                    if (it == 0 || !(rn_new < rn)) break;
                    rn = rn_new;
                }
            }
        }
        z.rel_residual = rel;
        // every rank's rows of x, then the whole solution in the caller's order
        S.gather(c->d_shard_x);
        k_from_sharded<<<nblk(c->n_pan, 128), 128, 0, s>>>(geo(c), body_dev(c), xs, x_out);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
        if (st) *st = z;
        return rel <= tol ? PGB_OK : PGB_ENOCONV;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.code;
    }
}

}  // extern "C"
