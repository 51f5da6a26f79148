// Batched pose solve: B independent problems (poses of one molecule, or of
// several molecules of different sizes) solved as ONE block-diagonal system.
// The problems' bodies sit side by side in one context; interaction lists
// and near-field entries never cross problems, so the treecode product of
// the union is the B products at once, and each stage (tree, lists, P2M,
// P2P, M2P, assembly, the Arnoldi step) is one launch over all problems.
// GMRES runs in lockstep: one product per iteration for the whole system,
// while every problem keeps its own Krylov coefficients (Hessenberg matrix,
// Givens rotations), its own stopping test and its own refinement steps, so
// each problem's iterate is exactly the one a solve of it alone would
// produce (up to the rounding of the shared kernels).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "pgb_internal.cuh"

namespace pgb {

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

#define SEG_THREADS 256

// part[p * nbp + bx] = sum of a . b over block bx's rows of problem p
__global__ void __launch_bounds__(SEG_THREADS) k_seg_dot(const double* __restrict__ a, const double* __restrict__ b,
                                                         const int64_t* __restrict__ poff, double* part) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    const int64_t hi = poff[p + 1], stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0;
    for (int64_t r = poff[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < hi; r += stride) s += a[r] * b[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[(int64_t)p * gridDim.x + blockIdx.x] = s;
}

// out[p] = sum_b part[p * nbp + b] (its square root when sqrt_out)
__global__ void k_seg_sum(const double* __restrict__ part, int nbp, double* out, int sqrt_out) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < nbp; b += blockDim.x) s += part[(int64_t)p * nbp + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[p] = sqrt_out ? sqrt(s) : s;
}

// v = w / nrm[p] on the rows of problem p (0 where nrm[p] == 0)
__global__ void k_seg_scale(const double* __restrict__ w, const double* __restrict__ nrm,
                            const int64_t* __restrict__ poff, double* v) {
    const int p = blockIdx.y;
    const double a = nrm[p];
    const double inv = a > 0 ? 1.0 / a : 0.0;
    const int64_t hi = poff[p + 1], stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = poff[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < hi; r += stride) v[r] = w[r] * inv;
}

// g_p = (beta_p, 0, ..., 0), m1 entries
__global__ void k_seg_init_g(double* g, int64_t sV, int m1, const double* beta) {
    const int p = blockIdx.x;
    for (int i = threadIdx.x; i < m1; i += blockDim.x) g[p * sV + i] = i == 0 ? beta[p] : 0.0;
}

// y_p = H_p(0:k, 0:k)^{-1} g_p(0:k), k = kcol[p] (upper triangular; one
// thread per problem)
__global__ void k_seg_backsolve(const double* H, int ld, int64_t sH, const double* g, int64_t sV, const int* kcol,
                                double* y, int B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B) return;
    const double* Hp = H + p * sH;
    const double* gp = g + p * sV;
    double* yp = y + p * sV;
    const int k = kcol[p];
    for (int i = k - 1; i >= 0; --i) {
        double s = gp[i];
        for (int j = i + 1; j < k; ++j) s -= Hp[(int64_t)j * ld + i] * yp[j];
        yp[i] = Hp[(int64_t)i * ld + i] != 0 ? s / Hp[(int64_t)i * ld + i] : 0.0;
    }
}

// x += sum_{i < kcol[p]} y_p[i] V_i on the rows of problem p
__global__ void k_seg_axpy(const double* __restrict__ V, int64_t ld, const int* __restrict__ kcol,
                           const double* __restrict__ y, int64_t sV, const int64_t* __restrict__ poff, double* x) {
    const int p = blockIdx.y;
    const int k = kcol[p];
    if (k == 0) return;
    const double* yp = y + p * sV;
    const int64_t hi = poff[p + 1], stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = poff[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < hi; r += stride) {
        double s = 0;
        for (int i = 0; i < k; ++i) s += yp[i] * V[i * ld + r];
        x[r] += s;
    }
}

__global__ void k_seg_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = a * x[r] + b * y[r];
}

// ---------------------------------------------------------------- replayed lockstep iterations
// The column the next replayed product reads: dst = V_j, j from the device.
__global__ void k_seg_select(const double* __restrict__ V, int64_t n, const int* __restrict__ jdev,
                             double* __restrict__ dst) {
    const int64_t j = *jdev;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        dst[r] = V[j * n + r];
}

// After the segmented Arnoldi step of column j, one thread per problem (at
// most 64): an active problem counts the column, keeps its estimate and
// leaves when it meets its tolerance or breaks down; the body mask of the
// next product keeps the problems still active; j advances and the loop goes
// on while a problem is active and columns remain (j + 1 < *jmax).
// ctl: {j, jmax}.
__global__ void __launch_bounds__(64) k_seg_check(const double* __restrict__ out, int B, int* act, int* kcol, int* itc,
                                                  double* estd, const double* __restrict__ told,
                                                  const unsigned long long* __restrict__ pmask,
                                                  unsigned long long* bmask, int* ctl, cudaGraphConditionalHandle h) {
    __shared__ unsigned long long keep;
    __shared__ int any;
    if (threadIdx.x == 0) {
        keep = 0;
        any = 0;
    }
    __syncthreads();
    const int j = ctl[0];
    const int p = threadIdx.x;
    if (p < B && act[p]) {
        kcol[p] = j + 1;
        ++itc[p];
        const double est = out[2 * p], hnext = out[2 * p + 1];
        estd[p] = est;
        if (est <= told[p] || !(hnext > 0)) {
            act[p] = 0;
        } else {
            atomicOr(&keep, pmask[p]);
            any = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl[0] = j + 1;
        *bmask = keep;
        cudaGraphSetConditional(h, (any && j + 1 < ctl[1]) ? 1u : 0u);
    }
}

// Leave the problems with on[p] == 0 out of the following products (their
// rows come out without the treecode sums and are not used).
static void set_products(pgb_ctx* c, const std::vector<int>& on) {
    for (int p = 0; p < c->n_prob; ++p)
        for (int k = c->prob_first[p]; k < c->prob_first[p + 1]; ++k) c->body_off[k] = !on[p];
}

static void all_products(pgb_ctx* c) {
    for (int k = 0; k < PGB_MAX_BODIES; ++k) c->body_off[k] = 0;
}

// Per-problem 2-norms of v (host copy).
static std::vector<double> seg_norms(pgb_ctx* c, const double* v) {
    const int B = c->n_prob, nbp = c->seg_nbp;
    cudaStream_t s = c->stream;
    c->d_seg_red.resize((size_t)nbp * B + B);
    double* out = c->d_seg_red.p + (size_t)nbp * B;
    k_seg_dot<<<dim3(nbp, B), SEG_THREADS, 0, s>>>(v, v, c->d_poff, c->d_seg_red);
    k_seg_sum<<<B, 128, 0, s>>>(c->d_seg_red, nbp, out, 1);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 2);
    std::vector<double> h(B);
    PGB_CUDA(cudaMemcpyAsync(h.data(), out, 8 * B, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    return h;
}

// Graph of the lockstep iterations after the first column of a cycle: a
// device-side while loop whose body takes column j (k_seg_select), applies
// the (preconditioned) operator to the problems the run-time body mask keeps,
// makes the segmented Arnoldi step of column j and updates every problem's
// state (k_seg_check).  Captured on the context's capture stream from the
// launches the host loop makes; the caller sizes every buffer first.
template <class ApplyPc>
static void seg_graph_capture(pgb_ctx* c, const ArnSeg& sg, int m, double* hc, double* cs, double* sn, double* g,
                              double* out, int* act, int* kcol, int* itc, double* estd, const double* told, int* ctl,
                              ApplyPc apply_pc) {
    const int64_t n = c->n_unk;
    const int B = c->n_prob;
    if (c->seg_exec) {
        PGB_CUDA(cudaGraphExecDestroy(c->seg_exec));
        c->seg_exec = nullptr;
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
    c->dev_bmask = c->d_segm.p;
    all_products(c);
    std::string why;
    PGB_CUDA(cudaStreamBeginCaptureToGraph(c->gm_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        k_seg_select<<<nblk(n, 256), 256, 0, c->gm_stream>>>(c->d_V, n, ctl, c->d_xsel);
        apply_pc(c->d_xsel.p, c->d_wk.p);
        arnoldi_step(c, 0, c->d_wk, c->d_H, hc, cs, sn, g, out, &sg, ctl, m);
        k_seg_check<<<1, 64, 0, c->gm_stream>>>(out, B, act, kcol, itc, estd, told, c->d_segm.p + 1, c->d_segm.p,
                                                 ctl, h);
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
    c->dev_bmask = nullptr;
    c->seg_body_launches = c->launches - l0;
    c->launches = l0;
    if (!why.empty() || le != cudaSuccess || ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        fail(PGB_ECUDA, "lockstep iteration graph capture: " +
                            (why.empty() ? std::string(cudaGetErrorString(le != cudaSuccess ? le : ce)) : why));
    }
    const cudaError_t ie = cudaGraphInstantiate(&c->seg_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) c->seg_exec = nullptr;
    PGB_CUDA(ie);
}

// Lockstep restarted GMRES on the c->n_prob problems of a block-diagonal
// system: each iteration is one product of the whole system and one
// segmented Arnoldi step; problem p stops on its own test (estimated
// residual <= abs_tol[p]) and then takes no further part (the products
// leave its sources out and its rows unused).  x_zero: x = 0 on entry.  iters[p]
// receives p's iterations, est[p] its last estimate; returns the lockstep
// iteration count.
static int gmres_seg(pgb_ctx* c, int prec, const double* b, double* x, const double* abs_tol, int max_it,
                     int restart, int* matvecs, int* iters, double* est, bool x_zero) {
    const bool pc = c->p.precond && c->pc_ready;
    const int B = c->n_prob, nbp = c->seg_nbp, m = restart;
    const int64_t n = c->n_unk, sV = m + 1, sH = (int64_t)(m + 1) * m;
    cudaStream_t s = c->stream;
    auto apply_pc = [&](const double* in, double* out) {
        if (!pc) return apply_operator(c, in, out, prec, false);
        precond_apply(c, in, c->d_pz, false, false);
        apply_operator(c, c->d_pz, out, prec, false);
    };
    c->d_V.resize((size_t)(m + 1) * n);
    c->d_H.resize((size_t)B * sH);
    c->d_wk.resize(n);
    c->d_seg.resize((size_t)5 * B * sV + 5 * B);
    c->d_segi.resize(3 * (size_t)B + 2);
    if (pc) c->d_pz.resize(n);
    double* cs = c->d_seg.p;
    double* sn = cs + B * sV;
    double* g = sn + B * sV;
    double* hc = g + B * sV;
    double* yv = hc + B * sV;
    double* out = yv + B * sV;  // 2 per problem
    double* nrm = out + 2 * B;  // 1 per problem
    double* estd = nrm + B;     // replayed iterations: each problem's last estimate
    double* told = estd + B;    // and its tolerance
    int* act = c->d_segi.p;
    int* kcol = act + B;
    int* itc = kcol + B;        // replayed iterations: columns each problem made
    int* ctl = itc + B;         // {column j, column limit}
    const ArnSeg sg{B, nbp, c->d_poff, act, sH, sV};
    std::vector<char> done(B, 0);
    std::vector<int> act_h(B, 0), kcol_h(B, 0);
    std::vector<double> hb(2 * B);
    for (int p = 0; p < B; ++p) {
        iters[p] = 0;
        est[p] = INFINITY;
    }
    // the iterations after a cycle's first column replayed from a graph
    // (captured afresh in each call, on its first use)
    const bool graph = c->p.graphs >= 2 && m >= 2 && B <= 64;
    std::vector<unsigned long long> pm(B + 1, 0);
    std::vector<int> ib(3 * B + 2);
    if (c->seg_exec) {
        PGB_CUDA(cudaGraphExecDestroy(c->seg_exec));
        c->seg_exec = nullptr;
    }
    if (graph) {
        // everything the replayed body touches is sized here, outside the capture
        c->d_segm.resize(B + 1);
        c->d_xsel.resize(n);
        reserve_product(c, prec);
        c->d_red.resize(std::max<size_t>(c->d_red.n, (size_t)2 * nbp * (m + 1) * B));
        for (int p = 0; p < B; ++p)
            for (int k = c->prob_first[p]; k < c->prob_first[p + 1]; ++k) pm[1 + p] |= 1ull << k;
        PGB_CUDA(cudaMemcpyAsync(c->d_segm.p + 1, pm.data() + 1, 8 * B, cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(told, abs_tol, 8 * B, cudaMemcpyHostToDevice, s));
    }
    int it = 0;
    while (it < max_it) {
        // r = b - A x (x = 0 on entry needs no product)
        if (x_zero) {
            PGB_CUDA(cudaMemcpyAsync(c->d_wk.p, b, 8 * n, cudaMemcpyDeviceToDevice, s));
            x_zero = false;
        } else {
            for (int p = 0; p < B; ++p) act_h[p] = !done[p];
            set_products(c, act_h);
            apply_operator(c, x, c->d_wk, prec, false);
            ++*matvecs;
            k_seg_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, b, -1.0, c->d_wk, c->d_wk, n);
            PGB_LAUNCHED(c, 1);
        }
        const std::vector<double> beta = seg_norms(c, c->d_wk);
        bool any = false;
        for (int p = 0; p < B; ++p) {
            if (!done[p]) {
                est[p] = beta[p];
                if (beta[p] <= abs_tol[p] || beta[p] == 0) done[p] = 1;
            }
            act_h[p] = !done[p];
            any = any || act_h[p];
        }
        if (!any) break;
        PGB_CUDA(cudaMemcpyAsync(nrm, c->d_seg_red.p + (size_t)nbp * B, 8 * B, cudaMemcpyDeviceToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(act, act_h.data(), 4 * B, cudaMemcpyHostToDevice, s));
        k_seg_scale<<<dim3(nbp, B), SEG_THREADS, 0, s>>>(c->d_wk, nrm, c->d_poff, c->d_V);
        k_seg_init_g<<<B, 64, 0, s>>>(g, sV, m + 1, nrm);
        PGB_LAUNCHED(c, 2);
        std::fill(kcol_h.begin(), kcol_h.end(), 0);
        for (int j = 0; j < m && it < max_it; ++j) {
            set_products(c, act_h);
            apply_pc(c->d_V.p + (size_t)j * n, c->d_wk);
            ++*matvecs;
            ++it;
            {
                StageTimer tm(c, PGB_STAGE_KRYLOV);
                arnoldi_step(c, j, c->d_wk, c->d_H.p + (size_t)j * (m + 1), hc, cs, sn, g, out, &sg);
                PGB_LAUNCHED(c, 4);
            }
            PGB_CUDA(cudaMemcpyAsync(hb.data(), out, 16 * B, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            bool left = false, changed = false;
            for (int p = 0; p < B; ++p) {
                if (!act_h[p]) continue;
                kcol_h[p] = j + 1;
                ++iters[p];
                est[p] = hb[2 * p];
                const double hnext = hb[2 * p + 1];
                if (est[p] <= abs_tol[p] || !(hnext > 0)) {
                    act_h[p] = 0;  // converged, or breakdown (restart next cycle)
                    changed = true;
                    if (est[p] <= abs_tol[p]) done[p] = 1;
                } else {
                    left = true;
                }
            }
            if (!left) break;
            if (changed) PGB_CUDA(cudaMemcpyAsync(act, act_h.data(), 4 * B, cudaMemcpyHostToDevice, s));
            if (graph && j == 0 && j + 1 < m && it < max_it) {
                // columns 1 .. from the graph: the first column sized every
                // buffer the body touches
                if (!c->seg_exec)
                    seg_graph_capture(c, sg, m, hc, cs, sn, g, out, act, kcol, itc, estd, told, ctl, apply_pc);
                const int jmax = (int)std::min<int64_t>(m, (int64_t)j + 1 + (max_it - it));
                unsigned long long keep = 0;
                for (int p = 0; p < B; ++p) {
                    ib[p] = act_h[p];
                    ib[B + p] = kcol_h[p];
                    ib[2 * B + p] = 0;
                    if (act_h[p]) keep |= pm[1 + p];
                }
                ib[3 * B] = 1;
                ib[3 * B + 1] = jmax;
                pm[0] = keep;
                PGB_CUDA(cudaMemcpyAsync(act, ib.data(), 4 * (3 * B + 2), cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaMemcpyAsync(c->d_segm.p, pm.data(), 8, cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaGraphLaunch(c->seg_exec, s));
                std::vector<double> eh(B);
                PGB_CUDA(cudaMemcpyAsync(ib.data(), act, 4 * (3 * B + 2), cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaMemcpyAsync(eh.data(), estd, 8 * B, cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaStreamSynchronize(s));
                const int cols = ib[3 * B] - 1;  // columns the graph made
                for (int p = 0; p < B; ++p) {
                    if (!act_h[p]) continue;
                    iters[p] += ib[2 * B + p];
                    if (ib[2 * B + p] > 0) {
                        est[p] = eh[p];
                        kcol_h[p] = ib[B + p];
                    }
                    if (!ib[p]) {
                        act_h[p] = 0;
                        if (est[p] <= abs_tol[p]) done[p] = 1;
                    }
                }
                it += cols;
                *matvecs += cols;
                c->launches += cols * c->seg_body_launches;
                c->graph_kernels += cols * c->seg_body_launches;
                ++c->graph_launches;
                break;
            }
        }
        // x += M^{-1} V y, problem by problem with its own column count
        PGB_CUDA(cudaMemcpyAsync(kcol, kcol_h.data(), 4 * B, cudaMemcpyHostToDevice, s));
        k_seg_backsolve<<<nblk(B, 32), 32, 0, s>>>(c->d_H, m + 1, sH, g, sV, kcol, yv, B);
        if (pc) {
            PGB_CUDA(cudaMemsetAsync(c->d_pz.p, 0, 8 * n, s));
            k_seg_axpy<<<dim3(nbp, B), SEG_THREADS, 0, s>>>(c->d_V, n, kcol, yv, sV, c->d_poff, c->d_pz);
            precond_apply(c, c->d_pz, x, false, true);
        } else {
            k_seg_axpy<<<dim3(nbp, B), SEG_THREADS, 0, s>>>(c->d_V, n, kcol, yv, sV, c->d_poff, x);
        }
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 2);
        bool all = true;
        for (int p = 0; p < B; ++p) all = all && done[p];
        if (all) break;
    }
    all_products(c);
    return it;
}

// Solve of the c->n_prob problems of the context (modes as solve()); the
// statistics of problem p into st[p].  PGB_OK when every problem met tol.
int solve_seg(pgb_ctx* c, int mode, double tol, int max_iter, int restart, double* x, pgb_solve_stats* st) {
    const int B = c->n_prob;
    const int64_t n = c->n_unk;
    cudaStream_t s = c->stream;
    if (mode != PGB_FP64 && mode != PGB_FP32_REFINE && mode != PGB_FP32)
        fail(PGB_EINVAL, "mode must be PGB_FP64, PGB_FP32_REFINE or PGB_FP32");
    c->d_b.resize(n);
    c->d_r.resize(n);
    c->d_xs.resize(n);
    const int rhs_prec = mode == PGB_FP64 ? PGB_FP64 : PGB_FP32;
    if (mode == PGB_FP32_REFINE) {  // Coulomb rows once: the outer residual's and the right-hand side's
        c->d_bc.resize(n);
        coulomb_rows(c, c->d_bc);
        build_rhs(c, c->d_b, rhs_prec, c->d_bc);
    } else {
        build_rhs(c, c->d_b, rhs_prec);
    }
    precond_prepare(c);
    int known_mv = 0;
    for (auto& b : c->bodies)
        if (b.kind != PGB_DIELECTRIC) known_mv = 1;
    std::vector<pgb_solve_stats> z(B);
    for (auto& q : z) {
        q = pgb_solve_stats{};
        q.matvecs = known_mv;
        q.matvecs_fp64 = rhs_prec == PGB_FP64 ? known_mv : 0;
    }
    const std::vector<double> bn = seg_norms(c, c->d_b);
    PGB_CUDA(cudaMemsetAsync(x, 0, 8 * n, s));
    std::vector<double> rel(B, 0.0), tolv(B), est(B);
    std::vector<int> its(B);
    if (mode != PGB_FP32_REFINE) {
        const int prec = mode == PGB_FP64 ? PGB_FP64 : PGB_FP32;
        for (int p = 0; p < B; ++p) tolv[p] = tol * bn[p];
        int mv = 0;
        gmres_seg(c, prec, c->d_b, x, tolv.data(), max_iter, restart, &mv, its.data(), est.data(), true);
        apply_operator(c, x, c->d_r, prec, false);
        k_seg_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_b, -1.0, c->d_r, c->d_r, n);
        PGB_LAUNCHED(c, 1);
        const std::vector<double> rn = seg_norms(c, c->d_r);
        for (int p = 0; p < B; ++p) {
            z[p].iterations = its[p];
            z[p].matvecs += mv + 1;
            if (prec == PGB_FP64) z[p].matvecs_fp64 += mv + 1;
            z[p].outer_steps = 1;
            rel[p] = bn[p] > 0 ? rn[p] / bn[p] : 0.0;
        }
    } else {
        // refinement as in solve(), per problem: inner FP32 solves aimed at
        // the final tolerance, the outer residual b_Coulomb - A64(x +
        // imposed) in FP64; a problem leaves when it meets tol or stalls
        PGB_CUDA(cudaMemcpyAsync(c->d_r.p, c->d_b.p, 8 * n, cudaMemcpyDeviceToDevice, s));
        std::vector<double> rn = bn;
        std::vector<char> done(B);
        for (int p = 0; p < B; ++p) {
            done[p] = !(bn[p] > 0);
            rel[p] = done[p] ? 0.0 : 1.0;
        }
        int total = 0, outer = 0;
        auto any_left = [&]() {
            for (int p = 0; p < B; ++p)
                if (!done[p]) return true;
            return false;
        };
        while (any_left() && total < max_iter && outer < 50) {
            for (int p = 0; p < B; ++p) {
                const double inner = std::max(0.5 * tol * bn[p] / rn[p], 1e-7);
                tolv[p] = done[p] ? INFINITY : inner * rn[p];
            }
            PGB_CUDA(cudaMemsetAsync(c->d_xs.p, 0, 8 * n, s));
            int mv = 0;
            const int it = gmres_seg(c, PGB_FP32, c->d_r, c->d_xs, tolv.data(), max_iter - total, restart, &mv,
                                     its.data(), est.data(), true);
            total += it;
            ++outer;
            k_seg_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, x, 1.0, c->d_xs, x, n);
            std::vector<int> on(B);
            for (int p = 0; p < B; ++p) on[p] = !done[p];
            set_products(c, on);
            apply_full(c, x, c->d_r, c->p.residual ? PGB_FP64_DS : PGB_FP64);
            all_products(c);
            k_seg_axpby<<<nblk(n, 256), 256, 0, s>>>(1.0, c->d_bc, -1.0, c->d_r, c->d_r, n);
            PGB_LAUNCHED(c, 2);
            const std::vector<double> rnew = seg_norms(c, c->d_r);
            for (int p = 0; p < B; ++p) {
                if (done[p]) continue;
                z[p].iterations += its[p];
                z[p].matvecs += mv + 1;
                ++z[p].matvecs_fp64;
                ++z[p].outer_steps;
                rel[p] = rnew[p] / bn[p];
                if (rel[p] <= tol || its[p] == 0 || !(rnew[p] < rn[p])) done[p] = 1;
                rn[p] = rnew[p];
            }
            if (it == 0) break;
        }
    }
    PGB_CUDA(cudaGetLastError());
    bool ok = true;
    for (int p = 0; p < B; ++p) {
        z[p].rel_residual = rel[p];
        ok = ok && rel[p] <= tol;
        if (st) st[p] = z[p];
    }
    return ok ? PGB_OK : PGB_ENOCONV;
}

// ---------------------------------------------------------------- the union context
void destroy_union(pgb_ctx* c) {
    if (c->union_ctx) pgb_destroy(c->union_ctx);
    c->union_ctx = nullptr;
    c->union_src.clear();
    c->union_gen.clear();
}

// The union context of the problems' source contexts src[p] (bodies copied,
// body k of problem p at index p * nb_p + k ...); rebuilt when the sequence
// of sources, their configuration or the parameters change.
static pgb_ctx* ensure_union(pgb_ctx* c, const std::vector<pgb_ctx*>& src) {
    bool ok = c->union_ctx && c->union_src == src;
    if (ok) {
        for (size_t p = 0; p < src.size() && ok; ++p) ok = c->union_gen[p] == src[p]->config_gen;
        const pgb_params &a = c->union_ctx->p, &b = c->p;
        ok = ok && a.K == b.K && a.K_near == b.K_near && a.n_edge == b.n_edge && a.P == b.P && a.theta == b.theta &&
             a.leaf_size == b.leaf_size && a.p2p_item == b.p2p_item && a.m2p_item == b.m2p_item &&
             a.precond == b.precond && a.graphs == b.graphs && a.residual == b.residual &&
             c->union_ctx->eps_out == c->eps_out &&
             c->union_ctx->kappa == c->kappa;
    }
    if (ok) return c->union_ctx;
    destroy_union(c);
    size_t nbod = 0;
    for (pgb_ctx* q : src) {
        if (q->eps_out != c->eps_out || q->kappa != c->kappa)
            fail(PGB_EINVAL, "every context of a pose batch needs the solvent (eps_out, kappa) of the first");
        if (q->bodies.empty()) fail(PGB_ESTATE, "a context of the pose batch has no bodies");
        if (nested(q)) fail(PGB_EINVAL, "pose batches do not take nested interfaces (use lanes)");
        nbod += q->bodies.size();
    }
    if (nbod > PGB_MAX_BODIES)
        fail(PGB_EINVAL, "a pose batch holds at most " + std::to_string(PGB_MAX_BODIES) + " bodies in all; this one " +
                             std::to_string(nbod) + " (lower pgb_params.batch)");
    pgb_ctx* u = new pgb_ctx;
    u->p = c->p;
    u->p.lanes = 1;
    u->p.overlap = 0;
    u->eps_out = c->eps_out;
    u->kappa = c->kappa;
    for (size_t p = 0; p < src.size(); ++p) {
        u->prob_first.push_back((int)u->bodies.size());
        for (const Body& b : src[p]->bodies) {
            u->bodies.push_back(b);
            u->bodies.back().prob = (int)p;
        }
    }
    u->prob_first.push_back((int)u->bodies.size());
    u->n_prob = (int)src.size();
    note_alloc();
    if (cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&u->h_pinned, 64) != cudaSuccess) {
        (void)cudaGetLastError();
        pgb_destroy(u);
        fail(PGB_ECUDA, "pose batch context creation failed");
    }
    u->owns_stream = true;
    c->union_ctx = u;
    c->union_src = src;
    for (pgb_ctx* q : src) c->union_gen.push_back(q->config_gen);
    return u;
}

// Problems p = 0 .. B-1: source context src[p] with body body_id at pose
// (R + 9 p, t + 3 p); the energies (Coulomb, solvation, surface, total) of
// problem p into F + 4 p.  Poses of the other bodies follow their source
// contexts.  Runs on the union's stream, ordered after c's.
int solve_union(pgb_ctx* c, const std::vector<pgb_ctx*>& src, int32_t body_id, const double* R, const double* t,
                int32_t mode, double tol, int32_t max_iter, int32_t restart, double* F, pgb_solve_stats* st) {
    pgb_ctx* u = ensure_union(c, src);
    const int B = (int)src.size();
    AllocScope scope(u->stream);
    u->timing = c->timing;
    for (int p = 0; p < B; ++p) {
        const int first = u->prob_first[p];
        for (size_t k = 0; k < src[p]->bodies.size(); ++k) {
            Body& ub = u->bodies[first + k];
            const Body& sb = src[p]->bodies[k];
            const double* Rp = (int32_t)k == body_id ? R + 9 * p : sb.R;
            const double* tp = (int32_t)k == body_id ? t + 3 * p : sb.t;
            if (memcmp(ub.R, Rp, sizeof(ub.R)) || memcmp(ub.t, tp, sizeof(ub.t))) {
                memcpy(ub.R, Rp, sizeof(ub.R));
                memcpy(ub.t, tp, sizeof(ub.t));
                u->tree_valid = false;
            }
        }
    }
    cudaEvent_t ev = nullptr;
    PGB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PGB_CUDA(cudaEventRecord(ev, c->stream));
    PGB_CUDA(cudaStreamWaitEvent(u->stream, ev, 0));
    PGB_CUDA(cudaEventDestroy(ev));
    {
        StageTimer tm(u, PGB_STAGE_TREE);
        if (!u->order_valid) {
            upload_bodies(u);
            build_order(u);
            u->intra_valid = false;
            std::vector<int64_t> po(B + 1);
            for (int p = 0; p < B; ++p) po[p] = u->bodies[u->prob_first[p]].unk_off;
            po[B] = u->n_unk;
            u->d_poff.resize(B + 1);
            PGB_CUDA(cudaMemcpyAsync(u->d_poff.p, po.data(), 8 * (B + 1), cudaMemcpyHostToDevice, u->stream));
            int dev = 0, sms = 0;
            PGB_CUDA(cudaGetDevice(&dev));
            PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            u->seg_nbp = std::max(2, (2 * sms + B - 1) / B);
        }
        if (!u->tree_valid) {
            build_geometry(u);
            build_lists(u);
            build_corrections(u);
            u->tree_valid = true;
        }
    }
    u->d_xbatch.resize(u->n_unk);
    const int rs = solve_seg(u, mode, tol, max_iter, restart, u->d_xbatch, st);
    std::vector<pgb_energies> eb(u->bodies.size());
    {
        StageTimer tm(u, PGB_STAGE_ENERGY);
        energies(u, u->d_xbatch, nullptr, eb.data());
    }
    for (int p = 0; p < B; ++p) {
        double e4[4] = {0, 0, 0, 0};
        for (int k = u->prob_first[p]; k < u->prob_first[p + 1]; ++k) {
            e4[0] += eb[k].coulomb;
            e4[1] += eb[k].solvation;
            e4[2] += eb[k].surface;
            e4[3] += eb[k].total;
        }
        for (int q = 0; q < 4; ++q) F[4 * p + q] = e4[q];
    }
    PGB_CUDA(cudaStreamSynchronize(u->stream));
    if (c->timing) {
        collect_timing(u);
        for (int k = 0; k < PGB_N_STAGES; ++k) {
            c->stage_ms[k] += u->stage_ms[k];
            c->stage_calls[k] += u->stage_calls[k];
            u->stage_ms[k] = 0;
            u->stage_calls[k] = 0;
        }
    }
    c->launches += u->launches;
    c->graph_kernels += u->graph_kernels;
    c->graph_launches += u->graph_launches;
    u->launches = u->graph_kernels = u->graph_launches = 0;
    return rs;
}

}  // namespace pgb
