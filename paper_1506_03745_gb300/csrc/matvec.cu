// Treecode matvec driver: source densities, upward pass + evaluation,
// near-field corrections and the block rows of Eq. 6 / Eq. 7.
#include <algorithm>

#include "treecode.cuh"

namespace pgb {

void treecode_launch_f32(int stage, int P, const UpArgs& up, const std::vector<int64_t>& lv, const EvalArgs& ev,
                         const void* src, const void* xrel, void* mom, void* far, cudaStream_t s);
void treecode_launch_f64(int stage, int P, const UpArgs& up, const std::vector<int64_t>& lv, const EvalArgs& ev,
                         const void* src, const void* xrel, void* mom, void* far, cudaStream_t s);
void treecode_launch_ds(int stage, int P, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel,
                        void* mom, const void* far, cudaStream_t s);
void convert_src_ds(const void* src64, void* src_ds, int64_t n, cudaStream_t s);

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// Panel densities (psi_L, psi_Y, phi) of the combined potential U = S_V - S_K
// for every sorted panel, and the per-point source terms
// A = {y - c_leaf, w psi_L}, B = {w phi n, w psi_Y}.
//   dielectric: psi_L = dphi, psi_Y = (eps_in/eps_out) dphi, phi = phi
//   imposed potential: psi_Y = u; imposed charge: phi = u
// known == true builds the imposed-boundary densities instead: phi0 as the
// double-layer density of an imposed-potential surface, dphi = -sigma0/eps_out
// as the single layer of an imposed-charge surface, zero on molecules.
// mode 0: densities of the unknowns x; 1: imposed parts only; 2: both (the
// unknowns plus the imposed sigma0 / phi0 of every surface).
template <typename real>
__global__ void k_src_prep(Geo g, BodyDev bd, const double* __restrict__ x, int mode,
                           const typename V4<real>::t* __restrict__ yrel, typename V4<real>::t* __restrict__ src,
                           real* __restrict__ dens, double eps_out) {
    const bool known = mode == 1;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    double psiL = 0, psiY = 0, phi = 0;
    const int kind = bd.kind[b];
    if (!known) {
        if (kind == PGB_DIELECTRIC) {
            phi = x[o + loc];
            psiL = x[o + N + loc];
            psiY = bd.eps_ratio[b] * psiL;
        } else if (kind == PGB_SET_POTENTIAL) {
            psiY = x[o + loc];
        } else {
            phi = x[o + loc];
        }
    } else {
        if (kind == PGB_SET_POTENTIAL) phi = bd.bc[b];
        else if (kind == PGB_SET_CHARGE) psiY = -bd.bc[b] / eps_out;
    }
    if (mode == 2) {
        if (kind == PGB_SET_POTENTIAL) phi = bd.bc[b];
        else if (kind == PGB_SET_CHARGE) psiY = -bd.bc[b] / eps_out;
    }
    // the FP32 product forms its source terms in FP32 (they are stored in
    // FP32 anyway); the FP64 product in FP64
    const real rL = (real)psiL, rY = (real)psiY, rp = (real)phi;
    dens[3 * i] = rL;
    dens[3 * i + 1] = rY;
    dens[3 * i + 2] = rp;
    const real nx = (real)g.n[3 * i], ny = (real)g.n[3 * i + 1], nz = (real)g.n[3 * i + 2];
    for (int m = 0; m < g.K; ++m) {
        const int64_t p = i * g.K + m;
        const real w = (real)g.w[p];
        typename V4<real>::t A = yrel[p], B;
        const real wp = w * rp;
        A.w = w * rL;
        B.x = wp * nx;
        B.y = wp * ny;
        B.z = wp * nz;
        B.w = w * rY;
        src[2 * p] = A;
        src[2 * p + 1] = B;
    }
}

// U += near-field corrections (FP64), then the rows of Eq. 6 / Eq. 7 in the
// caller's layout.  mode 0: y = A x.  mode 1: right-hand side of the imposed
// boundary terms, -(U + jump) on exterior and surface rows.  mode 2: the rows
// with the imposed densities included, so that b - A x = b_Coulomb - y.
// Treecode sums of panel i: the partial sums of its group's P2P items, then
// of its M2P items, in item order (a fixed order: the result does not depend
// on the schedule).
struct Parts {
    const int32_t *pan_group, *gstart;
    const int64_t *pitem_off, *fitem_off;
    const double *Up, *Uf;
    int64_t g_lo, g_hi;  // rows of the groups g_lo <= g < g_hi only (a rank's rows of a sharded product)
};

// real: the arithmetic of the near-field corrections (FP32 product: FP32
// copies of the FP64-computed corrections; FP64 product: FP64).
template <typename real>
__global__ void k_assemble(Geo g, BodyDev bd, Parts u, const real* __restrict__ dens,
                           const int64_t* __restrict__ coff, const int32_t* __restrict__ cj,
                           const typename V4<real>::t* __restrict__ cval, const int64_t* __restrict__ xoff,
                           const int32_t* __restrict__ xj, const typename V4<real>::t* __restrict__ xval, int mode,
                           const double* __restrict__ x, double* __restrict__ y) {
    using v4 = typename V4<real>::t;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const double inv4pi = 1.0 / PGB_FOUR_PI;
    const int gi = u.pan_group[i];
    if (gi < u.g_lo || gi >= u.g_hi) return;
    const int lane = (int)(i - u.gstart[gi]);
    double sL = 0, sY = 0;
    for (int64_t it = u.pitem_off[gi]; it < u.pitem_off[gi + 1]; ++it) {
        sL += u.Up[64 * it + lane];
        sY += u.Up[64 * it + 32 + lane];
    }
    for (int64_t it = u.fitem_off[gi]; it < u.fitem_off[gi + 1]; ++it) {
        sL += u.Uf[64 * it + lane];
        sY += u.Uf[64 * it + 32 + lane];
    }
    double UL = sL * inv4pi, UY = sY * inv4pi;
    // corrections: FP32 products with compensated sums in the FP32 product,
    // plain FP64 in the FP64 one
    real cL = 0, eL = 0, cY = 0, eY = 0;
    for (int64_t e = coff[i]; e < coff[i + 1]; ++e) {
        const int64_t j = cj[e];
        const v4 d = cval[e];
        const real psiL = dens[3 * j], psiY = dens[3 * j + 1], phi = dens[3 * j + 2];
        if (sizeof(real) == 4) {
            kadd(cL, eL, d.x * psiL - d.y * phi);
            kadd(cY, eY, d.z * psiY - d.w * phi);
        } else {
            cL += d.x * psiL - d.y * phi;
            cY += d.z * psiY - d.w * phi;
        }
    }
    for (int64_t e = xoff[i]; e < xoff[i + 1]; ++e) {  // cross-body entries (Yukawa only)
        const int64_t j = xj[e];
        const v4 d = xval[e];
        if (sizeof(real) == 4) kadd(cY, eY, d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2]);
        else cY += d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2];
    }
    UL += (double)cL + (double)eL;
    UY += (double)cY + (double)eY;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    const int kind = bd.kind[b];
    if (mode == 0 || mode == 2) {
        // the jump terms from the unknowns themselves, in FP64
        const double phi = kind == PGB_SET_POTENTIAL ? 0.0 : x[o + loc];
        if (kind == PGB_DIELECTRIC) {
            y[o + loc] = 0.5 * phi - UL;
            y[o + N + loc] = 0.5 * phi + UY;
        } else if (kind == PGB_SET_CHARGE) {
            y[o + loc] = UY + 0.5 * phi;
        } else {
            y[o + loc] = UY + (mode == 2 ? 0.5 * bd.bc[b] : 0.0);  // jump of the imposed phi0
        }
    } else {
        if (kind == PGB_DIELECTRIC) y[o + N + loc] = -UY;
        else if (kind == PGB_SET_CHARGE) y[o + loc] = -UY;
        else y[o + loc] = -(UY + 0.5 * bd.bc[b]);
    }
}

// ---------------------------------------------------------------- nested interfaces
// With nested interfaces every row is its body's jump term minus the
// representation sum of the region the row belongs to (the interior row of a
// dielectric body: its interior; the exterior row, or a surface's row: the
// region around it), and each region's sum runs as its own treecode pass.
// Rows start from the jump terms (modes 0 and 2; mode 1: minus the imposed
// jump).
__global__ void k_rows_init(Geo g, BodyDev bd, const double* x, int mode, double* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    const int kind = bd.kind[b];
    if (kind == PGB_DIELECTRIC) {
        const double v = mode == 1 ? 0.0 : 0.5 * x[o + loc];
        y[o + loc] = v;
        y[o + N + loc] = v;
    } else if (kind == PGB_SET_CHARGE) {
        y[o + loc] = mode == 1 ? 0.0 : 0.5 * x[o + loc];
    } else {
        y[o + loc] = mode == 0 ? 0.0 : (mode == 2 ? 0.5 * bd.bc[b] : -0.5 * bd.bc[b]);
    }
}

// Source terms of one region's pass: every body on the region's boundary
// with the densities of its side of the interface and the side's sign folded
// in, so that the pass sums s [V psi - K phi] (the Yukawa slots, at the
// region's screening; kappa = 0 is Laplace); all other bodies are zero.
//   dielectric: phi, psi = fac dphi (fac = 1 inside, eps_in / eps_R outside)
//   imposed potential: psi = u, phi = phi0 (known); imposed charge: phi = u,
//   psi = -sigma0 / eps_R (known).   mode as k_src_prep (x unused for 1).
template <typename real>
__global__ void k_src_region(Geo g, BodyDev bd, RegionDev rd, const double* __restrict__ x, int mode,
                             const typename V4<real>::t* __restrict__ yrel, typename V4<real>::t* __restrict__ src,
                             real* __restrict__ dens) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int sg = rd.sign[b];
    double psi = 0, phi = 0;
    if (sg != 0) {
        const int64_t loc = g.perm[i] - bd.pan_off[b];
        const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
        const int64_t o = bd.unk_off[b];
        const int kind = bd.kind[b];
        if (kind == PGB_DIELECTRIC) {
            if (mode != 1) {
                phi = x[o + loc];
                psi = rd.fac[b] * x[o + N + loc];
            }
        } else if (kind == PGB_SET_POTENTIAL) {
            if (mode != 1) psi = x[o + loc];
            if (mode != 0) phi = bd.bc[b];
        } else {
            if (mode != 1) phi = x[o + loc];
            if (mode != 0) psi = rd.psi_known[b];
        }
        psi *= sg;
        phi *= sg;
    }
    const real rY = (real)psi, rp = (real)phi;
    dens[3 * i] = 0;
    dens[3 * i + 1] = rY;
    dens[3 * i + 2] = rp;
    const real nx = (real)g.n[3 * i], ny = (real)g.n[3 * i + 1], nz = (real)g.n[3 * i + 2];
    for (int m = 0; m < g.K; ++m) {
        const int64_t p = i * g.K + m;
        const real w = (real)g.w[p];
        typename V4<real>::t A = yrel[p], B;
        const real wp = w * rp;
        A.w = 0;
        B.x = wp * nx;
        B.y = wp * ny;
        B.z = wp * nz;
        B.w = w * rY;
        src[2 * p] = A;
        src[2 * p + 1] = B;
    }
}

// One region's sums into its rows: the pass's item partials (Yukawa slots)
// plus the region's near-field corrections, subtracted from the row of the
// target's side (added for mode 1, the right-hand side of imposed terms).
template <typename real>
__global__ void k_assemble_region(Geo g, BodyDev bd, RegionDev rd, Parts u, const real* __restrict__ dens,
                                  const int64_t* __restrict__ coff, const int32_t* __restrict__ cj,
                                  const typename V4<real>::t* __restrict__ cval, const int64_t* __restrict__ xoff,
                                  const int32_t* __restrict__ xj, const typename V4<real>::t* __restrict__ xval,
                                  int mode, double* __restrict__ y) {
    using v4 = typename V4<real>::t;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int sg = rd.sign[b];
    if (sg == 0) return;
    const int gi = u.pan_group[i];
    if (gi < u.g_lo || gi >= u.g_hi) return;
    const int lane = (int)(i - u.gstart[gi]);
    double sY = 0;
    for (int64_t it = u.pitem_off[gi]; it < u.pitem_off[gi + 1]; ++it) sY += u.Up[64 * it + 32 + lane];
    for (int64_t it = u.fitem_off[gi]; it < u.fitem_off[gi + 1]; ++it) sY += u.Uf[64 * it + 32 + lane];
    double U = sY * (1.0 / PGB_FOUR_PI);
    real cY = 0, eY = 0;
    for (int64_t e = coff[i]; e < coff[i + 1]; ++e) {
        const int64_t j = cj[e];
        const v4 d = cval[e];
        if (sizeof(real) == 4) kadd(cY, eY, d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2]);
        else cY += d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2];
    }
    for (int64_t e = xoff[i]; e < xoff[i + 1]; ++e) {
        const int64_t j = xj[e];
        const v4 d = xval[e];
        if (sizeof(real) == 4) kadd(cY, eY, d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2]);
        else cY += d.z * dens[3 * j + 1] - d.w * dens[3 * j + 2];
    }
    U += (double)cY + (double)eY;
    const int64_t loc = g.perm[i] - bd.pan_off[b];
    const int64_t N = bd.pan_off[b + 1] - bd.pan_off[b];
    const int64_t o = bd.unk_off[b];
    const int64_t r = (bd.kind[b] == PGB_DIELECTRIC && sg < 0) ? o + N + loc : o + loc;
    y[r] += mode == 1 ? U : -U;
}

__global__ void k_f32_to_f64(const float* a, double* b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}
__global__ void k_f64_to_f32(const double* a, float* b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
void convert_f32_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
    k_f32_to_f64<<<nblk(n, 256), 256, 0, s>>>(a, b, n);
}
void convert_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    k_f64_to_f32<<<nblk(n, 256), 256, 0, s>>>(a, b, n);
}

void apply_mode(pgb_ctx* c, const double* x, double* y, int precision, int mode, const int* known_mask);

void apply_operator(pgb_ctx* c, const double* x, double* y, int precision, bool known_only, const int* known_mask) {
    apply_mode(c, x, y, precision, known_only ? 1 : 0, known_mask);
}

void apply_full(pgb_ctx* c, const double* x, double* y, int precision) { apply_mode(c, x, y, precision, 2, nullptr); }

// Upward pass as a CUDA graph: captured (on a private stream; nothing runs
// there) the first time a tree / buffer / source-activity combination is
// used, then one cudaGraphLaunch on the context stream per product.
static void upward_graph(pgb_ctx* c, int kind, const UpArgs& up, const EvalArgs& ev, const void* src, void* mom,
                         cudaStream_t on) {  // kind: 0 FP32, 1 FP64, 2 double-single
    auto& gr = c->up_graph[kind];
    bool ok = gr.exec && gr.tree_gen == c->tree_gen && gr.src == src && gr.mom == mom && gr.ncenter == up.ncenter &&
              gr.p2m_grid == up.p2m_grid && gr.far == up.far && gr.far_tab == up.far_tab;
    for (int b = 0; ok && b < PGB_MAX_BODIES; ++b) ok = gr.src_active[b] == up.src_active[b];
    if (!ok) {
        if (gr.exec) {
            PGB_CUDA(cudaGraphExecDestroy(gr.exec));
            gr.exec = nullptr;
        }
        if (!c->cap_stream) PGB_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        PGB_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        std::string why;
        try {
            if (kind == 0)
                treecode_launch_f32(PGB_STAGE_UPWARD, c->p.P, up, c->level_begin, ev, src, nullptr, mom, up.far,
                                    c->cap_stream);
            else if (kind == 1)
                treecode_launch_f64(PGB_STAGE_UPWARD, c->p.P, up, c->level_begin, ev, src, nullptr, mom, up.far,
                                    c->cap_stream);
            else
                treecode_launch_ds(PGB_STAGE_UPWARD, c->p.P, up, ev, src, nullptr, mom, up.far, c->cap_stream);
        } catch (const Error& e) {
            why = e.msg;
        }
        const cudaError_t le = cudaGetLastError();
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
        if (!why.empty() || le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            fail(PGB_ECUDA, "upward-pass graph capture: " + (why.empty() ? std::string(cudaGetErrorString(
                                                                               le != cudaSuccess ? le : ce))
                                                                          : why));
        }
        const cudaError_t ie = cudaGraphInstantiate(&gr.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) gr.exec = nullptr;
        PGB_CUDA(ie);
        gr.tree_gen = c->tree_gen;
        gr.src = src;
        gr.mom = mom;
        gr.far = up.far;
        gr.far_tab = up.far_tab;
        gr.ncenter = up.ncenter;
        gr.p2m_grid = up.p2m_grid;
        for (int b = 0; b < PGB_MAX_BODIES; ++b) gr.src_active[b] = up.src_active[b];
    }
    PGB_CUDA(cudaGraphLaunch(gr.exec, on));
}

// The upward-pass stream of a precision (created on first use).
static cudaStream_t upward_stream(pgb_ctx* c, int pi) {
    if (!c->up_stream[pi]) {
        int least = 0, greatest = 0;
        PGB_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        PGB_CUDA(cudaStreamCreateWithPriority(&c->up_stream[pi], cudaStreamNonBlocking, greatest));
        PGB_CUDA(cudaEventCreateWithFlags(&c->up_fork[pi], cudaEventDisableTiming));
        PGB_CUDA(cudaEventCreateWithFlags(&c->up_join[pi], cudaEventDisableTiming));
    }
    return c->up_stream[pi];
}

// Sizes every buffer a product of this precision writes (so that a product
// on another stream allocates nothing).
void reserve_product(pgb_ctx* c, int precision) {
    const int pi = precision == PGB_FP32 ? 0 : 1;
    const int T = n_terms(c->p.P);
    const int64_t nsrc = c->n_pan * c->p.K;
    c->d_dens[pi].resize(3 * c->n_pan);
    c->d_Up[pi].resize(64 * std::max<int64_t>(c->n_pitems, 1));
    c->d_Uf[pi].resize(64 * std::max<int64_t>(c->n_fitems, 1));
    c->d_work.resize(2);
    const int TP = n_terms_pad(c->p.P);
    if (pi == 0) {
        c->d_src32.resize(2 * nsrc);
        c->d_mom32.resize((size_t)c->n_nodes * 2 * T);
        c->d_far32.resize((size_t)c->n_nodes * 2 * TP);
    } else {
        c->d_src64.resize(2 * nsrc);
        c->d_src_ds.resize(2 * nsrc);
        c->d_mom64.resize((size_t)c->n_nodes * 2 * T);
        c->d_far64.resize((size_t)c->n_nodes * 2 * TP);
        c->d_mom_ds.resize((size_t)c->n_nodes * 2 * T);
        c->d_far_ds.resize((size_t)c->n_nodes * 2 * TP);
    }
    (void)far_table(c, c->kappa);
    for (const auto& reg : c->regions) (void)far_table(c, reg->dev.kappa);
    if (c->arrive_gen[pi] != c->tree_gen || c->d_arrive[pi].n < (size_t)c->n_nodes) {
        c->d_arrive[pi].resize(std::max<int64_t>(c->n_nodes, 1));
        PGB_CUDA(cudaMemsetAsync(c->d_arrive[pi].p, 0, sizeof(int) * c->d_arrive[pi].n, c->stream));
        c->arrive_gen[pi] = c->tree_gen;
    }
}

void apply_mode(pgb_ctx* c, const double* x, double* y, int precision, int mode, const int* known_mask) {
    const bool known_only = mode == 1;
    if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run for the current bodies and poses");
    cudaStream_t s = c->stream;
    Geo g = geo(c);
    BodyDev bd = body_dev(c);
    if (known_only && known_mask)  // imposed terms of the selected surfaces only
        for (int b = 0; b < bd.n_bodies; ++b)
            if (!known_mask[b]) bd.bc[b] = 0.0;
    const int P = c->p.P;
    const int T = n_terms(P);
    const int64_t nsrc = g.n_src;
    // per-precision work buffers: an FP64 product may run on a side stream
    // while FP32 products go on
    const int pi = precision == PGB_FP32 ? 0 : 1;
    auto& dens = c->d_dens[pi];
    auto& Up = c->d_Up[pi];
    auto& Uf = c->d_Uf[pi];
    dens.resize(3 * c->n_pan);
    Up.resize(64 * std::max<int64_t>(c->n_pitems, 1));
    Uf.resize(64 * std::max<int64_t>(c->n_fitems, 1));
    UpArgs up;
    up.n_leaves = c->n_leaves;
    up.leaf_node = c->d_leaf_node; up.nstart = c->d_node_start; up.nend = c->d_node_end;
    up.child = c->d_node_child; up.nchild = c->d_node_nchild;
    up.ncenter = c->d_node_center; up.K = c->p.K; up.nbody = c->d_node_body;
    up.lvl_begin = up.lvl_end = 0;
    up.p2m_grid = 0;
    up.n_nodes = c->n_nodes;
    up.parent = c->d_node_parent;
    {
        const int pi_up = precision == PGB_FP32 ? 0 : 1;
        auto& cnt = c->d_arrive[pi_up];
        if (c->arrive_gen[pi_up] != c->tree_gen || cnt.n < (size_t)c->n_nodes) {
            cnt.resize(std::max<int64_t>(c->n_nodes, 1));
            PGB_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * cnt.n, s));
            c->arrive_gen[pi_up] = c->tree_gen;
        }
        up.arrive = cnt.p;
    }
    if (precision != PGB_FP32 && c->persist_blocks > 0)  // side product: P2M on two blocks per SM
        up.p2m_grid = 2 * c->persist_blocks;
    EvalArgs ev;
    ev.n_groups = c->n_groups;
    ev.gstart = c->d_group_start; ev.gend = c->d_group_end; ev.gbody = c->d_group_body;
    ev.gcenter = c->d_group_center; ev.near_off = c->d_near_off; ev.far_off = c->d_far_off;
    ev.near_l = c->d_near; ev.far_l = c->d_far; ev.nstart = c->d_node_start; ev.nend = c->d_node_end;
    ev.nbody = c->d_node_body; ev.ncenter = c->d_node_center; ev.K = c->p.K; ev.kappa = c->kappa;
    for (int b = 0; b < PGB_MAX_BODIES; ++b) ev.lap_body[b] = ev.src_active[b] = up.src_active[b] = 0;
    for (size_t b = 0; b < c->bodies.size(); ++b) {
        ev.lap_body[b] = c->bodies[b].kind == PGB_DIELECTRIC;
        // imposed-boundary terms: molecules carry no known density
        ev.src_active[b] = up.src_active[b] =
            !c->body_off[b] && (known_only ? (known_mask ? known_mask[b] : (c->bodies[b].kind != PGB_DIELECTRIC)) : 1);
    }
    ev.all_active = 1;
    for (size_t b = 0; b < c->bodies.size(); ++b) ev.all_active &= ev.src_active[b];
    // a replayed lockstep iteration: which problems take part is known on the device only
    ev.bmask = up.bmask = c->dev_bmask;
    if (c->dev_bmask) ev.all_active = 0;
    // rows of bodies left out of the product (a lockstep batch's finished
    // problems) are not computed
    ev.tgt_mask = ~0ull;
    for (size_t b = 0; b < c->bodies.size(); ++b)
        if (c->body_off[b]) ev.tgt_mask &= ~(1ull << b);
    ev.g_lo = c->shard_g[0] >= 0 ? c->shard_g[0] : 0;
    ev.g_hi = c->shard_g[0] >= 0 ? c->shard_g[1] : c->n_groups;
    ev.near4 = c->d_near4;
    ev.far4 = c->d_far4;
    ev.tile_off = c->d_tile_off;
    ev.tile_d = c->d_tile_d;
    ev.tile_m = c->d_tile_m;
    ev.n_pitems = c->n_pitems;
    ev.n_fitems = c->n_fitems;
    ev.pitem_off = c->d_pitem_off;
    ev.fitem_off = c->d_fitem_off;
    ev.pitem_group = c->d_pitem_group;
    ev.fitem_group = c->d_fitem_group;
    ev.p2p_item = c->p.p2p_item;
    ev.m2p_item = c->p.m2p_item;
    ev.Up = Up;
    ev.Uf = Uf;
    ev.p2p_work = ev.m2p_work = nullptr;
    ev.persist_blocks = 0;
    if (c->persist_blocks > 0) {  // side-stream product: a few resident blocks per SM take items
        c->d_work.resize(2);
        PGB_CUDA(cudaMemsetAsync(c->d_work.p, 0, 16, s));
        ev.p2p_work = c->d_work.p;
        ev.m2p_work = c->d_work.p + 1;
        ev.persist_blocks = c->persist_blocks;
    }
    const bool f32 = precision == PGB_FP32;
    const int TP = n_terms_pad(P);
    if (f32) {
        c->d_src32.resize(2 * nsrc);
        c->d_mom32.resize((size_t)c->n_nodes * 2 * T);
        c->d_far32.resize((size_t)c->n_nodes * 2 * TP);
        up.far = c->d_far32.p;
    } else {
        c->d_src64.resize(2 * nsrc);
        c->d_mom64.resize((size_t)c->n_nodes * 2 * T);
        c->d_far64.resize((size_t)c->n_nodes * 2 * TP);
        up.far = c->d_far64.p;
        if (precision == PGB_FP64_DS) {
            c->d_src_ds.resize(2 * nsrc);
            c->d_mom_ds.resize((size_t)c->n_nodes * 2 * T);
            c->d_far_ds.resize((size_t)c->n_nodes * 2 * TP);
            up.far = c->d_far_ds.p;
        }
    }
    const bool dsp = precision == PGB_FP64_DS;
    auto tab_for = [&](double kappa) -> const void* {
        const FarTab& t = far_table(c, kappa);
        if (f32) return P > 8 ? (const void*)t.t32p.p : (const void*)t.t32.p;
        return dsp ? (const void*)t.tds.p : (const void*)t.t64.p;
    };
    up.far_tab = tab_for(c->kappa);
    if (nested(c)) {
        // one treecode pass per region: rows from the jump terms, then each
        // region's sum subtracted from the rows on its boundary
        if (known_mask) fail(PGB_EINVAL, "imposed-term selection is not available with nested interfaces");
        k_rows_init<<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, x, mode, y);
        PGB_LAUNCHED(c, 1);
        for (int b = 0; b < PGB_MAX_BODIES; ++b) ev.lap_body[b] = 0;
        for (const auto& reg : c->regions) {
            const RegionDev& rd = reg->dev;
            ev.kappa = rd.kappa;
            up.far_tab = tab_for(rd.kappa);
            if (ev.p2p_work)  // persistent launches take items from counters: fresh ones per pass
                PGB_CUDA(cudaMemsetAsync(c->d_work.p, 0, 16, s));
            ev.all_active = 1;
            ev.tgt_mask = 0;
            for (size_t b = 0; b < c->bodies.size(); ++b) {
                ev.src_active[b] = up.src_active[b] = rd.sign[b] != 0 && !c->body_off[b];
                ev.all_active &= ev.src_active[b];
                if (ev.src_active[b]) ev.tgt_mask |= 1ull << b;  // only the region's own rows
            }
            {
                StageTimer tm(c, PGB_STAGE_SOURCES + (f32 ? 0 : PGB_STAGE_FP64));
                if (f32)
                    k_src_region<float><<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, rd, x, mode, c->d_y32, c->d_src32,
                                                                             (float*)dens.p);
                else
                    k_src_region<double><<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, rd, x, mode, c->d_y64,
                                                                              c->d_src64, dens.p);
                if (precision == PGB_FP64_DS) convert_src_ds(c->d_src64, c->d_src_ds, 2 * nsrc, s);
                PGB_CUDA(cudaGetLastError());
                PGB_LAUNCHED(c, precision == PGB_FP64_DS ? 2 : 1);
            }
            for (int stage : {PGB_STAGE_UPWARD, PGB_STAGE_P2P, PGB_STAGE_M2P}) {
                StageTimer tm(c, stage + (f32 ? 0 : PGB_STAGE_FP64));
                if (f32)
                    treecode_launch_f32(stage, P, up, c->level_begin, ev, c->d_src32, c->d_x32, c->d_mom32,
                                        c->d_far32, s);
                else if (dsp)
                    treecode_launch_ds(stage, P, up, ev, c->d_src_ds, c->d_x64, c->d_mom_ds, c->d_far_ds, s);
                else
                    treecode_launch_f64(stage, P, up, c->level_begin, ev, c->d_src64, c->d_x64, c->d_mom64,
                                        c->d_far64, s);
                PGB_CUDA(cudaGetLastError());
                PGB_LAUNCHED(c, 1);
            }
            {
                StageTimer tm(c, PGB_STAGE_ASSEMBLE + (f32 ? 0 : PGB_STAGE_FP64));
                Parts u{c->d_pan_group, c->d_group_start, c->d_pitem_off, c->d_fitem_off, Up, Uf, ev.g_lo, ev.g_hi};
                if (f32)
                    k_assemble_region<float><<<nblk(c->n_pan, 128), 128, 0, s>>>(
                        g, bd, rd, u, (const float*)dens.p, reg->corr_off, reg->corr_j, reg->corr_val32,
                        reg->xcorr_off, reg->xcorr_j, reg->xcorr_val32, mode, y);
                else
                    k_assemble_region<double><<<nblk(c->n_pan, 128), 128, 0, s>>>(
                        g, bd, rd, u, dens.p, reg->corr_off, reg->corr_j, reg->corr_val, reg->xcorr_off, reg->xcorr_j,
                        reg->xcorr_val, mode, y);
                PGB_CUDA(cudaGetLastError());
                PGB_LAUNCHED(c, 1);
            }
        }
        return;
    }
    {
        StageTimer tm(c, PGB_STAGE_SOURCES + (f32 ? 0 : PGB_STAGE_FP64));
        if (f32)
            k_src_prep<float><<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, x, mode, c->d_y32, c->d_src32,
                                                                  (float*)dens.p, c->eps_out);
        else
            k_src_prep<double><<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, x, mode, c->d_y64, c->d_src64,
                                                                   dens.p, c->eps_out);
        if (precision == PGB_FP64_DS) convert_src_ds(c->d_src64, c->d_src_ds, 2 * nsrc, s);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, precision == PGB_FP64_DS ? 2 : 1);
    }
    // the upward pass on its own stream, beside P2P (which does not read the
    // moments); M2P waits for it
    cudaStream_t us = upward_stream(c, pi);
    PGB_CUDA(cudaEventRecord(c->up_fork[pi], s));
    PGB_CUDA(cudaStreamWaitEvent(us, c->up_fork[pi], 0));
    {
        StageTimer tm(c, PGB_STAGE_UPWARD + (f32 ? 0 : PGB_STAGE_FP64), us);
        const void* usrc = f32 ? (const void*)c->d_src32.p : dsp ? (const void*)c->d_src_ds.p : (const void*)c->d_src64.p;
        void* umom = f32 ? (void*)c->d_mom32.p : dsp ? (void*)c->d_mom_ds.p : (void*)c->d_mom64.p;
        if (c->p.graphs && !c->capturing) {
            upward_graph(c, f32 ? 0 : dsp ? 2 : 1, up, ev, usrc, umom, us);
            c->graph_kernels += 2;
            ++c->graph_launches;
        }
        else if (f32)
            treecode_launch_f32(PGB_STAGE_UPWARD, P, up, c->level_begin, ev, c->d_src32, c->d_x32, c->d_mom32,
                                c->d_far32, us);
        else if (dsp)
            treecode_launch_ds(PGB_STAGE_UPWARD, P, up, ev, c->d_src_ds, c->d_x64, c->d_mom_ds, c->d_far_ds, us);
        else
            treecode_launch_f64(PGB_STAGE_UPWARD, P, up, c->level_begin, ev, c->d_src64, c->d_x64, c->d_mom64,
                                c->d_far64, us);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 2);
    }
    PGB_CUDA(cudaEventRecord(c->up_join[pi], us));
    for (int stage : {PGB_STAGE_P2P, PGB_STAGE_M2P}) {
        if (stage == PGB_STAGE_M2P) PGB_CUDA(cudaStreamWaitEvent(s, c->up_join[pi], 0));
        StageTimer tm(c, stage + (f32 ? 0 : PGB_STAGE_FP64));
        if (f32)
            treecode_launch_f32(stage, P, up, c->level_begin, ev, c->d_src32, c->d_x32, c->d_mom32, c->d_far32, s);
        else if (dsp)
            treecode_launch_ds(stage, P, up, ev, c->d_src_ds, c->d_x64, c->d_mom_ds, c->d_far_ds, s);
        else
            treecode_launch_f64(stage, P, up, c->level_begin, ev, c->d_src64, c->d_x64, c->d_mom64, c->d_far64, s);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
    }
    {
        StageTimer tm(c, PGB_STAGE_ASSEMBLE + (f32 ? 0 : PGB_STAGE_FP64));
        Parts u{c->d_pan_group, c->d_group_start, c->d_pitem_off, c->d_fitem_off, Up, Uf, ev.g_lo, ev.g_hi};
        if (f32)
            k_assemble<float><<<nblk(c->n_pan, 128), 128, 0, s>>>(
                g, bd, u, (const float*)dens.p, c->d_corr_off, c->d_corr_j, c->d_corr_val32, c->d_xcorr_off,
                c->d_xcorr_j, c->d_xcorr_val32, mode, x, y);
        else
            k_assemble<double><<<nblk(c->n_pan, 128), 128, 0, s>>>(g, bd, u, dens.p, c->d_corr_off, c->d_corr_j,
                                                                   c->d_corr_val, c->d_xcorr_off, c->d_xcorr_j,
                                                                   c->d_xcorr_val, mode, x, y);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
    }
}

}  // namespace pgb
