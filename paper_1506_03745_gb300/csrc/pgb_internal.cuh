// Internal declarations shared by the translation units of libpgb.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/pgb.h"

#define PGB_MAX_P 15
// Taylor orders with compiled kernels: 0..8, 10, 12 and 15 (the adjoint: 0..8)
inline bool p_supported(int P) { return (P >= 0 && P <= 8) || P == 10 || P == 12 || P == 15; }
#define PGB_MAX_BODIES 64
#define PGB_LIST_STACK 96

namespace pgb {

struct __align__(32) dbl4 {
    double x, y, z, w;
};

// Status carried through host code as an exception inside the library only;
// the C entry points turn it into a return code.
struct Error {
    int code;
    std::string msg;
};

void cuda_check(cudaError_t e, const char* what);
#define PGB_CUDA(call) ::pgb::cuda_check((call), #call)
void fail(int code, const std::string& msg);

// Allocation stream of the calling thread (set by AllocScope for the
// duration of a library call on a context).
extern thread_local cudaStream_t g_alloc_stream;
extern thread_local bool g_alloc_scoped;
// Allocations the library has made in this process (device buffers and
// pinned host buffers), reported by pgb_alloc_count.
void note_alloc();
struct AllocScope {
    cudaStream_t prev_stream;
    bool prev_scoped;
    explicit AllocScope(cudaStream_t s) : prev_stream(g_alloc_stream), prev_scoped(g_alloc_scoped) {
        g_alloc_stream = s;
        g_alloc_scoped = true;
    }
    ~AllocScope() {
        g_alloc_stream = prev_stream;
        g_alloc_scoped = prev_scoped;
    }
};

template <typename T>
struct DBuf {  // owning device buffer
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;  // stream of a stream-ordered allocation
    bool async = false;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) {
            if (async) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
        async = false;
    }
    // Inside a library call (AllocScope active) the buffer is allocated and
    // freed in stream order on the context's stream, so temporaries cost no
    // device-wide synchronisation; elsewhere plain cudaMalloc / cudaFree.
    void resize(size_t count) {  // contents undefined after growth
        if (count <= n && p) return;
        release();
        size_t c = count ? count : 1;
        cudaError_t e;
        if (g_alloc_scoped) {
            e = cudaMallocAsync((void**)&p, c * sizeof(T), g_alloc_stream);
            async = e == cudaSuccess;
            st = g_alloc_stream;
        } else {
            e = cudaMalloc(&p, c * sizeof(T));
        }
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            fail(PGB_ENOMEM, "cudaMalloc of " + std::to_string(c * sizeof(T)) + " bytes failed");
        }
        note_alloc();
        n = c;
    }
    operator T*() const { return p; }
};

// Taylor term count of total degree <= P in three variables.
__host__ __device__ constexpr int n_terms(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// Far-field coefficient tables (farfield.cu) of one Taylor order and
// screening: moments -> the coefficients the M2P kernels evaluate.
struct FarTab {
    int P = -1;
    double kappa = 0.0;
    DBuf<double> t64;
    DBuf<float> t32;
    DBuf<double> tds;  // the FP64 table split into double-single pairs (8 bytes each)
    DBuf<float> t32p;  // the packed layout of t64 rounded to FP32 (orders above 8)
};
// padded coefficient count per kernel: rows of 16 bytes for vector loads
__host__ __device__ constexpr int n_terms_pad(int P) { return (n_terms(P) + 3) & ~3; }
void far_tables(int P, double kappa, std::vector<double>& tab);

struct Body {
    int kind = PGB_DIELECTRIC;
    double eps_in = 1.0;
    double bc = 0.0;  // internal units: sigma0 in e/A^2, phi0 in e/(eps0 A)
    int64_t N = 0, nv = 0, nq = 0;
    std::vector<double> verts;  // body frame
    std::vector<int32_t> tris;
    std::vector<double> qxyz, qval;
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double t[3] = {0, 0, 0};
    bool identity_pose = true;
    // offsets into global arrays
    int64_t pan_off = 0, unk_off = 0, q_off = 0, v_off = 0;
    // tree frame
    double lo[3] = {0, 0, 0}, ext = 1.0;
    int32_t root = 0;
    // independent problem the body belongs to: bodies of different problems
    // do not interact (a batch of poses solved as one block-diagonal system)
    int prob = 0;
    // nesting: the body lies in the interior region of body `parent` (-1: in
    // the solvent); kappa_in screens its own interior (dielectric bodies)
    int parent = -1;
    double kappa_in = 0.0;
};

// Device-side view of the problem passed by value to kernels.
struct Geo {
    int64_t n_pan, n_src;
    int K;
    // per sorted panel
    const int32_t* perm;       // sorted -> global original panel index
    const int32_t* pbody;      // body id
    const double* v;           // 9 per panel, world
    const double* c;           // 3 per panel (world centroid)
    const double* n;           // 3 per panel (unit normal)
    const double* A;           // area
    const int32_t* pleaf;      // leaf index of the panel
    // per source point
    const double* y;           // 3 per point
    const double* w;           // weight * area
};

struct BodyDev {  // per-body constants for kernels
    int kind[PGB_MAX_BODIES];
    double eps_ratio[PGB_MAX_BODIES];  // eps_in / eps_out (dielectric)
    double bc[PGB_MAX_BODIES];
    int64_t pan_off[PGB_MAX_BODIES + 1];
    int64_t unk_off[PGB_MAX_BODIES];
    int parent[PGB_MAX_BODIES];        // enclosing body, -1: the solvent
    int n_bodies;
};

// One region of a nested system for a treecode pass: the bodies bounding it
// (sign +1: the region is the body's interior, -1: its exterior, 0: not on
// the boundary), the factor of each body's dphi on the region's side
// (eps_in(b) / eps_R from outside, 1 from inside), the imposed normal
// derivative -sigma0 / eps_R of charged surfaces, and its screening.
struct RegionDev {
    int sign[PGB_MAX_BODIES];
    double fac[PGB_MAX_BODIES];
    double psi_known[PGB_MAX_BODIES];
    double kappa;
};

}  // namespace pgb

#define PGB_CORR_CAP 48  // near-field candidates kept per target by the counting pass

struct pgb_ctx {
    pgb_params p;
    cudaStream_t stream = nullptr;
    std::string err;
    double eps_out = 80.0, kappa = 0.0;
    std::vector<pgb::Body> bodies;
    bool tree_valid = false;
    bool order_valid = false;  // Morton order / octree structure (body frame)
    bool lists_valid = false;  // interaction lists of the current order (pgb_tree_refresh keeps them)
    int64_t n_pan = 0, n_unk = 0, n_q = 0, n_verts = 0;

    // inputs on the device
    pgb::DBuf<double> d_vb;      // body-frame vertices, all bodies
    pgb::DBuf<int32_t> d_tris;   // global vertex ids, original panel order
    pgb::DBuf<int32_t> d_pan_body;
    pgb::DBuf<double> d_qxyz_body, d_qval, d_qxyz;  // charges (body frame / world)
    pgb::DBuf<int32_t> d_q_body;
    pgb::DBuf<double> d_pose;    // 12 per body (R row-major, t)

    // ordering and tree structure (body frame; rebuilt when meshes change)
    pgb::DBuf<int32_t> d_perm, d_inv;    // sorted -> original global, and inverse
    pgb::DBuf<uint32_t> d_key;           // sorted keys
    pgb::DBuf<int32_t> d_qcell;          // 3 per sorted panel
    int64_t n_nodes = 0, n_leaves = 0;
    pgb::DBuf<int32_t> d_node_start, d_node_end, d_node_level, d_node_child, d_node_nchild, d_node_body;
    pgb::DBuf<int32_t> d_node_leaf0, d_node_leaf1, d_leaf_node, d_node_parent;
    pgb::DBuf<unsigned int> d_up_counter;
    std::vector<int32_t> h_node_level;   // for per-level passes
    std::vector<int64_t> level_begin;    // node id ranges by level
    pgb::DBuf<int32_t> d_pan_leaf;

    // world geometry (per pose)
    pgb::DBuf<double> d_v, d_c, d_n, d_A, d_y, d_w;
    pgb::DBuf<int32_t> d_pbody;          // body of sorted panel
    pgb::DBuf<double> d_node_center, d_node_r2, d_node_clo, d_node_chi, d_node_a8;
    pgb::DBuf<float4> d_y32;             // point - leaf centre, weight
    pgb::DBuf<pgb::dbl4> d_y64;
    // target groups
    int64_t n_groups = 0;
    pgb::DBuf<int32_t> d_group_start, d_group_end, d_group_body;
    pgb::DBuf<double> d_group_lo, d_group_hi, d_group_center;
    pgb::DBuf<float4> d_x32;             // centroid - group centre
    pgb::DBuf<pgb::dbl4> d_x64;
    // lists
    int64_t n_near = 0, n_far = 0;
    pgb::DBuf<int64_t> d_near_off, d_far_off;
    pgb::DBuf<int32_t> d_near, d_far;
    pgb::DBuf<float4> d_near4, d_far4;   // FP32 entry offsets (node centre - group centre), node id
    pgb::DBuf<int32_t> d_list_tmp;       // entries kept by the counting traversal (fixed rows per group)
    int64_t n_tiles = 0;                 // P2P tiles (<= 32 points of one near leaf) over all groups
    pgb::DBuf<int64_t> d_tile_off;
    pgb::DBuf<float4> d_tile_d;
    pgb::DBuf<int4> d_tile_m;
    // work items: a group's P2P tiles and its far entries in runs of at most
    // p.p2p_item / p.m2p_item, one block each, so that no block carries a
    // whole heavy group; each item leaves 32 (L) + 32 (Y) partial sums
    int64_t n_pitems = 0, n_fitems = 0;
    pgb::DBuf<int64_t> d_pitem_off, d_fitem_off;  // per group (+ total)
    pgb::DBuf<int32_t> d_pitem_group, d_fitem_group;
    pgb::DBuf<int32_t> d_pan_group;                // sorted panel -> its group
    // near-field corrections (CSR over sorted targets)
    // intra-body entries depend only on each body's own geometry and kappa, so
    // they survive pose changes; cross-body entries are rebuilt per pose
    bool intra_valid = false;
    int64_t n_corr = 0, n_xcorr = 0;
    pgb::DBuf<int64_t> d_corr_off, d_xcorr_off;
    pgb::DBuf<int32_t> d_corr_j, d_xcorr_j;
    pgb::DBuf<pgb::dbl4> d_corr_val, d_xcorr_val;  // dVL, dKL, dVY, dKY
    pgb::DBuf<float4> d_corr_val32, d_xcorr_val32;  // their FP32 copies (the FP32 product)
    pgb::DBuf<double> d_yfine;             // 19-point nodes per panel (3 each), for the corrections
    pgb::DBuf<double> d_yfine_ds, d_y_ds;  // the 19- and K-point nodes as double-single pairs (8 bytes each)
    pgb::DBuf<float4> d_corr_pf4, d_corr_nlo4, d_corr_nhi4;  // FP32 prefilter of the near-field search
    pgb::DBuf<int32_t> d_corr_tmp;         // candidates kept by the counting pass (PGB_CORR_CAP per panel)
    pgb::DBuf<double> d_xbatch;            // solution buffer of pgb_solve_batch
    // adjoint (transposed treecode): built on first use after each tree build
    bool adj_valid = false;
    std::vector<int64_t> group_begin;      // first group of each body (+ total)
    pgb::DBuf<float4> d_yT32, d_n32, d_cT32;
    pgb::DBuf<pgb::dbl4> d_yT64, d_n64, d_cT64;
    pgb::DBuf<double> d_rT2, d_gTlo, d_gThi;
    int64_t n_Tnear = 0, n_Tfar = 0;
    pgb::DBuf<int64_t> d_Tnear_off, d_Tfar_off, d_ct_off;
    pgb::DBuf<int32_t> d_Tnear, d_Tfar, d_ct_i;
    pgb::DBuf<float4> d_Tnear4, d_Tfar4;
    pgb::DBuf<pgb::dbl4> d_ct_val;
    pgb::DBuf<int32_t> d_near_group;     // group of each forward near entry
    pgb::DBuf<int64_t> d_tn_off, d_tn_e;   // forward near entries by source leaf (CSR over nodes)
    pgb::DBuf<float4> d_srcT32;
    pgb::DBuf<pgb::dbl4> d_srcT64;
    pgb::DBuf<float> d_momT32;
    pgb::DBuf<double> d_momT64, d_Tout, d_sT, d_lam, d_gx, d_bu;

    // matvec work buffers
    pgb::DBuf<float4> d_src32;           // 2 per point
    pgb::DBuf<pgb::dbl4> d_src64;
    pgb::DBuf<pgb::dbl4> d_src_ds;       // the same split into double-single (32 bytes each)
    pgb::DBuf<double> d_dens[2];            // 3 per sorted panel: psiL, psiY, phi
    pgb::DBuf<float> d_mom32;            // 2*T per node
    pgb::DBuf<double> d_mom64;
    pgb::DBuf<int> d_arrive[2];          // upward pass: children finished per node, per precision
    uint64_t arrive_gen[2] = {~0ull, ~0ull};  // tree_gen the counters were zeroed for
    pgb::DBuf<float> d_far32;            // far-field coefficients: 2 * n_terms_pad(P) per node
    pgb::DBuf<double> d_far64;
    pgb::DBuf<double> d_mom_ds, d_far_ds;  // moments and coefficients of the double-single product (8 bytes each)
    std::vector<std::unique_ptr<pgb::FarTab>> far_tabs;  // per (P, kappa)
    pgb::DBuf<double> d_phi_part;        // chunk partial sums of phi_reac (few charges)
    pgb::DBuf<pgb::dbl4> d_qw;           // charge weights per sorted panel (energies): own charges
                                         // (wV, wK), then the enclosing body's (wV, wK)
    uint64_t qw_key[4] = {~0ull, ~0ull, 0, 0};  // tree_gen, config_gen, K, K_near they were made for
    pgb::DBuf<double> d_Up[2], d_Uf[2];        // P2P / M2P partial sums: 64 per work item (32 L, then 32 Y)
    pgb::DBuf<double> d_xtmp, d_ytmp;    // FP64 staging for FP32 matvec API
    // scratch
    pgb::DBuf<int64_t> d_scan_tmp;
    pgb::DBuf<unsigned char> d_scratch;

    // solver
    pgb::DBuf<double> d_V, d_H, d_red, d_gv, d_b, d_bc, d_r, d_wk, d_xs, d_small;
    pgb::DBuf<pgb::dbl4> d_pc;           // block-diagonal preconditioner, per sorted panel
    pgb::DBuf<double> d_pz;              // its work vector
    bool pc_ready = false;
    int arn_blocks = 0;                  // grid of the Arnoldi-step kernels (0: not yet set)
    int persist_blocks = 0;              // > 0: products launch P2P/M2P persistently with this grid
    pgb::DBuf<unsigned long long> d_work;  // their item counters
    cudaStream_t side_stream = nullptr;  // FP64 residual overlapped with FP32 iterations (lowest priority)
    cudaStream_t hp_stream = nullptr;    // the refinement's FP32 iterations (highest priority)
    pgb::DBuf<double> d_xspec, d_r64;    // its iterate (and x - x*), its product
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double* h_pinned = nullptr;

    // upward pass captured as a CUDA graph per precision, replayed on the
    // context stream; recaptured when the tree or a buffer it uses changes
    struct UpGraph {
        cudaGraphExec_t exec = nullptr;
        uint64_t tree_gen = 0;
        const void* src = nullptr;
        void* mom = nullptr;
        void* far = nullptr;
        const void* far_tab = nullptr;
        const double* ncenter = nullptr;
        int p2m_grid = 0;
        int src_active[PGB_MAX_BODIES] = {0};
    } up_graph[3];  // FP32, FP64, double-single
    cudaStream_t cap_stream = nullptr;   // capture only (nothing runs on it)
    // GMRES iterations replayed from a graph with a device-side loop
    // (pgb_params.graphs = 2): one graph per operator setup, rebuilt when a
    // pointer or size it holds changes
    struct GmGraph {
        cudaGraphExec_t exec = nullptr;
        uint64_t tree_gen = 0;
        int prec = -1, m = 0, pc = -1;
        const void *V = nullptr, *w = nullptr, *H = nullptr, *g = nullptr;
        int64_t n = 0;
        int P = -1;
        double theta = -1;
        int64_t body_launches = 0;
    } gm_graph;
    cudaStream_t gm_stream = nullptr;    // stream of its capture
    bool capturing = false;              // products enqueue plain launches (no nested graph launch)
    // a lockstep batch's replayed iterations (batch.cu), captured per solve call
    cudaGraphExec_t seg_exec = nullptr;
    int64_t seg_body_launches = 0;
    // device body mask the products of a capture read (nullptr: none)
    const unsigned long long* dev_bmask = nullptr;
    // sharded products: the target groups [shard_g[0], shard_g[1]) of this
    // rank (shard_g[0] < 0: every group)
    int64_t shard_g[2] = {-1, -1};
    pgb::DBuf<double> d_shard_tmp, d_shard_part, d_shard_V, d_shard_w, d_shard_h;  // sharded solve (shard.cu)
    pgb::DBuf<double> d_shard_b, d_shard_bc, d_shard_x, d_shard_r, d_shard_d;
    pgb::DBuf<int> d_gmi;                // device column index of the replayed iterations
    pgb::DBuf<double> d_gmd;             // tolerance, column limit, last estimate
    pgb::DBuf<double> d_xsel;            // the column the replayed product reads
    // the upward pass of a product runs on its own (highest-priority) stream
    // beside the P2P kernel, which does not need the moments; per precision
    cudaStream_t up_stream[2] = {nullptr, nullptr};
    cudaEvent_t up_fork[2] = {nullptr, nullptr}, up_join[2] = {nullptr, nullptr};
    uint64_t tree_gen = 0;               // bumped whenever the octree structure is rebuilt
    uint64_t config_gen = 0;             // bumped when bodies, charges, boundary values or solvent change
    bool owns_stream = false;            // lane contexts create (and destroy) their stream
    std::vector<pgb_ctx*> lane_ctx;      // pose lanes of pgb_solve_batch
    uint64_t lane_gen = ~0ull;           // config_gen the lanes were copied at
    // block-diagonal pose batches: this context as the union of n_prob
    // independent problems (bodies prob_first[p] .. prob_first[p + 1]; rows
    // d_poff[p] .. d_poff[p + 1]), and, on the caller's context, the union
    // it keeps with the sources it was copied from
    int n_prob = 1;
    std::vector<int> prob_first;
    pgb::DBuf<int64_t> d_poff;
    int seg_nbp = 0;                     // blocks per problem of the segmented kernels
    pgb::DBuf<double> d_seg, d_seg_red;  // per-problem Krylov vectors; segmented partial sums
    pgb::DBuf<int> d_segi;               // per-problem activity and column counts
    pgb::DBuf<unsigned long long> d_segm;  // run-time body mask, then each problem's bodies
    // bodies left out of the products (1: its sources and rows are not
    // computed; the problems that no longer iterate in a lockstep solve)
    char body_off[PGB_MAX_BODIES] = {0};
    // nested interfaces (pgb_set_region): regions and their near-field
    // corrections, one treecode pass per region in every product
    struct Region {
        pgb::RegionDev dev;
        int64_t n_corr = 0, n_xcorr = 0;
        pgb::DBuf<int64_t> corr_off, xcorr_off;
        pgb::DBuf<int32_t> corr_j, xcorr_j;
        pgb::DBuf<pgb::dbl4> corr_val, xcorr_val;
        pgb::DBuf<float4> corr_val32, xcorr_val32;
    };
    std::vector<std::unique_ptr<Region>> regions;
    pgb_ctx* union_ctx = nullptr;
    std::vector<pgb_ctx*> union_src;
    std::vector<uint64_t> union_gen;

    // statistics and stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    double stage_ms[PGB_N_STAGES] = {0};
    int64_t stage_calls[PGB_N_STAGES] = {0};
    int64_t launches = 0;
    // of those, kernels run inside replayed graphs, and the graph launches
    int64_t graph_kernels = 0, graph_launches = 0;
    pgb_tree_info info{};
    int64_t p2p_pairs = 0, p2p_lap = 0, m2p_pairs = 0, m2p_lap = 0;
};

namespace pgb {
// Whether the context holds nested interfaces (a body inside another, or a
// screened interior): products then run one treecode pass per region.
inline bool nested(const pgb_ctx* c) {
    for (const auto& b : c->bodies)
        if (b.parent >= 0 || b.kappa_in != 0.0) return true;
    return false;
}
// CUDA-event interval on the context stream around one stage (no-op when
// timing is off).
struct StageTimer {
    pgb_ctx* c;
    int stage;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t on = nullptr;
    StageTimer(pgb_ctx* ctx, int st, cudaStream_t on = nullptr);  // on: a stream other than the context's
    ~StageTimer();
};
void collect_timing(pgb_ctx* c);
#define PGB_LAUNCHED(c, k) ((c)->launches += (k))
// geometry / tree (tree.cu)
void upload_bodies(pgb_ctx* c);
void build_order(pgb_ctx* c);
void build_geometry(pgb_ctx* c);
void build_lists(pgb_ctx* c);
const FarTab& far_table(pgb_ctx* c, double kappa);
void refresh_lists(pgb_ctx* c);
void make_lists(pgb_ctx* c, const double* r2, const double* glo, const double* ghi, DBuf<int64_t>& noff,
                DBuf<int32_t>& nearl, DBuf<int64_t>& foff, DBuf<int32_t>& farl, DBuf<float4>& near4,
                DBuf<float4>& far4, int64_t& n_near, int64_t& n_far, unsigned long long* stats4);
void build_corrections(pgb_ctx* c);
BodyDev body_dev(const pgb_ctx* c);
Geo geo(const pgb_ctx* c);
// scans (tree.cu)
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host);
// matvec (matvec.cu)
void apply_operator(pgb_ctx* c, const double* x, double* y, int precision, bool known_only,
                    const int* known_mask = nullptr);
void apply_transpose(pgb_ctx* c, const double* lam, double* y, int precision);
// mode 0: A x; 1: the imposed-boundary terms only; 2: A (x + imposed); known_mask
// selects the surfaces of mode 1 (nullptr: all)
void apply_mode(pgb_ctx* c, const double* x, double* y, int precision, int mode, const int* known_mask);
void apply_full(pgb_ctx* c, const double* x, double* y, int precision);
void coulomb_rows(pgb_ctx* c, double* b);
void grad(pgb_ctx* c, const double* x, int precision, double tol, int max_iter, int restart, double* dq, double* dbc,
          double* dt, pgb_solve_stats* st);
// Speculation hook of gmres_op: the first time the residual estimate falls to
// abs_thresh (and not yet to the tolerance) the current iterate is formed in
// xs and fork(xs) is called; fork may start work on another stream.
struct GmresSpec {
    double abs_thresh = 0;
    double* xs = nullptr;
    bool forked = false;
    void (*fork)(pgb_ctx* c, const double* xs, void* user) = nullptr;
    void* user = nullptr;
};
int gmres_op(pgb_ctx* c, int prec, bool transpose, const double* b, double* x, double abs_tol, int max_it,
             int restart, int* matvecs, double* est_out, bool x_zero, GmresSpec* spec = nullptr);
double vec_dot(pgb_ctx* c, const double* a, const double* b);
// Problems of a block-diagonal system for arnoldi_step: B problems, rows
// poff[p] .. poff[p + 1] (device), act[p] (device) = 0 to skip problem p,
// nbp blocks per problem; per-problem strides of H (sH) and of the
// rotation / coefficient vectors (sV).
struct ArnSeg {
    int B, nbp;
    const int64_t* poff;
    const int* act;
    int64_t sH, sV;
};
// jdev != nullptr: the step of the column index held at jdev on the device
// (h is then the base of H, column j at h + j (mcap + 1)); buffers sized for
// columns up to mcap
void arnoldi_step(pgb_ctx* c, int j, double* w, double* h, double* hc, double* cs, double* sn, double* g,
                  double* out, const ArnSeg* sg, const int* jdev = nullptr, int mcap = 0);
double energy_unit_kcal();
void phi_reac(pgb_ctx* c, const double* x, double* out);
// solver (solver.cu)
void build_rhs(pgb_ctx* c, double* b, int precision, const double* bc = nullptr);
int solve(pgb_ctx* c, int mode, double tol, int max_iter, int restart, double* x, pgb_solve_stats* st);
void precond_prepare(pgb_ctx* c);
void precond_apply(pgb_ctx* c, const double* v, double* z, bool transpose, bool add);
// batched poses (batch.cu)
int solve_seg(pgb_ctx* c, int mode, double tol, int max_iter, int restart, double* x, pgb_solve_stats* st);
int solve_union(pgb_ctx* c, const std::vector<pgb_ctx*>& src, int32_t body_id, const double* R, const double* t,
                int32_t mode, double tol, int32_t max_iter, int32_t restart, double* F, pgb_solve_stats* st);
void destroy_union(pgb_ctx* c);
void reserve_product(pgb_ctx* c, int precision);
// energy (energy.cu)
void energies(pgb_ctx* c, const double* x, pgb_energies* e, pgb_energies* per_body);
void energies_noalloc(pgb_ctx* c, const double* x, pgb_energies* e);
// quadrature tables on the device (geometry.cu)
void rule_host(int K, const double** mu, const double** w);
}  // namespace pgb
