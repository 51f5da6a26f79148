/*
 * pgb -- treecode-accelerated boundary-element Poisson-Boltzmann solver for a
 * molecule near surfaces of imposed charge or potential (Cooper & Barba,
 * arXiv 1506.03745), for NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every call returns 0 (PGB_OK) or a negative status; no exception
 * crosses the boundary.  pgb_last_error() gives a one-line message for the
 * last failing call on a context.  All device pointers are plain CUDA device
 * addresses on the context's device, used on the context's stream; the
 * caller owns them.  Host pointers are only read during the call.
 *
 * Units (Section 2 of the paper): lengths in Angstrom, charges in e,
 * permittivities relative, kappa in 1/Angstrom, imposed surface charge in
 * C/m^2, imposed potential in volts, energies in kcal/mol.  Internally the
 * library works in e, Angstrom and eps0 = 1.
 *
 * Unknown vector layout (Eq. 6 / Eq. 7): bodies in load order; a dielectric
 * body (molecule) contributes [phi (N), dphi/dn (N)] -- the interior potential
 * and its normal derivative at its panel centroids -- and a surface body
 * contributes one block of N values: dphi/dn (imposed potential, Eq. 6) or
 * phi (imposed charge, Eq. 7).  Within a block, panels are in the order of
 * the triangles given to pgb_mesh_load.
 */
#ifndef PGB_H
#define PGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PGB_OK 0
#define PGB_EINVAL (-1)     /* bad argument; nothing changed */
#define PGB_ENOMEM (-2)     /* device allocation failed */
#define PGB_ECUDA (-3)      /* CUDA runtime error (message in pgb_last_error) */
#define PGB_ENOCONV (-4)    /* GMRES did not reach tol; solution and stats still written */
#define PGB_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define PGB_ESTATE (-6)     /* call out of order (e.g. matvec before pgb_tree_build) */
#define PGB_ECOLL (-7)      /* a collective callback of a sharded solve reported failure */

/* body kinds (Eq. 1): molecule interface Gamma_1, or surface Gamma_2 */
#define PGB_DIELECTRIC 0
#define PGB_SET_CHARGE 1
#define PGB_SET_POTENTIAL 2

/* precisions / solve modes */
#define PGB_FP32 0          /* matvec: P2P/M2P/P2M in FP32 with compensated accumulation;
                               solve: FP32 operator throughout (right-hand side included),
                               FP64 Arnoldi/Givens, no FP64 matvec */
#define PGB_FP64 1          /* every treecode kernel in FP64 */
#define PGB_FP32_REFINE 2   /* solve: FP32 inner GMRES, FP64 outer residual b - A x (one FP64
                               product with the imposed densities folded in per outer step) */
#define PGB_FP64_DS 3       /* matvec: the FP64 product with P2P and M2P evaluated in double-single
                               arithmetic (pairs of FP32, about 48 significant bits, relative
                               error near 1e-13) on the FP32 pipe; upward pass, near-field
                               corrections and assembly in FP64 (pgb_params.residual) */

/* Numerical parameters: the seven columns of the paper's parameter tables
 * (Tables 1, 2, 4: Gauss points in-element per edge, close-by, far-away;
 * treecode N_crit, P, theta; GMRES tol -- tol is passed to pgb_solve) plus
 * the target group size of the interaction lists. */
typedef struct pgb_params {
    int32_t K;            /* far-field points per panel: 1, 3, 4 or 7 (Section 3.1) */
    int32_t K_near;       /* fine rule inside 2L: 19 or 37 (Section 3.1; Table 1 uses 37) */
    int32_t n_edge;       /* Gauss points per edge for the self panel: 3, 6, 9 or 12 */
    int32_t P;            /* Taylor order: 0..8, 10, 12 or 15 (Section 3.2; Tables 1
                             and 2 use 15); pgb_grad takes 0..8 */
    double theta;         /* multipole acceptance criterion; 0 = direct sum */
    int32_t leaf_size;    /* N_crit: max panels per octree leaf, 1..1024 */
    int32_t group_size;   /* targets per interaction list: 32 (one warp) */
    int32_t p2p_item;     /* P2P work item: at most this many 32-point tiles of one group, 1..4096 (0 = 64) */
    int32_t m2p_item;     /* M2P work item: at most this many far nodes of one group, 1..4096 (0 = 64) */
    int32_t precond;      /* GMRES preconditioner: 0 none (the paper's solver), 1 block-diagonal: per
                             panel, the inverse of the 2x2 (molecule) or 1x1 (surface) block of its own
                             self terms, applied on the right so the residual test is unchanged */
    int32_t graphs;       /* 2 (default): the GMRES iterations after the first column of each restart
                             cycle are replayed from one CUDA graph whose device-side loop stops on
                             the residual estimate (no host round trip per iteration; for pose
                             batches the loop also tracks every pose's estimate and leaves finished
                             poses out of the products), and the
                             upward pass of every other product (P2M, moment shifts, far-field
                             coefficients) is captured once per tree and replayed; 1: the upward
                             pass only; 0: plain launches */
    int32_t lanes;        /* pgb_solve_batch: poses in flight at once, 1..16 (0 = 4); each lane is a copy
                             of the context with its own CUDA stream and host thread, kept between calls */
    int32_t overlap;      /* PGB_FP32_REFINE: 1 starts the FP64 product of the outer residual on a side
                             stream at the inner iterate whose residual is 1e-2 of its right-hand side
                             (1e4 tol if smaller) and finishes the residual with the FP32 product of the
                             remaining change, so the FP64 work overlaps the FP32 iterations (it pays
                             with residual = 0, whose kernels use the FP64 pipe); 0 (default): the
                             residual's product of the final iterate, after the inner solve */
    int32_t batch;        /* pgb_solve_batch / pgb_solve_poses: poses solved together as one
                             block-diagonal system, 1..64 (0 = 1); > 1 replaces the lanes: every stage
                             is one launch over the batch and GMRES runs in lockstep with per-pose
                             coefficients and stopping tests.  The batch's bodies (poses x bodies of
                             a pose) must not exceed 64. */
    int32_t residual;     /* PGB_FP32_REFINE: precision of the outer residual's product: 1 (default)
                             PGB_FP64_DS (GB300 issues FP64 at 1/64 of its FP32 rate), 0 native FP64 */
} pgb_params;

typedef struct pgb_solve_stats {
    int32_t iterations;        /* total inner GMRES iterations */
    int32_t outer_steps;       /* refinement steps (1 for PGB_FP64) */
    int32_t matvecs;           /* operator applications, all precisions */
    int32_t matvecs_fp64;      /* of which FP64 */
    double rel_residual;       /* final ||b - A x|| / ||b|| (FP64 operator) */
} pgb_solve_stats;

typedef struct pgb_energies {
    double coulomb;            /* Coulomb energy of the point charges */
    double solvation;          /* Eq. 11: 1/2 sum_k q_k phi_reac(r_k) */
    double surface;            /* Eq. 15 */
    double total;              /* Eq. 16 */
} pgb_energies;

typedef struct pgb_tree_info {
    int64_t n_panels;          /* all bodies */
    int64_t n_unknowns;
    int64_t n_nodes;
    int64_t n_leaves;
    int64_t n_groups;
    int64_t n_near;            /* (group, leaf) near pairs */
    int64_t n_far;             /* (group, node) far pairs */
    int64_t p2p_pairs;         /* target x source-point P2P interactions per matvec */
    int64_t p2p_laplace_pairs; /* of which also need the Laplace kernel */
    int64_t m2p_pairs;         /* target x node M2P evaluations per matvec */
    int64_t m2p_laplace_pairs;
    int64_t n_corrections;     /* near-field correction entries */
    int64_t n_p2p_items;       /* P2P work items (one block each) per matvec */
    int64_t n_m2p_items;       /* M2P work items */
} pgb_tree_info;

/* Device time per stage of the hot path, accumulated with CUDA events on
 * the context's stream while timing is enabled (pgb_timing). */
#define PGB_STAGE_SOURCES 0   /* FP32 matvec: panel densities and per-point source terms */
#define PGB_STAGE_UPWARD 1    /* FP32 matvec: P2M at the leaves + moment shifts to the root */
#define PGB_STAGE_P2P 2       /* FP32 matvec: P2P over the near leaves */
#define PGB_STAGE_M2P 3       /* FP32 matvec: M2P over the far nodes */
#define PGB_STAGE_ASSEMBLE 4  /* FP32 matvec: near-field corrections + block rows */
#define PGB_STAGE_KRYLOV 5    /* Arnoldi (CGS2), Givens, updates */
#define PGB_STAGE_TREE 6      /* pgb_tree_build */
#define PGB_STAGE_ENERGY 7    /* pgb_energy */
#define PGB_STAGE_RHS 8       /* right-hand side (Coulomb rows; imposed terms are FP64 matvecs) */
#define PGB_STAGE_FP64 9      /* add to stages 0-4 for the FP64 matvec */
#define PGB_N_STAGES 14
typedef struct pgb_stage_times {
    double ms[PGB_N_STAGES];        /* summed device milliseconds */
    int64_t calls[PGB_N_STAGES];    /* timed intervals */
    int64_t kernel_launches;        /* kernels the library ran (all stages; a replayed
                                       graph counts the kernels it ran) */
    int64_t host_launches;          /* launch calls the host made: kernels launched
                                       directly plus graph launches */
} pgb_stage_times;

/* Create a context on the current CUDA device.  p may be NULL (defaults:
 * K=7, K_near=19, n_edge=9, P=6, theta=0.5, leaf_size=32, group_size=32,
 * p2p_item=64, m2p_item=64, precond=0, graphs=2, lanes=4, overlap=0,
 * batch=1, residual=1).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).  Returns
 * PGB_EINVAL for out-of-range parameters. */
int pgb_create(struct pgb_ctx** ctx, const pgb_params* p, void* cuda_stream);
int pgb_destroy(struct pgb_ctx* ctx);
const char* pgb_last_error(const struct pgb_ctx* ctx);
int pgb_default_params(pgb_params* p);

/* Load one body (Section 2, Eq. 1; Section 3.1 discretisation).
 * verts: nv*3 doubles (Angstrom), tris: nt*3 int32, counter-clockwise seen
 * from the solvent so the normal points into the solvent.  For
 * PGB_DIELECTRIC: eps_in > 0 and nq >= 0 charges (charge_xyz nq*3, charge_q
 * nq, in e); bc_value ignored.  For PGB_SET_CHARGE: bc_value = sigma0 (C/m^2);
 * for PGB_SET_POTENTIAL: bc_value = phi0 (V); charges must be empty.
 * Host arrays are copied.  *body_id_out receives the body index.  Loading a
 * body invalidates the tree (call pgb_tree_build again). */
int pgb_mesh_load(struct pgb_ctx* ctx, int32_t kind, const double* verts, int64_t nv,
                  const int32_t* tris, int64_t nt, double eps_in,
                  const double* charge_xyz, const double* charge_q, int64_t nq,
                  double bc_value, int32_t* body_id_out);

/* Replace the charge values of dielectric body body_id (nq must equal the
 * loaded count; positions are kept).  Does not invalidate the tree. */
int pgb_set_charges(struct pgb_ctx* ctx, int32_t body_id, const double* charge_q, int64_t nq);

/* Replace the imposed sigma0 (C/m^2) or phi0 (V) of surface body body_id.
 * Does not invalidate the tree. */
int pgb_set_bc(struct pgb_ctx* ctx, int32_t body_id, double bc_value);

/* Solvent permittivity and inverse Debye length (Eq. 1); kappa >= 0. */
int pgb_set_solvent(struct pgb_ctx* ctx, double eps_out, double kappa);

/* Rigid pose of a body: world = R * body + t (R row-major 3x3, proper
 * rotation within 1e-9).  Invalidates interaction lists and cross-body
 * near-field entries (pgb_tree_build again). */
int pgb_set_pose(struct pgb_ctx* ctx, int32_t body_id, const double R[9], const double t[3]);

/* Geometry, octree, interaction lists and near-field corrections for the
 * current bodies and poses (Section 3.1 tiers, Section 3.2 treecode). */
int pgb_tree_build(struct pgb_ctx* ctx);
int pgb_tree_stats(struct pgb_ctx* ctx, pgb_tree_info* info);

/* Recompute what the current poses change -- world geometry, node and group
 * centres, the offsets of the list entries and P2P tiles, cross-body
 * near-field entries -- while keeping the near/far interaction lists (and the
 * work items) of the last pgb_tree_build.  The product is then the treecode
 * with those lists at the new poses: a small pose change (finite differences
 * of an energy in a translation, as for the adjoint gradient of pgb_grad)
 * moves no node across the acceptance criterion, so the difference carries no
 * jump from a changed list.  The caller keeps the poses close to the ones the
 * lists were built for (the criterion is not re-tested).  PGB_ESTATE without
 * such a tree (nothing built, or bodies loaded since). */
int pgb_tree_refresh(struct pgb_ctx* ctx);

/* Drop every cached geometric structure (Morton order, octree, each body's
 * own near-field entries), so that the next pgb_tree_build recomputes all of
 * them (pgb_tree_build otherwise rebuilds only what loads, poses and the
 * solvent changed). */
int pgb_tree_reset(struct pgb_ctx* ctx);

/* Number of unknowns 2*N_dielectric + N_surface. */
int pgb_num_unknowns(struct pgb_ctx* ctx, int64_t* n);

/* y = A x, the block operator of Eq. 6 / Eq. 7 applied by the treecode
 * (Section 3.2): x, y device arrays of n_unknowns floats (PGB_FP32) or
 * doubles (PGB_FP64).  x and y must not overlap. */
int pgb_matvec(struct pgb_ctx* ctx, const void* x, void* y, int32_t precision);

/* Right-hand side of Eq. 6 / Eq. 7 (Coulomb rows with the 1/eps_in of Eq. 5,
 * imposed-boundary terms moved to the right) into device doubles b. */
int pgb_rhs(struct pgb_ctx* ctx, double* b);

/* GMRES solve of Eq. 6 / Eq. 7 (Section 3.2).  mode PGB_FP64, PGB_FP32_REFINE
 * or PGB_FP32; tol on ||b - A x||/||b|| (measured with the FP64 operator,
 * except in PGB_FP32 mode where the FP32 operator is used); max_iter total inner iterations;
 * restart = Krylov dimension (1..256).  x_out: device doubles, n_unknowns.
 * Returns PGB_ENOCONV (x_out and stats still written) when tol is not met. */
int pgb_solve(struct pgb_ctx* ctx, int32_t mode, double tol, int32_t max_iter, int32_t restart,
              double* x_out, pgb_solve_stats* stats);

/* Gradients of the total free energy (Eq. 16) of the solved system by the
 * discrete adjoint (the paper has no gradient; this is the adjoint of
 * Eq. 6 / Eq. 7): solves A^T lam = dF/dx with the transposed treecode
 * (GMRES, FP64 Arnoldi; operator in `precision` = PGB_FP32 or PGB_FP64, tol
 * relative to ||dF/dx||), then
 *   dF_dq[n_q]      dF/dq_k for every charge (kcal/mol/e), bodies in load order;
 *   dF_dbc[n_bodies] dF/dsigma0 (kcal/mol per C/m^2) or dF/dphi0 (per V) for
 *                   surfaces, 0 for molecules;
 *   dF_dt[3 n_bodies] dF/dt for a rigid translation of each body (kcal/mol/A).
 * x: the solution of pgb_solve (device doubles).  Host output pointers may be
 * NULL.  Needs the bodies farther apart than 2L (no cross-body near-field
 * entries), else PGB_EINVAL.  adj (may be NULL) receives the
 * adjoint iterations and the relative residual of A^T lam = dF/dx. */
int pgb_grad(struct pgb_ctx* ctx, const double* x, int32_t precision, double tol, int32_t max_iter, int32_t restart,
             double* dF_dq, double* dF_dbc, double* dF_dt, pgb_solve_stats* adj);

/* y = A^T lam, the transposed operator (device doubles, n_unknowns each). */
int pgb_matvec_transpose(struct pgb_ctx* ctx, const double* lam, double* y, int32_t precision);

/* Rigid-pose sweep (the orientation studies of Section 1): for each of B
 * poses (R: B x 9 row-major, t: B x 3) of body body_id, set the pose,
 * rebuild what the pose changes (world geometry, lists, cross-body near-field
 * entries; each body's own near-field entries and tree are reused), solve
 * (mode, tol, max_iter, restart as pgb_solve) and evaluate the energies:
 * F_out[4b..4b+3] = Coulomb, solvation, surface, total (kcal/mol); stats may be
 * NULL or hold B entries.  The body keeps the last pose.  Returns PGB_ENOCONV
 * if any pose missed tol (all poses are still written). */
/* With pgb_params.batch > 1 the poses go in chunks of `batch` to a union
 * context (kept on ctx between calls) that holds every pose's bodies side by
 * side, as independent problems of one block-diagonal system: the tree,
 * lists and near-field entries never couple two poses, each treecode stage
 * is one launch over the chunk, and GMRES advances all poses together, each
 * with its own Krylov coefficients and stopping test (the residual each pose
 * reaches is its own).  A last partial chunk is padded with repeats of its
 * last pose, whose results are dropped. */
int pgb_solve_batch(struct pgb_ctx* ctx, int32_t body_id, const double* R, const double* t, int64_t B, int32_t mode,
                    double tol, int32_t max_iter, int32_t restart, double* F_out, pgb_solve_stats* stats);

/* Poses of several molecules (contexts of possibly different mesh sizes,
 * each with the same solvent and the same body layout) solved in batches as
 * above: pose b is body body_id of ctxs[pose_ctx[b]] at (R + 9 b, t + 3 b);
 * the other bodies keep their poses in their own contexts.  ctxs[0] holds
 * the union context and its parameters (batch, K, P, theta, ...) apply; a
 * chunk is the next ctxs[0]->p.batch poses in order, so listing the poses
 * with a repeating sequence of contexts lets every chunk reuse one union
 * (its trees and near-field entries).  F_out and stats as pgb_solve_batch;
 * the contexts' own trees are left as they were.  ctxs[k] must stay alive
 * and unchanged while the call runs. */
int pgb_solve_poses(struct pgb_ctx* const* ctxs, int32_t n_ctx, const int32_t* pose_ctx, int32_t body_id,
                    const double* R, const double* t, int64_t B, int32_t mode, double tol, int32_t max_iter,
                    int32_t restart, double* F_out, pgb_solve_stats* stats);

/* Energies (Section 3.3, Eq. 11-16) of a solution x (device doubles):
 * Coulomb, solvation (phi_reac of Eq. 13 at the charges with the three-tier
 * rule), surface (Eq. 15) and total, summed over bodies.  per_body may be
 * NULL or an array of n_bodies entries. */
int pgb_energy(struct pgb_ctx* ctx, const double* x, pgb_energies* e, pgb_energies* per_body);

/* Energies like pgb_energy, for callers that must not allocate device
 * memory: code running under an external memory budget or a pool that owns
 * all of the device's memory, and code paths where cudaMalloc would
 * serialise the device (for example between launches of a latency-bound
 * pose sweep).  The paper has no counterpart; this is a library feature.
 *
 * It allocates nothing: its scratch (reaction potential at every charge,
 * per-body sums and charge offsets) lives in one file-scope device array of
 * PGB_NOALLOC_MAX_CHARGES + 4*64 + 1 doubles (about 514 KB) that every GPU
 * which loads libpgb holds until the process exits.  The context must have been
 * built (pgb_tree_build) beforehand; its buffers are reused, not grown.
 * Returns PGB_EINVAL when the context holds more than PGB_NOALLOC_MAX_CHARGES
 * charges.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and each call overwrites every entry it reads,
 * so calls that overlap on the GPU (different streams or threads without
 * ordering) race and must be serialised by the caller. */
#define PGB_NOALLOC_MAX_CHARGES 65536
int pgb_energy_noalloc(struct pgb_ctx* ctx, const double* x, pgb_energies* e);

/* Nested interfaces (Section 2 after Eq. 7: Stern layers and solvent-filled
 * cavities add surfaces, hence block rows).  Places body `id` in the interior
 * region of the dielectric body `parent` (-1: in the solvent, the default)
 * and gives its own interior the screening kappa_in (A^-1, default 0; only
 * dielectric bodies without charges may have one).  Every region -- the
 * solvent and each dielectric body's interior -- then has its permittivity
 * (eps_out, or the body's eps_in) and screening, and each row is Green's
 * representation in the region it belongs to: a dielectric body's interior
 * row in its interior, its exterior row in the region around it, with the
 * bodies bounding that region as sources (from inside: dphi; from outside:
 * (eps_in / eps_region) dphi, the flux condition).  A Stern layer around a
 * molecule M is a dielectric body S with eps_in = eps_out and kappa_in = 0
 * that is M's parent; a cavity in M is a dielectric body with parent M.  The
 * solvation energy of M includes its cavities' share of the reaction
 * potential.  Surfaces with imposed values stay in the solvent; gradients,
 * pgb_matvec_transpose, pgb_energy_noalloc and pose batches (batch > 1) are
 * not available with nesting (PGB_EINVAL).  Products run one treecode pass
 * per region.  PGB_EINVAL for a bad id, a non-dielectric parent, a cycle, a
 * negative kappa_in, or a screened interior holding charges. */
int pgb_set_region(struct pgb_ctx* ctx, int32_t id, int32_t parent, double kappa_in);

/* Treecode parameter autotuner (a library feature; the paper fixes its
 * parameters by hand, Tables 1, 2, 4).  For every candidate (theta, P,
 * leaf_size) of the given lists it builds the tree, times `reps` FP32
 * matvecs with CUDA events and solves in PGB_FP32_REFINE mode to `tol` for
 * the total energy (so the FP64-class residual product, whose near field
 * grows with the leaf size, is in the time).  The reference is the candidate with the smallest theta, largest P
 * and first leaf size; among the candidates whose total energy is within
 * target_rel_err of the reference, the one with the shortest solve time
 * (tree build + solve) is chosen.  With it, the work-item sizes p2p_item and
 * m2p_item (one after the other, from {16, 32, 64, 128}) are then chosen by
 * the time of `reps` FP32 matvecs; the product does not depend on them.  The
 * context keeps the chosen parameters and a built tree; *chosen receives them.  report (may be NULL) receives, per
 * candidate in loop order theta-major, then P, then leaf: matvec ms, solve ms,
 * relative energy difference to the reference. */
int pgb_autotune(struct pgb_ctx* ctx, const double* thetas, int32_t n_theta, const int32_t* Ps, int32_t n_P,
                 const int32_t* leaves, int32_t n_leaf, int32_t reps, double tol, double target_rel_err,
                 pgb_params* chosen, double* report);

/* Enable (1) or disable (0) stage timing.  If out is not NULL the stream
 * is synchronised and the times and launch count accumulated since the last
 * read are written to out and reset.  Launch counting is always on. */
int pgb_timing(struct pgb_ctx* ctx, int32_t enable, pgb_stage_times* out);

/* Debug/test export of the tree (host arrays sized from pgb_tree_stats):
 * perm[n_panels] (sorted position -> panel index within its body, bodies
 * concatenated), near_off[n_groups+1], near_node[n_near], far_off[n_groups+1],
 * far_node[n_far].  Any pointer may be NULL. */
int pgb_tree_export(struct pgb_ctx* ctx, int32_t* perm, int64_t* near_off, int32_t* near_node,
                    int64_t* far_off, int32_t* far_node);

/* Diagnostic: evaluate the device's FP64 elementary functions of the
 * near-field sums at n host points x (no context; the current device, its
 * default stream, synchronous).  out (host, n x 7, row-major) receives per
 * point: the one-step and two-step Newton reciprocal square roots (valid for
 * 1e-30 < x < 1e30), the Taylor 2^x (valid for -2^30 < x <= 1020), the CUDA
 * library's rsqrt(x) and exp2(x) for comparison, and the double-single
 * reciprocal square root (1e-30 < x < 1e30) and 2^x (-100 < x < 127) of the
 * PGB_FP64_DS product, each converted back to a double.  PGB_EINVAL for n < 0 or a
 * NULL pointer with n > 0; PGB_ECUDA on a CUDA error. */
int pgb_math_check(const double* x, int64_t n, double* out);

/* Orientation free-energy landscape of a pose sweep (the application the
 * paper motivates, Section 1: how a protein orients near a charged surface):
 * F holds total free energies (kcal/mol) of n_orient orientations x n_gap
 * separations, orientation-major (F[o * n_gap + g], the order of
 * pgb_solve_batch poses listed orientation by orientation).  For each
 * separation g, with Boltzmann weights p_o = e^{-F_o/kT} / sum e^{-F/kT} at
 * the given temperature (K; k = 0.0019872043 kcal/(mol K)):
 *   out[3g]     the most likely orientation (its index, as a double),
 *   out[3g + 1] its probability,
 *   out[3g + 2] the orientation-averaged free energy -kT ln <e^{-F/kT}>
 *               (the mean over the n_orient orientations), kcal/mol.
 * Host arrays; no device call.  PGB_EINVAL for bad sizes, a non-positive
 * temperature or a non-finite energy. */
int pgb_orientation_landscape(const double* F, int32_t n_orient, int32_t n_gap, double temperature, double* out);

/* ---- one solve sharded over ranks (one process per GPU) ----
 * The GMRES solve of Section 3.2 split by target rows: every rank holds the
 * whole geometry, tree and near field and computes the upward pass itself;
 * rank r computes the rows of a contiguous range of target groups (Morton
 * order, balanced by their P2P and M2P work) from the full density vector,
 * assembled by one allgather per product, and the Arnoldi dot products are
 * summed by allreduce.  The unknowns are taken in the sharded order: sorted
 * panel by sorted panel, each panel's rows together (phi, dphi/dn for a
 * molecule; u for a surface), so that each rank's rows are contiguous.
 * Nested interfaces are not sharded (PGB_EINVAL). */

/* Balanced contiguous split of n_groups groups of the given (host) work over
 * world ranks: bounds[r] .. bounds[r+1] (world + 1 entries) are rank r's
 * groups.  Host only, no device call. */
int pgb_shard_partition(const double* work, int64_t n_groups, int32_t world, int64_t* bounds);

/* The ranks' rows in the sharded order: row_begin[r] .. row_begin[r+1]
 * (world + 1 host entries) for the context's built tree. */
int pgb_shard_rows(struct pgb_ctx* ctx, int32_t world, int64_t* row_begin);

/* x (caller order) -> xs (sharded order), or back with inverse != 0; device
 * doubles, n_unknowns each. */
int pgb_to_sharded(struct pgb_ctx* ctx, const double* x, double* xs, int32_t inverse);

/* Rank `rank`'s rows of y = A x: xs the whole vector in the sharded order,
 * ys its rows (row_begin[rank+1] - row_begin[rank] device doubles; the
 * product's precision as pgb_matvec, in and out FP64).  The rows are those of
 * the whole product (same arithmetic). */
int pgb_matvec_shard(struct pgb_ctx* ctx, int32_t rank, int32_t world, const double* xs, double* ys,
                     int32_t precision);

/* Collectives of a sharded solve, done by the caller (torch.distributed over
 * NCCL or gloo, MPI, ...).  op PGB_COLL_ALLGATHER: the exchange buffer xs
 * (n_unknowns device doubles, sharded order) holds this rank's rows;
 * fill every other rank's rows from the other ranks (count = n_unknowns).
 * op PGB_COLL_ALLREDUCE: replace the first count doubles of the reduce buffer
 * by their sum over the ranks.  The library has synchronised its stream
 * before the call; the callback returns 0 once the exchange is complete in
 * device memory, non-zero on failure (the solve then returns PGB_ECOLL). */
#define PGB_COLL_ALLGATHER 0
#define PGB_COLL_ALLREDUCE 1
typedef int (*pgb_collective_fn)(void* user, int32_t op, int64_t count);

/* Sharded solve of Eq. 6 / Eq. 7: mode PGB_FP64 or PGB_FP32_REFINE (FP32
 * inner GMRES, FP64-class outer residual), tol, max_iter and restart as
 * pgb_solve.  xs: exchange buffer (n_unknowns device doubles), red: reduce
 * buffer (restart + 2 device doubles), both the caller's and used by coll.
 * Every rank must make the call with the same arguments but its rank; on
 * return x_out (device doubles, caller order) holds the whole solution on
 * every rank and stats (may be NULL) the iterations. */
int pgb_solve_shard(struct pgb_ctx* ctx, int32_t rank, int32_t world, double* xs, double* red,
                    pgb_collective_fn coll, void* user, int32_t mode, double tol, int32_t max_iter,
                    int32_t restart, double* x_out, pgb_solve_stats* stats);

/* Diagnostic: the host-computed table that turns a node's Taylor moments
 * (Section 3.2) into the coefficients its far field is evaluated from, for
 * order P (0..15) and screening kappa >= 0.  With T = (P+1)(P+2)(P+3)/6, out
 * (host, n = 2 T^2 doubles) receives the Yukawa table then the Laplace
 * table, each T x T row-major: row = coefficient of S^(a,b,c), S = R/|R|^2,
 * in the order a = 0..P, b = 0..P-a, c = 0..P-a-b; column = moment M_k with
 * k in the graded order (total degree, then k_x and k_y descending).  The
 * far field at R from the node centre is
 *   U_Y = e^{-kappa r}/r sum_p g_p(kappa r) sum_{a+b+c=p} Y[.][k] M_k S^(a,b,c),
 *   U_L = 1/r sum L[.][k] M_k S^(a,b,c),
 * g_0 = 1, g_1 = -(1+x), g_p = x^2 g_{p-2} - (2p-1) g_{p-1} (the sum over
 * k of G_k(R) M_k with G_k the Taylor coefficients of e^{-kappa r}/r or 1/r,
 * without the 1/(4 pi)).  No device call; PGB_EINVAL for a bad P, kappa,
 * pointer or n. */
int pgb_far_table(int32_t P, double kappa, double* out, int64_t n);

/* Diagnostic: *n receives the number of memory allocations libpgb has made
 * in this process so far (device buffers, stream-ordered or not, and pinned
 * host buffers).  No context and no device call; PGB_EINVAL for n = NULL.
 * Two reads around a call show whether that call allocated. */
int pgb_alloc_count(int64_t* n);


#ifdef __cplusplus
}
#endif
#endif
