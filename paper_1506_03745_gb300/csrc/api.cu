// C entry points of libpgb (declared in include/pgb.h).
#include <math.h>

#include <atomic>
#include <cstring>
#include <exception>
#include <new>
#include <thread>

#include "common.cuh"
#include "ds.cuh"
#include "pgb_internal.cuh"

namespace pgb {
thread_local cudaStream_t g_alloc_stream = nullptr;
thread_local bool g_alloc_scoped = false;
static std::atomic<int64_t> g_alloc_count{0};
void note_alloc() { g_alloc_count.fetch_add(1, std::memory_order_relaxed); }
void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error{PGB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
    }
}
void fail(int code, const std::string& msg) { throw Error{code, msg}; }

__global__ void k_math_check(int64_t n, const double* x, double* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    y[7 * i] = rsqrt_nr<1>(v);
    y[7 * i + 1] = rsqrt_nr<2>(v);
    y[7 * i + 2] = exp2_taylor(v);
    y[7 * i + 3] = rsqrt(v);
    y[7 * i + 4] = exp2(v);
    y[7 * i + 5] = ds_to_double(ds_rsqrt(ds_from_double(v)));
    y[7 * i + 6] = ds_to_double(ds_exp2(ds_from_double(v)));
}

static cudaEvent_t get_event(pgb_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

StageTimer::StageTimer(pgb_ctx* ctx, int st, cudaStream_t s) : c(ctx), stage(st), on(s) {
    if (!c->timing) return;
    e0 = get_event(c);
    e1 = get_event(c);
    cudaEventRecord(e0, on ? on : c->stream);
}

StageTimer::~StageTimer() {
    if (!e0) return;
    cudaEventRecord(e1, on ? on : c->stream);
    c->ev_pending.push_back({stage, {e0, e1}});
}

void collect_timing(pgb_ctx* c) {
    if (c->ev_pending.empty()) return;
    cuda_check(cudaStreamSynchronize(c->stream), "timing sync");
    for (auto& p : c->ev_pending) {
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, p.second.first, p.second.second), "cudaEventElapsedTime");
        c->stage_ms[p.first] += ms;
        c->stage_calls[p.first] += 1;
        c->ev_pool.push_back(p.second.first);
        c->ev_pool.push_back(p.second.second);
    }
    c->ev_pending.clear();
}
void convert_f32_f64(const float* a, double* b, int64_t n, cudaStream_t s);
void convert_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s);
}  // namespace pgb

using namespace pgb;

template <class F>
static int guard(pgb_ctx* c, F f) {
    AllocScope scope(c ? c->stream : nullptr);
    try {
        int r = f();
        if (c && r == PGB_OK) c->err.clear();
        return r;
    } catch (const Error& e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return PGB_ENOMEM;
    } catch (const std::exception& e) {
        if (c) c->err = e.what();
        return PGB_EINVAL;
    }
}

static int check_params(const pgb_params* p, std::string& why) {
    if (!(p->K == 1 || p->K == 3 || p->K == 4 || p->K == 7)) why = "K must be 1, 3, 4 or 7";
    else if (p->K_near != 19 && p->K_near != 37) why = "K_near must be 19 or 37";
    else if (!(p->n_edge == 3 || p->n_edge == 6 || p->n_edge == 9 || p->n_edge == 12)) why = "n_edge must be 3, 6, 9 or 12";
    else if (!p_supported(p->P)) why = "P must be in 0..8, or 10, 12 or 15";
    else if (!(p->theta >= 0 && p->theta < 1)) why = "theta must be in [0, 1)";
    else if (p->leaf_size < 1 || p->leaf_size > 1024) why = "leaf_size must be in 1..1024";
    else if (p->group_size != 32) why = "group_size must be 32";
    else if (p->p2p_item < 0 || p->p2p_item > 4096) why = "p2p_item must be in 1..4096 (0 = default)";
    else if (p->m2p_item < 0 || p->m2p_item > 4096) why = "m2p_item must be in 1..4096 (0 = default)";
    else if (p->precond != 0 && p->precond != 1) why = "precond must be 0 or 1";
    else if (p->graphs < 0 || p->graphs > 2) why = "graphs must be 0, 1 or 2";
    else if (p->lanes < 0 || p->lanes > 16) why = "lanes must be in 1..16 (0 = default)";
    else if (p->overlap != 0 && p->overlap != 1) why = "overlap must be 0 or 1";
    else if (p->batch < 0 || p->batch > PGB_MAX_BODIES) why = "batch must be in 1..64 (0 = 1)";
    else if (p->residual != 0 && p->residual != 1) why = "residual must be 0 or 1";
    else return PGB_OK;
    return PGB_EINVAL;
}

// Why (R, t) is not a rigid pose (R orthonormal with det > 0, t finite), or
// nullptr.
static const char* pose_error(const double* R, const double* t) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[3 * i + k] * R[3 * j + k];
            if (!(fabs(s - (i == j ? 1.0 : 0.0)) < 1e-9)) return "R is not orthonormal";
        }
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) + R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (!(det > 0) || !isfinite(t[0]) || !isfinite(t[1]) || !isfinite(t[2]))
        return "R must be a proper rotation and t finite";
    return nullptr;
}

// Poses b = 0 .. B-1 (body body_id of ctxs[pose_ctx[b]], or of ctxs[0] when
// pose_ctx is null) through c's union context in chunks of c->p.batch.  A
// last partial chunk is padded: with the union's own sources at their
// current poses when its sequence of sources starts like the chunk (the
// union is then reused), else with repeats of the chunk's last pose.
static int solve_chunks(pgb_ctx* c, pgb_ctx* const* ctxs, const int32_t* pose_ctx, int32_t body_id,
                        const double* R, const double* t, int64_t B, int32_t mode, double tol, int32_t max_iter,
                        int32_t restart, double* F_out, pgb_solve_stats* stats) {
    for (int64_t b = 0; b < B; ++b) {
        const char* why = pose_error(R + 9 * b, t + 3 * b);
        if (why) fail(PGB_EINVAL, "pose " + std::to_string(b) + ": " + why);
    }
    const int Bc = (int)std::min<int64_t>(c->p.batch, B);
    auto src_of = [&](int64_t b) { return ctxs[pose_ctx ? pose_ctx[b] : 0]; };
    std::vector<pgb_ctx*> src(Bc);
    std::vector<double> Rc(9 * Bc), tc(3 * Bc), Fc(4 * Bc);
    std::vector<pgb_solve_stats> sc(Bc);
    int out = PGB_OK;
    for (int64_t k0 = 0; k0 < B; k0 += Bc) {
        const int nk = (int)std::min<int64_t>(Bc, B - k0);
        bool prefix = c->union_ctx && (int)c->union_src.size() == Bc;
        for (int q = 0; q < nk && prefix; ++q) prefix = c->union_src[q] == src_of(k0 + q);
        for (int q = 0; q < Bc; ++q) {
            const double *Rq, *tq;
            if (q < nk || !prefix) {
                const int64_t b = k0 + std::min(q, nk - 1);
                src[q] = src_of(b);
                Rq = R + 9 * b;
                tq = t + 3 * b;
            } else {
                src[q] = c->union_src[q];
                Rq = src[q]->bodies[body_id].R;
                tq = src[q]->bodies[body_id].t;
            }
            memcpy(&Rc[9 * q], Rq, 9 * sizeof(double));
            memcpy(&tc[3 * q], tq, 3 * sizeof(double));
        }
        const int r = solve_union(c, src, body_id, Rc.data(), tc.data(), mode, tol, max_iter, restart, Fc.data(),
                                  sc.data());
        if (r != PGB_OK && r != PGB_ENOCONV) return r;
        for (int q = 0; q < nk; ++q) {
            memcpy(F_out + 4 * (k0 + q), &Fc[4 * q], 4 * sizeof(double));
            if (stats) stats[k0 + q] = sc[q];
            if (!(sc[q].rel_residual <= tol)) out = PGB_ENOCONV;
        }
    }
    return out;
}

// ---------------------------------------------------------------- pose lanes
// One pose of a batch on context c: set the pose, rebuild what it changes,
// solve and evaluate the energies into F4 (Coulomb, solvation, surface, total).
static int solve_pose(pgb_ctx* c, int32_t body_id, int64_t index, const double* R, const double* t, int32_t mode,
                      double tol, int32_t max_iter, int32_t restart, double* F4, pgb_solve_stats* stp) {
    const int r = pgb_set_pose(c, body_id, R, t);
    if (r != PGB_OK) fail(r, "pose " + std::to_string(index) + ": " + c->err);
    {
        StageTimer tm(c, PGB_STAGE_TREE);
        if (!c->order_valid) {
            upload_bodies(c);
            build_order(c);
            c->intra_valid = false;
        }
        build_geometry(c);
        build_lists(c);
        build_corrections(c);  // intra-body entries are reused across poses
        c->tree_valid = true;
    }
    c->d_xbatch.resize(c->n_unk);
    pgb_solve_stats st{};
    const int rs = solve(c, mode, tol, max_iter, restart, c->d_xbatch, &st);
    pgb_energies e{};
    {
        StageTimer tm(c, PGB_STAGE_ENERGY);
        energies(c, c->d_xbatch, &e, nullptr);
    }
    F4[0] = e.coulomb;
    F4[1] = e.solvation;
    F4[2] = e.surface;
    F4[3] = e.total;
    if (stp) *stp = st;
    return rs;
}

static void destroy_lanes(pgb_ctx* c) {
    for (pgb_ctx* l : c->lane_ctx) pgb_destroy(l);
    c->lane_ctx.clear();
}

static bool same_params(const pgb_params& a, const pgb_params& b) {
    return a.K == b.K && a.K_near == b.K_near && a.n_edge == b.n_edge && a.P == b.P && a.theta == b.theta &&
           a.leaf_size == b.leaf_size && a.group_size == b.group_size && a.p2p_item == b.p2p_item &&
           a.m2p_item == b.m2p_item && a.precond == b.precond && a.graphs == b.graphs && a.overlap == b.overlap &&
           a.residual == b.residual;
}

// Lane contexts: copies of c (bodies, solvent, parameters) with their own
// non-blocking stream; kept while c's configuration is unchanged.  The other
// bodies' poses follow c at every call.
static void ensure_lanes(pgb_ctx* c, int L, int32_t body_id) {
    bool ok = (int)c->lane_ctx.size() >= L && c->lane_gen == c->config_gen;
    for (pgb_ctx* l : c->lane_ctx) ok = ok && same_params(l->p, c->p);
    if (!ok) {
        destroy_lanes(c);
        for (int i = 0; i < L; ++i) {
            pgb_ctx* l = new pgb_ctx;
            l->p = c->p;
            l->p.lanes = 1;
            l->eps_out = c->eps_out;
            l->kappa = c->kappa;
            l->bodies = c->bodies;
            note_alloc();
            if (cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaMallocHost(&l->h_pinned, 64) != cudaSuccess) {
                (void)cudaGetLastError();
                pgb_destroy(l);
                fail(PGB_ECUDA, "lane context creation failed");
            }
            l->owns_stream = true;
            c->lane_ctx.push_back(l);
        }
        c->lane_gen = c->config_gen;
    }
    for (pgb_ctx* l : c->lane_ctx) {
        l->timing = c->timing;
        for (size_t k = 0; k < c->bodies.size(); ++k) {
            if ((int32_t)k == body_id) continue;
            auto &a = l->bodies[k], &b = c->bodies[k];
            if (memcmp(a.R, b.R, sizeof(a.R)) || memcmp(a.t, b.t, sizeof(a.t))) {
                memcpy(a.R, b.R, sizeof(a.R));
                memcpy(a.t, b.t, sizeof(a.t));
                l->tree_valid = false;
            }
        }
    }
}

// B poses over L lanes, each lane a host thread that takes the next pose
// until none is left; the lanes' kernels overlap on the GPU.
static int solve_lanes(pgb_ctx* c, int L, int32_t body_id, const double* R, const double* t, int64_t B, int32_t mode,
                       double tol, int32_t max_iter, int32_t restart, double* F_out, pgb_solve_stats* stats) {
    ensure_lanes(c, L, body_id);
    int dev = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    std::atomic<int64_t> next(0);
    std::vector<int> rc(L, PGB_OK);
    std::vector<std::string> msg(L);
    std::vector<std::thread> th;
    for (int l = 0; l < L; ++l)
        th.emplace_back([&, l]() {
            pgb_ctx* lc = c->lane_ctx[l];
            AllocScope scope(lc->stream);
            try {
                cuda_check(cudaSetDevice(dev), "cudaSetDevice");
                for (int64_t b; (b = next.fetch_add(1)) < B;) {
                    const int r = solve_pose(lc, body_id, b, R + 9 * b, t + 3 * b, mode, tol, max_iter, restart,
                                             F_out + 4 * b, stats ? stats + b : nullptr);
                    if (r != PGB_OK && rc[l] == PGB_OK) rc[l] = r;
                }
                cuda_check(cudaStreamSynchronize(lc->stream), "lane sync");
            } catch (const Error& e) {
                rc[l] = e.code;
                msg[l] = e.msg;
            } catch (const std::exception& e) {
                rc[l] = PGB_EINVAL;
                msg[l] = e.what();
            }
        });
    for (auto& x : th) x.join();
    int out = PGB_OK;
    for (int l = 0; l < L; ++l) {
        pgb_ctx* lc = c->lane_ctx[l];
        if (c->timing) {
            collect_timing(lc);
            for (int k = 0; k < PGB_N_STAGES; ++k) {
                c->stage_ms[k] += lc->stage_ms[k];
                c->stage_calls[k] += lc->stage_calls[k];
                lc->stage_ms[k] = 0;
                lc->stage_calls[k] = 0;
            }
        }
        c->launches += lc->launches;
        c->graph_kernels += lc->graph_kernels;
        c->graph_launches += lc->graph_launches;
        lc->launches = lc->graph_kernels = lc->graph_launches = 0;
    }
    for (int l = 0; l < L; ++l)
        if (rc[l] != PGB_OK && rc[l] != PGB_ENOCONV) {
            const int code = rc[l];
            const std::string m = msg[l];
            destroy_lanes(c);
            fail(code, "lane " + std::to_string(l) + ": " + m);
        }
    for (int l = 0; l < L; ++l)
        if (rc[l] == PGB_ENOCONV) out = PGB_ENOCONV;
    return out;
}

extern "C" {

int pgb_default_params(pgb_params* p) {
    if (!p) return PGB_EINVAL;
    p->K = 7;
    p->K_near = 19;
    p->n_edge = 9;
    p->P = 6;
    p->theta = 0.5;
    p->leaf_size = 32;
    p->group_size = 32;
    p->p2p_item = 64;
    p->m2p_item = 64;
    p->precond = 0;
    p->graphs = 2;
    p->lanes = 4;
    p->overlap = 0;
    p->batch = 1;
    p->residual = 1;
    return PGB_OK;
}

int pgb_create(pgb_ctx** out, const pgb_params* p, void* stream) {
    if (!out) return PGB_EINVAL;
    *out = nullptr;
    pgb_params q;
    pgb_default_params(&q);
    if (p) q = *p;
    std::string why;
    if (check_params(&q, why) != PGB_OK) return PGB_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return PGB_ECUDA;
    }
    {
        // temporaries are allocated in stream order from the device's default
        // pool: let the pool keep freed memory for reuse (this process only)
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        (void)cudaGetLastError();
    }
    pgb_ctx* c = new (std::nothrow) pgb_ctx;
    if (!c) return PGB_ENOMEM;
    if (q.p2p_item == 0) q.p2p_item = 64;
    if (q.lanes == 0) q.lanes = 4;
    if (q.m2p_item == 0) q.m2p_item = 64;
    if (q.batch == 0) q.batch = 1;
    c->p = q;
    c->stream = (cudaStream_t)stream;
    note_alloc();
    if (cudaMallocHost(&c->h_pinned, 64) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return PGB_ENOMEM;
    }
    *out = c;
    return PGB_OK;
}

int pgb_destroy(pgb_ctx* c) {
    if (!c) return PGB_EINVAL;
    destroy_lanes(c);
    destroy_union(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& p : c->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto& gr : c->up_graph)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (c->gm_graph.exec) cudaGraphExecDestroy(c->gm_graph.exec);
    if (c->seg_exec) cudaGraphExecDestroy(c->seg_exec);
    if (c->gm_stream) {
        cudaStreamSynchronize(c->gm_stream);
        cudaStreamDestroy(c->gm_stream);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int q = 0; q < 2; ++q) {
        if (c->up_stream[q]) {
            cudaStreamSynchronize(c->up_stream[q]);
            cudaStreamDestroy(c->up_stream[q]);
        }
        if (c->up_fork[q]) cudaEventDestroy(c->up_fork[q]);
        if (c->up_join[q]) cudaEventDestroy(c->up_join[q]);
    }
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->side_stream) cudaStreamSynchronize(c->side_stream);
    if (c->hp_stream) cudaStreamSynchronize(c->hp_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    cudaStream_t own = c->owns_stream ? c->stream : nullptr;
    cudaStream_t side = c->side_stream, hp = c->hp_stream;
    delete c;  // device buffers are freed in the order of the stream they were allocated on
    for (cudaStream_t x : {side, hp, own})
        if (x) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
    return PGB_OK;
}

const char* pgb_last_error(const pgb_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pgb_mesh_load(pgb_ctx* c, int32_t kind, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                  double eps_in, const double* charge_xyz, const double* charge_q, int64_t nq, double bc_value,
                  int32_t* body_id_out) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (kind != PGB_DIELECTRIC && kind != PGB_SET_CHARGE && kind != PGB_SET_POTENTIAL) fail(PGB_EINVAL, "bad kind");
        if (!verts || !tris || nv < 3 || nt < 1) fail(PGB_EINVAL, "empty mesh");
        if (nt > (int64_t)1 << 26) fail(PGB_EINVAL, "too many panels");
        if ((int)c->bodies.size() >= PGB_MAX_BODIES) fail(PGB_EINVAL, "too many bodies");
        if (nq < 0 || (nq > 0 && (!charge_xyz || !charge_q))) fail(PGB_EINVAL, "bad charges");
        if (kind != PGB_DIELECTRIC && nq != 0) fail(PGB_EINVAL, "surfaces carry no point charges");
        if (kind == PGB_DIELECTRIC && !(eps_in > 0 && isfinite(eps_in))) fail(PGB_EINVAL, "eps_in must be > 0");
        if (!isfinite(bc_value)) fail(PGB_EINVAL, "bc_value must be finite");
        Body b;
        b.kind = kind;
        b.eps_in = kind == PGB_DIELECTRIC ? eps_in : 1.0;
        b.N = nt;
        b.nv = nv;
        b.nq = nq;
        b.verts.assign(verts, verts + 3 * nv);
        b.tris.assign(tris, tris + 3 * nt);
        for (double v : b.verts)
            if (!isfinite(v)) fail(PGB_EINVAL, "non-finite vertex coordinate");
        for (int32_t t : b.tris)
            if (t < 0 || t >= nv) fail(PGB_EINVAL, "triangle index out of range");
        for (int64_t i = 0; i < nt; ++i) {
            const double* v0 = &b.verts[3 * b.tris[3 * i]];
            const double* v1 = &b.verts[3 * b.tris[3 * i + 1]];
            const double* v2 = &b.verts[3 * b.tris[3 * i + 2]];
            double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
            double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
            double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
            if (!(cx * cx + cy * cy + cz * cz > 0)) fail(PGB_EINVAL, "degenerate triangle " + std::to_string(i));
        }
        if (nq) {
            b.qxyz.assign(charge_xyz, charge_xyz + 3 * nq);
            b.qval.assign(charge_q, charge_q + nq);
            for (double v : b.qxyz)
                if (!isfinite(v)) fail(PGB_EINVAL, "non-finite charge position");
            for (double v : b.qval)
                if (!isfinite(v)) fail(PGB_EINVAL, "non-finite charge");
        }
        const double e = 1.602176634e-19, eps0 = 8.8541878128e-12;
        if (kind == PGB_SET_CHARGE) b.bc = bc_value * 1e-20 / e;          // C/m^2 -> e/A^2
        if (kind == PGB_SET_POTENTIAL) b.bc = bc_value * eps0 * 1e-10 / e;  // V -> e/(eps0 A)
        c->bodies.push_back(std::move(b));
        ++c->config_gen;
        c->tree_valid = false;
        c->order_valid = false;
        c->lists_valid = false;
        c->intra_valid = false;
        if (body_id_out) *body_id_out = (int32_t)c->bodies.size() - 1;
        return PGB_OK;
    });
}

int pgb_set_charges(pgb_ctx* c, int32_t id, const double* q, int64_t nq) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (id < 0 || id >= (int32_t)c->bodies.size()) fail(PGB_EINVAL, "bad body id");
        auto& b = c->bodies[id];
        if (b.kind != PGB_DIELECTRIC) fail(PGB_EINVAL, "only molecules carry charges");
        if (nq != b.nq || (nq && !q)) fail(PGB_EINVAL, "charge count differs from the loaded body");
        for (int64_t k = 0; k < nq; ++k)
            if (!isfinite(q[k])) fail(PGB_EINVAL, "non-finite charge");
        b.qval.assign(q, q + nq);
        ++c->config_gen;
        if (c->order_valid && nq)  // device copy exists: update it in place
            PGB_CUDA(cudaMemcpyAsync(c->d_qval.p + b.q_off, q, 8 * nq, cudaMemcpyHostToDevice, c->stream));
        PGB_CUDA(cudaStreamSynchronize(c->stream));
        return PGB_OK;
    });
}

int pgb_set_bc(pgb_ctx* c, int32_t id, double bc_value) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (id < 0 || id >= (int32_t)c->bodies.size()) fail(PGB_EINVAL, "bad body id");
        auto& b = c->bodies[id];
        if (b.kind == PGB_DIELECTRIC) fail(PGB_EINVAL, "molecules have no imposed boundary value");
        if (!isfinite(bc_value)) fail(PGB_EINVAL, "bc_value must be finite");
        const double e = 1.602176634e-19, eps0 = 8.8541878128e-12;
        b.bc = b.kind == PGB_SET_CHARGE ? bc_value * 1e-20 / e : bc_value * eps0 * 1e-10 / e;
        ++c->config_gen;
        return PGB_OK;
    });
}

int pgb_set_solvent(pgb_ctx* c, double eps_out, double kappa) {
    if (!c) return PGB_EINVAL;
    if (!(eps_out > 0 && isfinite(eps_out)) || !(kappa >= 0 && isfinite(kappa))) {
        c->err = "eps_out must be > 0 and kappa >= 0";
        return PGB_EINVAL;
    }
    if (kappa != c->kappa) c->intra_valid = false;
    ++c->config_gen;
    c->eps_out = eps_out;
    c->kappa = kappa;
    c->tree_valid = false;
    return PGB_OK;
}

int pgb_set_region(pgb_ctx* c, int32_t id, int32_t parent, double kappa_in) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        const int nb = (int)c->bodies.size();
        if (id < 0 || id >= nb) fail(PGB_EINVAL, "bad body id");
        if (parent < -1 || parent >= nb || parent == id) fail(PGB_EINVAL, "bad parent id");
        if (!(kappa_in >= 0 && isfinite(kappa_in))) fail(PGB_EINVAL, "kappa_in must be >= 0");
        auto& b = c->bodies[id];
        if (b.kind != PGB_DIELECTRIC && (parent >= 0 || kappa_in != 0))
            fail(PGB_EINVAL, "surfaces with an imposed value lie in the solvent");
        if (parent >= 0 && c->bodies[parent].kind != PGB_DIELECTRIC) fail(PGB_EINVAL, "a parent must be a dielectric body");
        if (kappa_in != 0 && b.nq > 0) fail(PGB_EINVAL, "a body with charges has an unscreened interior");
        for (int p = parent, steps = 0; p >= 0; p = c->bodies[p].parent)
            if (p == id || ++steps > nb) fail(PGB_EINVAL, "nesting would form a cycle");
        b.parent = parent;
        b.kappa_in = kappa_in;
        ++c->config_gen;
        c->tree_valid = false;
        return PGB_OK;
    });
}

int pgb_set_pose(pgb_ctx* c, int32_t id, const double R[9], const double t[3]) {
    if (!c) return PGB_EINVAL;
    if (id < 0 || id >= (int32_t)c->bodies.size() || !R || !t) {
        c->err = "bad body id or pose";
        return PGB_EINVAL;
    }
    const char* why = pose_error(R, t);
    if (why) {
        c->err = why;
        return PGB_EINVAL;
    }
    auto& b = c->bodies[id];
    memcpy(b.R, R, sizeof(b.R));
    memcpy(b.t, t, sizeof(b.t));
    c->tree_valid = false;
    return PGB_OK;
}

int pgb_tree_build(pgb_ctx* c) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (c->bodies.empty()) fail(PGB_ESTATE, "no bodies loaded");
        StageTimer tm(c, PGB_STAGE_TREE);
        if (!c->order_valid) {
            upload_bodies(c);
            build_order(c);
            c->intra_valid = false;
        }
        build_geometry(c);
        build_lists(c);
        build_corrections(c);
        c->tree_valid = true;
        return PGB_OK;
    });
}

int pgb_tree_refresh(pgb_ctx* c) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!c->order_valid || !c->lists_valid)
            fail(PGB_ESTATE, "pgb_tree_refresh needs a tree built by pgb_tree_build for the loaded bodies");
        StageTimer tm(c, PGB_STAGE_TREE);
        build_geometry(c);
        refresh_lists(c);
        build_corrections(c);
        c->tree_valid = true;
        return PGB_OK;
    });
}

int pgb_tree_reset(pgb_ctx* c) {
    if (!c) return PGB_EINVAL;
    c->order_valid = false;
    c->lists_valid = false;
    c->intra_valid = false;
    c->tree_valid = false;
    c->adj_valid = false;
    return PGB_OK;
}

int pgb_tree_stats(pgb_ctx* c, pgb_tree_info* info) {
    if (!c || !info) return PGB_EINVAL;
    if (!c->tree_valid) {
        c->err = "pgb_tree_build has not run";
        return PGB_ESTATE;
    }
    info->n_panels = c->n_pan;
    info->n_unknowns = c->n_unk;
    info->n_nodes = c->n_nodes;
    info->n_leaves = c->n_leaves;
    info->n_groups = c->n_groups;
    info->n_near = c->n_near;
    info->n_far = c->n_far;
    info->p2p_pairs = c->p2p_pairs;
    info->p2p_laplace_pairs = c->p2p_lap;
    info->m2p_pairs = c->m2p_pairs;
    info->m2p_laplace_pairs = c->m2p_lap;
    info->n_corrections = c->n_corr + c->n_xcorr;
    info->n_p2p_items = c->n_pitems;
    info->n_m2p_items = c->n_fitems;
    return PGB_OK;
}

int pgb_num_unknowns(pgb_ctx* c, int64_t* n) {
    if (!c || !n) return PGB_EINVAL;
    int64_t s = 0;
    for (auto& b : c->bodies) s += b.kind == PGB_DIELECTRIC ? 2 * b.N : b.N;
    *n = s;
    return PGB_OK;
}

int pgb_matvec(pgb_ctx* c, const void* x, void* y, int32_t precision) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!x || !y) fail(PGB_EINVAL, "null vector");
        if (precision != PGB_FP32 && precision != PGB_FP64 && precision != PGB_FP64_DS)
            fail(PGB_EINVAL, "precision must be PGB_FP32, PGB_FP64 or PGB_FP64_DS");
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run for the current bodies and poses");
        if (precision != PGB_FP32) {
            apply_operator(c, (const double*)x, (double*)y, precision, false);
        } else {
            c->d_xtmp.resize(c->n_unk);
            c->d_ytmp.resize(c->n_unk);
            convert_f32_f64((const float*)x, c->d_xtmp, c->n_unk, c->stream);
            apply_operator(c, c->d_xtmp, c->d_ytmp, PGB_FP32, false);
            convert_f64_f32(c->d_ytmp, (float*)y, c->n_unk, c->stream);
        }
        PGB_CUDA(cudaGetLastError());
        return PGB_OK;
    });
}

int pgb_rhs(pgb_ctx* c, double* b) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!b) fail(PGB_EINVAL, "null vector");
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        build_rhs(c, b, PGB_FP64);
        return PGB_OK;
    });
}

int pgb_solve(pgb_ctx* c, int32_t mode, double tol, int32_t max_iter, int32_t restart, double* x,
              pgb_solve_stats* st) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!x) fail(PGB_EINVAL, "null x_out");
        if (!(tol > 0 && tol < 1)) fail(PGB_EINVAL, "tol must be in (0, 1)");
        if (max_iter < 1 || restart < 1 || restart > 256) fail(PGB_EINVAL, "max_iter >= 1 and restart in 1..256");
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        int r = solve(c, mode, tol, max_iter, restart, x, st);
        PGB_CUDA(cudaStreamSynchronize(c->stream));
        if (r == PGB_ENOCONV) c->err = "GMRES did not reach tol";
        return r;
    });
}

int pgb_solve_batch(pgb_ctx* c, int32_t body_id, const double* R, const double* t, int64_t B, int32_t mode, double tol,
                    int32_t max_iter, int32_t restart, double* F_out, pgb_solve_stats* stats) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!R || !t || !F_out || B < 0) fail(PGB_EINVAL, "null argument or negative batch");
        if (body_id < 0 || body_id >= (int32_t)c->bodies.size()) fail(PGB_EINVAL, "bad body id");
        if (!(tol > 0 && tol < 1)) fail(PGB_EINVAL, "tol must be in (0, 1)");
        if (max_iter < 1 || restart < 1 || restart > 256) fail(PGB_EINVAL, "max_iter >= 1 and restart in 1..256");
        if (B == 0) return PGB_OK;
        const int L = c->p.batch > 1 ? 0 : (int)std::min<int64_t>(c->p.lanes, B);
        int first_err = PGB_OK;
        if (c->p.batch > 1) {
            pgb_ctx* self = c;
            first_err = solve_chunks(c, &self, nullptr, body_id, R, t, B, mode, tol, max_iter, restart, F_out, stats);
        } else if (L <= 1) {
            for (int64_t b = 0; b < B; ++b) {
                const int rs = solve_pose(c, body_id, b, R + 9 * b, t + 3 * b, mode, tol, max_iter, restart,
                                          F_out + 4 * b, stats ? stats + b : nullptr);
                if (rs != PGB_OK && first_err == PGB_OK) first_err = rs;
            }
        } else {
            first_err = solve_lanes(c, L, body_id, R, t, B, mode, tol, max_iter, restart, F_out, stats);
        }
        // the body keeps the last pose, with its tree built as after a serial batch
        if (L > 1 || c->p.batch > 1) {
            memcpy(c->bodies[body_id].R, R + 9 * (B - 1), 9 * sizeof(double));
            memcpy(c->bodies[body_id].t, t + 3 * (B - 1), 3 * sizeof(double));
            c->tree_valid = false;
            if (!c->order_valid) {
                upload_bodies(c);
                build_order(c);
                c->intra_valid = false;
            }
            build_geometry(c);
            build_lists(c);
            build_corrections(c);
            c->tree_valid = true;
        }
        PGB_CUDA(cudaStreamSynchronize(c->stream));
        if (first_err == PGB_ENOCONV) c->err = "GMRES did not reach tol for at least one pose";
        return first_err;
    });
}

int pgb_solve_poses(pgb_ctx* const* ctxs, int32_t n_ctx, const int32_t* pose_ctx, int32_t body_id, const double* R,
                    const double* t, int64_t B, int32_t mode, double tol, int32_t max_iter, int32_t restart,
                    double* F_out, pgb_solve_stats* stats) {
    if (!ctxs || n_ctx < 1 || !ctxs[0]) return PGB_EINVAL;
    pgb_ctx* c = ctxs[0];
    return guard(c, [&]() -> int {
        if (!R || !t || !F_out || !pose_ctx || B < 0) fail(PGB_EINVAL, "null argument or negative batch");
        for (int32_t k = 0; k < n_ctx; ++k) {
            if (!ctxs[k]) fail(PGB_EINVAL, "null context " + std::to_string(k));
            if (body_id < 0 || body_id >= (int32_t)ctxs[k]->bodies.size())
                fail(PGB_EINVAL, "bad body id for context " + std::to_string(k));
        }
        for (int64_t b = 0; b < B; ++b)
            if (pose_ctx[b] < 0 || pose_ctx[b] >= n_ctx) fail(PGB_EINVAL, "pose_ctx out of range at " + std::to_string(b));
        if (!(tol > 0 && tol < 1)) fail(PGB_EINVAL, "tol must be in (0, 1)");
        if (max_iter < 1 || restart < 1 || restart > 256) fail(PGB_EINVAL, "max_iter >= 1 and restart in 1..256");
        if (B == 0) return PGB_OK;
        const int r = solve_chunks(c, ctxs, pose_ctx, body_id, R, t, B, mode, tol, max_iter, restart, F_out, stats);
        if (r == PGB_ENOCONV) c->err = "GMRES did not reach tol for at least one pose";
        return r;
    });
}

int pgb_grad(pgb_ctx* c, const double* x, int32_t precision, double tol, int32_t max_iter, int32_t restart,
             double* dq, double* dbc, double* dt, pgb_solve_stats* adj) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!x) fail(PGB_EINVAL, "null x");
        if (!(tol > 0 && tol < 1)) fail(PGB_EINVAL, "tol must be in (0, 1)");
        if (max_iter < 1 || restart < 1 || restart > 256) fail(PGB_EINVAL, "max_iter >= 1 and restart in 1..256");
        if (nested(c)) fail(PGB_EINVAL, "gradients are not available with nested interfaces");
        if (c->p.P > 8) fail(PGB_EINVAL, "adjoint gradients take P in 0..8");
        pgb_solve_stats st{};
        grad(c, x, precision, tol, max_iter, restart, dq, dbc, dt, &st);
        if (adj) *adj = st;
        if (st.rel_residual > tol) {
            c->err = "adjoint GMRES did not reach tol";
            return PGB_ENOCONV;
        }
        return PGB_OK;
    });
}

int pgb_matvec_transpose(pgb_ctx* c, const double* lam, double* y, int32_t precision) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!lam || !y) fail(PGB_EINVAL, "null vector");
        if (precision != PGB_FP32 && precision != PGB_FP64) fail(PGB_EINVAL, "precision must be PGB_FP32 or PGB_FP64");
        if (nested(c)) fail(PGB_EINVAL, "the transposed operator is not available with nested interfaces");
        apply_transpose(c, lam, y, precision);
        PGB_CUDA(cudaGetLastError());
        return PGB_OK;
    });
}

int pgb_energy(pgb_ctx* c, const double* x, pgb_energies* e, pgb_energies* per_body) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!x || !e) fail(PGB_EINVAL, "null argument");
        {
            StageTimer tm(c, PGB_STAGE_ENERGY);
            energies(c, x, e, per_body);
        }
        return PGB_OK;
    });
}

int pgb_energy_noalloc(pgb_ctx* c, const double* x, pgb_energies* e) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!x || !e) fail(PGB_EINVAL, "null argument");
        if (nested(c)) fail(PGB_EINVAL, "pgb_energy_noalloc does not take nested interfaces (use pgb_energy)");
        energies_noalloc(c, x, e);
        return PGB_OK;
    });
}

int pgb_autotune(pgb_ctx* c, const double* thetas, int32_t n_theta, const int32_t* Ps, int32_t n_P,
                 const int32_t* leaves, int32_t n_leaf, int32_t reps, double tol, double target, pgb_params* chosen,
                 double* report) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!thetas || !Ps || !leaves || n_theta < 1 || n_P < 1 || n_leaf < 1 || reps < 1)
            fail(PGB_EINVAL, "empty candidate list");
        if (!(tol > 0 && tol < 1) || !(target > 0)) fail(PGB_EINVAL, "tol in (0,1) and target > 0");
        if (c->bodies.empty()) fail(PGB_ESTATE, "no bodies loaded");
        const pgb_params base = c->p;
        struct Cand {
            pgb_params p;
            double mv_ms, solve_ms, E;
        };
        std::vector<Cand> cands;
        for (int it = 0; it < n_theta; ++it)
            for (int ip = 0; ip < n_P; ++ip)
                for (int il = 0; il < n_leaf; ++il) {
                    pgb_params q = base;
                    q.theta = thetas[it];
                    q.P = Ps[ip];
                    q.leaf_size = leaves[il];
                    std::string why;
                    if (check_params(&q, why) != PGB_OK) fail(PGB_EINVAL, "bad candidate: " + why);
                    cands.push_back({q, 0, 0, 0});
                }
        int ref = 0;
        for (size_t k = 1; k < cands.size(); ++k) {
            const auto &a = cands[k].p, &b = cands[ref].p;
            if (a.theta < b.theta || (a.theta == b.theta && a.P > b.P)) ref = (int)k;
        }
        cudaEvent_t e0, e1;
        PGB_CUDA(cudaEventCreate(&e0));
        PGB_CUDA(cudaEventCreate(&e1));
        DBuf<double> x, y;
        for (auto& cd : cands) {
            const bool tree_changes = cd.p.leaf_size != c->p.leaf_size;
            c->p = cd.p;
            if (tree_changes) c->order_valid = false;
            if (tree_changes) c->lists_valid = false;
            c->tree_valid = false;
            PGB_CUDA(cudaEventRecord(e0, c->stream));
            int r = pgb_tree_build(c);
            if (r != PGB_OK) fail(r, c->err);
            x.resize(c->n_unk);
            y.resize(c->n_unk);
            pgb_solve_stats st{};
            r = solve(c, PGB_FP32_REFINE, tol, 5000, 100, x, &st);  // the refinement residual counts too
            if (r != PGB_OK && r != PGB_ENOCONV) fail(r, c->err);
            PGB_CUDA(cudaEventRecord(e1, c->stream));
            PGB_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            PGB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            cd.solve_ms = ms;
            pgb_energies en{};
            energies(c, x, &en, nullptr);
            cd.E = en.total;
            apply_operator(c, x, y, PGB_FP32, false);  // warm
            PGB_CUDA(cudaEventRecord(e0, c->stream));
            for (int k = 0; k < reps; ++k) apply_operator(c, x, y, PGB_FP32, false);
            PGB_CUDA(cudaEventRecord(e1, c->stream));
            PGB_CUDA(cudaEventSynchronize(e1));
            PGB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            cd.mv_ms = ms / reps;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double Eref = cands[ref].E;
        int best = ref;
        for (size_t k = 0; k < cands.size(); ++k) {
            const double err = fabs(cands[k].E - Eref) / std::max(fabs(Eref), 1e-300);
            if (report) {
                report[3 * k] = cands[k].mv_ms;
                report[3 * k + 1] = cands[k].solve_ms;
                report[3 * k + 2] = err;
            }
            if (err <= target && cands[k].solve_ms < cands[best].solve_ms) best = (int)k;
        }
        const bool tree_changes = cands[best].p.leaf_size != c->p.leaf_size;
        c->p = cands[best].p;
        if (tree_changes) c->order_valid = false;
        if (tree_changes) c->lists_valid = false;
        c->tree_valid = false;
        int r = pgb_tree_build(c);
        if (r != PGB_OK) fail(r, c->err);
        // then the work-item sizes (the product does not depend on them): each
        // of p2p_item and m2p_item in turn from {16, 32, 64, 128}, by the FP32
        // product time with the chosen parameters
        PGB_CUDA(cudaEventCreate(&e0));
        PGB_CUDA(cudaEventCreate(&e1));
        for (int which = 0; which < 2; ++which) {
            const int32_t keep = which ? c->p.m2p_item : c->p.p2p_item;
            int32_t best_item = keep;
            float best_ms = INFINITY;
            for (int32_t item : {16, 32, 64, 128}) {
                (which ? c->p.m2p_item : c->p.p2p_item) = item;
                c->tree_valid = false;
                r = pgb_tree_build(c);
                if (r != PGB_OK) fail(r, c->err);
                apply_operator(c, x, y, PGB_FP32, false);  // warm
                PGB_CUDA(cudaEventRecord(e0, c->stream));
                for (int k = 0; k < reps; ++k) apply_operator(c, x, y, PGB_FP32, false);
                PGB_CUDA(cudaEventRecord(e1, c->stream));
                PGB_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                PGB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best_item = item;
                }
            }
            (which ? c->p.m2p_item : c->p.p2p_item) = best_item;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->tree_valid = false;
        r = pgb_tree_build(c);
        if (r != PGB_OK) fail(r, c->err);
        if (chosen) *chosen = c->p;
        return PGB_OK;
    });
}

int pgb_timing(pgb_ctx* c, int32_t enable, pgb_stage_times* out) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (out) {
            collect_timing(c);
            for (int i = 0; i < PGB_N_STAGES; ++i) {
                out->ms[i] = c->stage_ms[i];
                out->calls[i] = c->stage_calls[i];
                c->stage_ms[i] = 0;
                c->stage_calls[i] = 0;
            }
            out->kernel_launches = c->launches;
            out->host_launches = c->launches - c->graph_kernels + c->graph_launches;
            c->launches = c->graph_kernels = c->graph_launches = 0;
        }
        c->timing = enable != 0;
        return PGB_OK;
    });
}

int pgb_tree_export(pgb_ctx* c, int32_t* perm, int64_t* near_off, int32_t* near_node, int64_t* far_off,
                    int32_t* far_node) {
    if (!c) return PGB_EINVAL;
    return guard(c, [&]() -> int {
        if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
        cudaStream_t s = c->stream;
        if (perm) PGB_CUDA(cudaMemcpyAsync(perm, c->d_perm.p, 4 * c->n_pan, cudaMemcpyDeviceToHost, s));
        if (near_off) PGB_CUDA(cudaMemcpyAsync(near_off, c->d_near_off.p, 8 * (c->n_groups + 1), cudaMemcpyDeviceToHost, s));
        if (far_off) PGB_CUDA(cudaMemcpyAsync(far_off, c->d_far_off.p, 8 * (c->n_groups + 1), cudaMemcpyDeviceToHost, s));
        if (near_node && c->n_near) PGB_CUDA(cudaMemcpyAsync(near_node, c->d_near.p, 4 * c->n_near, cudaMemcpyDeviceToHost, s));
        if (far_node && c->n_far) PGB_CUDA(cudaMemcpyAsync(far_node, c->d_far.p, 4 * c->n_far, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        return PGB_OK;
    });
}

int pgb_math_check(const double* x, int64_t n, double* out) {
    if (n < 0 || (n > 0 && (!x || !out))) return PGB_EINVAL;
    if (n == 0) return PGB_OK;
    double *dx = nullptr, *dy = nullptr;
    int rc = PGB_OK;
    pgb::note_alloc();
    pgb::note_alloc();
    if (cudaMalloc(&dx, 8 * n) != cudaSuccess || cudaMalloc(&dy, 56 * n) != cudaSuccess) rc = PGB_ECUDA;
    if (rc == PGB_OK && cudaMemcpy(dx, x, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = PGB_ECUDA;
    if (rc == PGB_OK) {
        pgb::k_math_check<<<(unsigned)((n + 255) / 256), 256>>>(n, dx, dy);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, dy, 56 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = PGB_ECUDA;
    }
    if (rc != PGB_OK) (void)cudaGetLastError();
    cudaFree(dx);
    cudaFree(dy);
    return rc;
}

int pgb_orientation_landscape(const double* F, int32_t n_orient, int32_t n_gap, double temperature, double* out) {
    if (!F || !out || n_orient < 1 || n_gap < 1 || !(temperature > 0) || !isfinite(temperature)) return PGB_EINVAL;
    for (int64_t k = 0; k < (int64_t)n_orient * n_gap; ++k)
        if (!isfinite(F[k])) return PGB_EINVAL;
    const double kT = 0.0019872043 * temperature;  // Boltzmann constant in kcal/(mol K)
    for (int gi = 0; gi < n_gap; ++gi) {
        double fmin = INFINITY;
        int best = 0;
        for (int o = 0; o < n_orient; ++o) {
            const double f = F[(int64_t)o * n_gap + gi];
            if (f < fmin) {
                fmin = f;
                best = o;
            }
        }
        // weights relative to the lowest energy (no overflow), summed in orientation order
        double z = 0;
        for (int o = 0; o < n_orient; ++o) z += exp(-(F[(int64_t)o * n_gap + gi] - fmin) / kT);
        out[3 * gi] = best;
        out[3 * gi + 1] = 1.0 / z;
        out[3 * gi + 2] = fmin - kT * log(z / n_orient);
    }
    return PGB_OK;
}

int pgb_alloc_count(int64_t* n) {
    if (!n) return PGB_EINVAL;
    *n = pgb::g_alloc_count.load(std::memory_order_relaxed);
    return PGB_OK;
}

}  // extern "C"
