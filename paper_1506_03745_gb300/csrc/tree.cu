// Geometry, Morton ordering, octree, target groups, interaction lists and
// near-field corrections (Sections 3.1 and 3.2 of the paper).
#include <math.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "ds.cuh"
#include "pgb_internal.cuh"

namespace pgb {

Rules make_rules(int K, int Kn, int ne) {
    Rules r;
    memset(&r, 0, sizeof(r));
    r.K = K;
    r.Kn = Kn;
    r.ne = ne;
    const double(*mu)[3] = nullptr;
    const double* w = nullptr;
    switch (K) {
        case 1: mu = PGB_TRI1_MU; w = PGB_TRI1_W; break;
        case 3: mu = PGB_TRI3_MU; w = PGB_TRI3_W; break;
        case 4: mu = PGB_TRI4_MU; w = PGB_TRI4_W; break;
        case 7: mu = PGB_TRI7_MU; w = PGB_TRI7_W; break;
        default: fail(PGB_EINVAL, "K must be 1, 3, 4 or 7");
    }
    for (int i = 0; i < K; ++i) {
        for (int a = 0; a < 3; ++a) r.mu[i][a] = mu[i][a];
        r.w[i] = w[i];
    }
    const double(*mun)[3] = nullptr;
    const double* wn = nullptr;
    switch (Kn) {
        case 19: mun = PGB_TRI19_MU; wn = PGB_TRI19_W; break;
        case 37: mun = PGB_TRI37_MU; wn = PGB_TRI37_W; break;
        default: fail(PGB_EINVAL, "K_near must be 19 or 37");
    }
    for (int i = 0; i < Kn; ++i) {
        for (int a = 0; a < 3; ++a) r.mun[i][a] = mun[i][a];
        r.wn[i] = wn[i];
    }
    const double *ex = nullptr, *ew = nullptr;
    switch (ne) {
        case 3: ex = PGB_GL3_X; ew = PGB_GL3_W; break;
        case 6: ex = PGB_GL6_X; ew = PGB_GL6_W; break;
        case 9: ex = PGB_GL9_X; ew = PGB_GL9_W; break;
        case 12: ex = PGB_GL12_X; ew = PGB_GL12_W; break;
        default: fail(PGB_EINVAL, "n_edge must be 3, 6, 9 or 12");
    }
    for (int i = 0; i < ne; ++i) {
        r.ex[i] = ex[i];
        r.ew[i] = ew[i];
    }
    return r;
}

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------- scan
// Exclusive scan of n int64 values by one block: each thread scans a
// contiguous chunk, the chunk totals are scanned across the block.
__global__ void k_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total) {
    __shared__ int64_t sh[1024];
    int t = threadIdx.x;
    int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    int64_t b = t * chunk, e = min(n, b + chunk);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    sh[t] = s;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        int64_t v = (t >= off) ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int64_t run = sh[t] - s;
    for (int64_t i = b; i < e; ++i) {
        int64_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (t == blockDim.x - 1) *total = sh[t];
}

// Exclusive scan of long arrays over many blocks: each block of SCAN_T
// threads takes SCAN_CHUNK consecutive values; k_scan_part sums every chunk,
// the chunk sums are scanned by k_scan_i64, and k_scan_chunk scans each chunk
// in shared memory from its offset.  (Integer sums: the same result as the
// one-block scan.)
#define SCAN_T 256
#define SCAN_PER 16
#define SCAN_CHUNK (SCAN_T * SCAN_PER)
__global__ void __launch_bounds__(SCAN_T) k_scan_part(const int64_t* __restrict__ in, int64_t n, int64_t* part) {
    __shared__ int64_t sh[SCAN_T / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CHUNK;
    int64_t t = 0;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += SCAN_T)
        if (b0 + k < n) t += in[b0 + k];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t u = 0;
        for (int w = 0; w < SCAN_T / 32; ++w) u += sh[w];
        part[blockIdx.x] = u;
    }
}
__global__ void __launch_bounds__(SCAN_T) k_scan_chunk(const int64_t* __restrict__ in, int64_t* out, int64_t n,
                                                       const int64_t* __restrict__ poff) {
    __shared__ int64_t v[SCAN_CHUNK];
    __shared__ int64_t wsum[SCAN_T / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CHUNK;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += SCAN_T) v[k] = b0 + k < n ? in[b0 + k] : 0;
    __syncthreads();
    // each thread its SCAN_PER consecutive values, then the threads' totals
    int64_t own = 0;
    for (int q = 0; q < SCAN_PER; ++q) own += v[threadIdx.x * SCAN_PER + q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = own;  // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int64_t before = poff[blockIdx.x] + inc - own;
    for (int k = 0; k < w; ++k) before += wsum[k];
    __syncthreads();
    for (int q = 0; q < SCAN_PER; ++q) {
        const int idx = threadIdx.x * SCAN_PER + q;
        const int64_t x = v[idx];
        v[idx] = before;
        before += x;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += SCAN_T)
        if (b0 + k < n) out[b0 + k] = v[k];
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    // one total slot per host thread, outside any stream order, freed when the thread ends
    struct Slot {
        int64_t* p = nullptr;
        ~Slot() {
            if (p) cudaFree(p);
        }
    };
    static thread_local Slot slot;
    if (!slot.p) {
        note_alloc();
        PGB_CUDA(cudaMalloc(&slot.p, sizeof(int64_t)));
    }
    int64_t* tot = slot.p;
    if (n > 4 * SCAN_CHUNK) {
        const int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
        DBuf<int64_t> part, poff;
        part.resize(nb);
        poff.resize(nb);
        k_scan_part<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, part);
        k_scan_i64<<<1, 1024, 0, s>>>(part, poff, nb, tot);
        k_scan_chunk<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, poff);
    } else {
        k_scan_i64<<<1, 1024, 0, s>>>(in, out, n, tot);
    }
    PGB_CUDA(cudaGetLastError());
    if (total_host) {
        PGB_CUDA(cudaMemcpyAsync(total_host, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
    }
}

// ---------------------------------------------------------------- upload
void upload_bodies(pgb_ctx* c) {
    int64_t np = 0, nv = 0, nq = 0, nu = 0;
    for (auto& b : c->bodies) {
        b.pan_off = np;
        b.v_off = nv;
        b.q_off = nq;
        b.unk_off = nu;
        np += b.N;
        nv += b.nv;
        nq += b.nq;
        nu += (b.kind == PGB_DIELECTRIC) ? 2 * b.N : b.N;
    }
    c->n_pan = np;
    c->n_verts = nv;
    c->n_q = nq;
    c->n_unk = nu;
    std::vector<double> vb(3 * nv), qb(3 * nq), qv(nq), pose(12 * c->bodies.size());
    std::vector<int32_t> tr(3 * np), pb(np), qbody(nq);
    for (size_t bi = 0; bi < c->bodies.size(); ++bi) {
        auto& b = c->bodies[bi];
        std::copy(b.verts.begin(), b.verts.end(), vb.begin() + 3 * b.v_off);
        for (int64_t i = 0; i < 3 * b.N; ++i) tr[3 * b.pan_off + i] = b.tris[i] + (int32_t)b.v_off;
        for (int64_t i = 0; i < b.N; ++i) pb[b.pan_off + i] = (int32_t)bi;
        std::copy(b.qxyz.begin(), b.qxyz.end(), qb.begin() + 3 * b.q_off);
        std::copy(b.qval.begin(), b.qval.end(), qv.begin() + b.q_off);
        for (int64_t i = 0; i < b.nq; ++i) qbody[b.q_off + i] = (int32_t)bi;
        for (int a = 0; a < 9; ++a) pose[12 * bi + a] = b.R[a];
        for (int a = 0; a < 3; ++a) pose[12 * bi + 9 + a] = b.t[a];
    }
    cudaStream_t s = c->stream;
    c->d_vb.resize(vb.size());
    c->d_tris.resize(tr.size());
    c->d_pan_body.resize(np);
    c->d_qxyz_body.resize(qb.size());
    c->d_qval.resize(qv.size());
    c->d_q_body.resize(qbody.size());
    c->d_qxyz.resize(qb.size());
    c->d_pose.resize(pose.size());
    PGB_CUDA(cudaMemcpyAsync(c->d_vb.p, vb.data(), vb.size() * 8, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(c->d_tris.p, tr.data(), tr.size() * 4, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(c->d_pan_body.p, pb.data(), pb.size() * 4, cudaMemcpyHostToDevice, s));
    if (nq) {
        PGB_CUDA(cudaMemcpyAsync(c->d_qxyz_body.p, qb.data(), qb.size() * 8, cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(c->d_qval.p, qv.data(), qv.size() * 8, cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(c->d_q_body.p, qbody.data(), qbody.size() * 4, cudaMemcpyHostToDevice, s));
    }
    PGB_CUDA(cudaMemcpyAsync(c->d_pose.p, pose.data(), pose.size() * 8, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- ordering
// Body-frame centroids ((v0 + v1) + v2) / 3, evaluated without fused products.
__global__ void k_body_centroids(const double* vb, const int32_t* tris, int64_t n, double* cen) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* v0 = vb + 3 * (int64_t)tris[3 * i];
    const double* v1 = vb + 3 * (int64_t)tris[3 * i + 1];
    const double* v2 = vb + 3 * (int64_t)tris[3 * i + 2];
    for (int a = 0; a < 3; ++a) cen[3 * i + a] = __ddiv_rn(dadd(dadd(v0[a], v1[a]), v2[a]), 3.0);
}

// Per body min/max of the centroids (one block per body).
__global__ void k_bbox(const double* cen, const int64_t* off, double* out) {
    __shared__ double sh[6][32];
    int b = blockIdx.x;
    int64_t s = off[b], e = off[b + 1];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], cen[3 * i + a]);
            hi[a] = fmax(hi[a], cen[3 * i + a]);
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            sh[a][w] = lo[a];
            sh[3 + a][w] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x / 32;
        for (int k = 1; k < nw; ++k)
            for (int a = 0; a < 3; ++a) {
                sh[a][0] = fmin(sh[a][0], sh[a][k]);
                sh[3 + a][0] = fmax(sh[3 + a][0], sh[3 + a][k]);
            }
        for (int a = 0; a < 6; ++a) out[6 * b + a] = sh[a][0];
    }
}

struct BodyFrame {
    double lo[PGB_MAX_BODIES][3];
    double scale[PGB_MAX_BODIES];  // 1024 / ext
};

// 30-bit Morton key of the 10-bit cell q = floor((c - lo) * (1024/ext)),
// x bit highest in each triple; the body index goes above bit 30 so one sort
// orders all bodies.
__global__ void k_morton(const double* cen, const int32_t* pbody, int64_t n, BodyFrame f,
                         uint64_t* key, int32_t* idx, int32_t* qc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = pbody[i];
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        double u = dmul(dsub(cen[3 * i + a], f.lo[b][a]), f.scale[b]);
        double fl = floor(u);
        int v = (int)fl;
        v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
        q[a] = (uint32_t)v;
        qc[3 * i + a] = v;
    }
    uint64_t k = 0;
    for (int bit = 0; bit < 10; ++bit) {
        k |= (uint64_t)((q[0] >> bit) & 1u) << (3 * bit + 2);
        k |= (uint64_t)((q[1] >> bit) & 1u) << (3 * bit + 1);
        k |= (uint64_t)((q[2] >> bit) & 1u) << (3 * bit);
    }
    key[i] = k | ((uint64_t)b << 30);
    idx[i] = (int32_t)i;
}

// Stable LSD radix sort, 4 bits per pass.  Tiles of 1024 elements.
#define RS_TILE 1024
__global__ void k_rs_hist(const uint64_t* key, int64_t n, int shift, int64_t* hist, int ntiles) {
    __shared__ int cnt[16];
    if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        int64_t g = base + i;
        if (g < n) atomicAdd(&cnt[(key[g] >> shift) & 15], 1);
    }
    __syncthreads();
    if (threadIdx.x < 16) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one 4-bit pass: thread t owns the tile's items 4t..4t+3;
// its offset for digit d = tile base of d + number of d-items held by the
// threads before it (per-digit exclusive scan over the block) + its own
// earlier d-items.
__global__ void __launch_bounds__(256) k_rs_scatter(const uint64_t* key, const int32_t* val, int64_t n, int shift,
                                                    const int64_t* off, int ntiles, uint64_t* okey, int32_t* oval) {
    __shared__ int cnt[16][256];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + 4 * t;
    uint64_t k[4];
    int32_t v[4];
    int d[4];
    int mine[16];
    for (int q = 0; q < 16; ++q) mine[q] = 0;
    for (int q = 0; q < 4; ++q) {
        const int64_t g = base + q;
        if (g < n) {
            k[q] = key[g];
            v[q] = val[g];
            d[q] = (int)((k[q] >> shift) & 15);
        } else {
            d[q] = -1;
        }
    }
    for (int q = 0; q < 16; ++q) {
        int c = 0;
        for (int r = 0; r < 4; ++r) c += d[r] == q;
        cnt[q][t] = c;
    }
    __syncthreads();
    // exclusive scan of every digit row: warp w scans rows 2w and 2w+1, each
    // lane holding 8 consecutive entries
    const int w = t >> 5, lane = t & 31;
    for (int row = 2 * w; row < 2 * w + 2; ++row) {
        int loc[8], s = 0;
        for (int e = 0; e < 8; ++e) {
            loc[e] = s;
            s += cnt[row][8 * lane + e];
        }
        int inc = s;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int excl = inc - s;
        for (int e = 0; e < 8; ++e) cnt[row][8 * lane + e] = excl + loc[e];
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        if (d[q] < 0) continue;
        const int64_t pos = off[(int64_t)d[q] * ntiles + blockIdx.x] + cnt[d[q]][t] + mine[d[q]];
        ++mine[d[q]];
        okey[pos] = k[q];
        oval[pos] = v[q];
    }
}

__global__ void k_gather_i32x3(const int32_t* src, const int32_t* perm, int64_t n, int32_t* dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int a = 0; a < 3; ++a) dst[3 * i + a] = src[3 * j + a];
}

__global__ void k_invert(const int32_t* perm, int64_t n, int32_t* inv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) inv[perm[i]] = (int32_t)i;
}

__global__ void k_key30(const uint64_t* k64, int64_t n, uint32_t* k32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) k32[i] = (uint32_t)(k64[i] & 0x3fffffffull);
}

// Octree in one pass.  A node at depth l with more than leaf_size panels
// splits into its non-empty octants, depth limited to 10.  With the panels in
// key order the cells of a level are runs of equal key prefixes within a
// body, and the counts only shrink going down, so a level-l cell (l >= 1) is
// a node exactly when its parent cell holds more than leaf_size panels (its
// ancestors then hold more too).  Every (level, panel) pair is tested at once
// and one scan numbers the nodes level by level in key order.
#define OCT_LEVELS 11  // levels 0 (a body's root) .. 10

// body of sorted panel i (bodies are contiguous ranges off[b] .. off[b+1])
__device__ __forceinline__ int sorted_body(const int64_t* off, int nb, int64_t i) {
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (off[m] <= i) lo = m;
        else hi = m;
    }
    return lo;
}
// first j in [s, e) with (key[j] >> sh) >= p (keys ascending within a body)
__device__ __forceinline__ int64_t key_lower(const uint32_t* key, int64_t s, int64_t e, int sh, uint64_t p) {
    while (s < e) {
        const int64_t m = (s + e) >> 1;
        if ((uint64_t)(key[m] >> sh) < p) s = m + 1;
        else e = m;
    }
    return s;
}

// M[l n + i] = 1 when sorted panel i starts a node of level l; M[11 n] = 0
// (the scan's total lands after it).
__global__ void k_oct_marks(const uint32_t* key, const int64_t* off, int nb, int64_t n, int leaf_size, int64_t* M) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > OCT_LEVELS * n) return;
    if (t == OCT_LEVELS * n) {
        M[t] = 0;
        return;
    }
    const int l = (int)(t / n);
    const int64_t i = t - l * n;
    const int b = sorted_body(off, nb, i);
    const bool body_first = i == off[b];
    int64_t m = 0;
    if (l == 0) {
        m = body_first;
    } else {
        const int sh = 3 * (10 - l);
        if (body_first || (key[i] >> sh) != (key[i - 1] >> sh)) {
            const int ps = sh + 3;  // the parent's level
            const uint64_t pp = key[i] >> ps;
            const int64_t a = key_lower(key, off[b], off[b + 1], ps, pp);
            const int64_t e = key_lower(key, off[b], off[b + 1], ps, pp + 1);
            m = (e - a) > leaf_size;
        }
    }
    M[t] = m;
}

// Node S[t] of every mark t = l n + i: its panel range, body, level and
// children (the level-(l+1) nodes that start inside its range).
__global__ void k_oct_nodes(const uint32_t* key, const int64_t* off, int nb, int64_t n, const int64_t* M,
                            const int64_t* S, int32_t* nstart, int32_t* nend, int32_t* nbody, int32_t* nlevel,
                            int32_t* first_child, int32_t* nch) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= OCT_LEVELS * n || !M[t]) return;
    const int l = (int)(t / n);
    const int64_t i = t - l * n;
    const int b = sorted_body(off, nb, i);
    const int sh = 3 * (10 - l);
    const int64_t end = l == 0 ? off[b + 1] : key_lower(key, i, off[b + 1], sh, (uint64_t)(key[i] >> sh) + 1);
    const int64_t id = S[t];
    nstart[id] = (int32_t)i;
    nend[id] = (int32_t)end;
    nbody[id] = b;
    nlevel[id] = l;
    int64_t c0 = 0, c1 = 0;
    if (l < OCT_LEVELS - 1) {
        c0 = S[(int64_t)(l + 1) * n + i];
        c1 = S[(int64_t)(l + 1) * n + end];
    }
    nch[id] = (int32_t)(c1 - c0);
    first_child[id] = c1 > c0 ? (int32_t)c0 : -1;
}

// the first node id of every level (lb[l] = S[l n], lb[11] = the total)
__global__ void k_oct_levels(const int64_t* S, int64_t n, int64_t* lb) {
    const int l = threadIdx.x;
    if (l <= OCT_LEVELS) lb[l] = S[(int64_t)l * n];
}

__global__ void k_parents(const int32_t* child, const int32_t* nch, int64_t n, int32_t* parent) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nch[i]; ++k) parent[child[i] + k] = (int32_t)i;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// leaves in key order: mark leaf starts over panels, scan gives leaf index.
__global__ void k_mark_leaves(const int32_t* start, const int32_t* nch, int64_t n, int64_t* mark) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && nch[i] == 0) mark[start[i]] = 1;
}
__global__ void k_leaf_ids(const int32_t* start, const int32_t* end, const int32_t* nch, int64_t n,
                           const int64_t* lscan, int64_t n_pan, int64_t n_leaves, int32_t* leaf0, int32_t* leaf1,
                           int32_t* leaf_node) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = start[i], e = end[i];
    leaf0[i] = (int32_t)lscan[s];
    leaf1[i] = (int32_t)(e < n_pan ? lscan[e] : n_leaves);
    if (nch[i] == 0) leaf_node[lscan[s]] = (int32_t)i;
}
__global__ void k_pan_leaf(const int32_t* leaf_node, const int32_t* start, const int32_t* end, int64_t nl,
                           int32_t* pan_leaf) {
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= nl) return;
    int nd = leaf_node[l];
    for (int64_t p = start[nd]; p < end[nd]; ++p) pan_leaf[p] = (int32_t)l;
}

void build_order(pgb_ctx* c) {
    ++c->tree_gen;  // node structure and level ranges change: recapture graphs
    cudaStream_t s = c->stream;
    int64_t n = c->n_pan;
    int nb = (int)c->bodies.size();
    DBuf<double> cen;
    cen.resize(3 * n);
    k_body_centroids<<<nblk(n, 256), 256, 0, s>>>(c->d_vb, c->d_tris, n, cen);
    PGB_CUDA(cudaGetLastError());
    std::vector<int64_t> off(nb + 1);
    for (int b = 0; b < nb; ++b) off[b] = c->bodies[b].pan_off;
    off[nb] = n;
    DBuf<int64_t> d_off;
    d_off.resize(nb + 1);
    DBuf<double> d_bb;
    d_bb.resize(6 * nb);
    PGB_CUDA(cudaMemcpyAsync(d_off.p, off.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    k_bbox<<<nb, 256, 0, s>>>(cen, d_off, d_bb);
    PGB_CUDA(cudaGetLastError());
    std::vector<double> bb(6 * nb);
    PGB_CUDA(cudaMemcpyAsync(bb.data(), d_bb.p, 8 * 6 * nb, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    BodyFrame f;
    for (int b = 0; b < nb; ++b) {
        double ext = 0;
        for (int a = 0; a < 3; ++a) ext = std::max(ext, bb[6 * b + 3 + a] - bb[6 * b + a]);
        if (!(ext > 0)) ext = 1.0;
        c->bodies[b].ext = ext;
        for (int a = 0; a < 3; ++a) c->bodies[b].lo[a] = f.lo[b][a] = bb[6 * b + a];
        f.scale[b] = 1024.0 / ext;
    }
    DBuf<uint64_t> k0, k1;
    DBuf<int32_t> v0, v1, qc;
    k0.resize(n); k1.resize(n); v0.resize(n); v1.resize(n); qc.resize(3 * n);
    k_morton<<<nblk(n, 256), 256, 0, s>>>(cen, c->d_pan_body, n, f, k0, v0, qc);
    PGB_CUDA(cudaGetLastError());
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    DBuf<int64_t> hist, hoff;
    hist.resize(16 * (int64_t)ntiles);
    hoff.resize(16 * (int64_t)ntiles);
    int top = 30;
    while ((1 << (top - 30)) < nb) ++top;  // bits needed for the body index
    uint64_t *ka = k0.p, *kb = k1.p;
    int32_t *va = v0.p, *vb = v1.p;
    for (int shift = 0; shift < top; shift += 4) {
        k_rs_hist<<<ntiles, 256, 0, s>>>(ka, n, shift, hist, ntiles);
        exclusive_scan_i64(hist, hoff, 16 * (int64_t)ntiles, s, nullptr);
        k_rs_scatter<<<ntiles, 256, 0, s>>>(ka, va, n, shift, hoff, ntiles, kb, vb);
        PGB_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    c->d_perm.resize(n);
    c->d_inv.resize(n);
    c->d_key.resize(n);
    c->d_qcell.resize(3 * n);
    PGB_CUDA(cudaMemcpyAsync(c->d_perm.p, va, 4 * n, cudaMemcpyDeviceToDevice, s));
    k_key30<<<nblk(n, 256), 256, 0, s>>>(ka, n, c->d_key);
    k_gather_i32x3<<<nblk(n, 256), 256, 0, s>>>(qc, c->d_perm, n, c->d_qcell);
    k_invert<<<nblk(n, 256), 256, 0, s>>>(c->d_perm, n, c->d_inv);
    PGB_CUDA(cudaGetLastError());

    // octree: every level at once (roots first, then each level in key order)
    DBuf<int64_t> M, S, lb;
    M.resize(OCT_LEVELS * n + 1);
    S.resize(OCT_LEVELS * n + 1);
    lb.resize(OCT_LEVELS + 1);
    k_oct_marks<<<nblk(OCT_LEVELS * n + 1, 256), 256, 0, s>>>(c->d_key, d_off, nb, n, c->p.leaf_size, M);
    PGB_CUDA(cudaGetLastError());
    exclusive_scan_i64(M, S, OCT_LEVELS * n + 1, s, nullptr);
    k_oct_levels<<<1, 32, 0, s>>>(S, n, lb);
    PGB_CUDA(cudaGetLastError());
    std::vector<int64_t> hl(OCT_LEVELS + 1);
    PGB_CUDA(cudaMemcpyAsync(hl.data(), lb.p, 8 * (OCT_LEVELS + 1), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    int nlev = 0;
    while (nlev < OCT_LEVELS && hl[nlev + 1] > hl[nlev]) ++nlev;
    const int64_t nn = hl[nlev];
    c->level_begin.assign(hl.begin(), hl.begin() + nlev + 1);
    c->n_nodes = nn;
    c->d_node_start.resize(nn); c->d_node_end.resize(nn); c->d_node_body.resize(nn);
    c->d_node_child.resize(nn); c->d_node_nchild.resize(nn); c->d_node_level.resize(nn);
    k_oct_nodes<<<nblk(OCT_LEVELS * n, 256), 256, 0, s>>>(c->d_key, d_off, nb, n, M, S, c->d_node_start,
                                                          c->d_node_end, c->d_node_body, c->d_node_level,
                                                          c->d_node_child, c->d_node_nchild);
    PGB_CUDA(cudaGetLastError());
    c->h_node_level.assign(nn, 0);
    for (int l = 0; l < nlev; ++l)
        for (int64_t k = c->level_begin[l]; k < c->level_begin[l + 1]; ++k) c->h_node_level[k] = l;
    for (int b = 0; b < nb; ++b) c->bodies[b].root = b;
    c->d_node_parent.resize(nn);
    k_fill_i32<<<nblk(nn, 256), 256, 0, s>>>(c->d_node_parent, nn, -1);
    k_parents<<<nblk(nn, 256), 256, 0, s>>>(c->d_node_child, c->d_node_nchild, nn, c->d_node_parent);
    c->d_up_counter.resize(nn);
    PGB_CUDA(cudaMemsetAsync(c->d_up_counter.p, 0, 4 * nn, s));
    // leaves
    DBuf<int64_t> mark, lscan;
    mark.resize(n);
    lscan.resize(n);
    PGB_CUDA(cudaMemsetAsync(mark.p, 0, 8 * n, s));
    k_mark_leaves<<<nblk(nn, 256), 256, 0, s>>>(c->d_node_start, c->d_node_nchild, nn, mark);
    int64_t nl = 0;
    exclusive_scan_i64(mark, lscan, n, s, &nl);
    c->n_leaves = nl;
    c->d_node_leaf0.resize(nn);
    c->d_node_leaf1.resize(nn);
    c->d_leaf_node.resize(nl);
    c->d_pan_leaf.resize(n);
    k_leaf_ids<<<nblk(nn, 256), 256, 0, s>>>(c->d_node_start, c->d_node_end, c->d_node_nchild, nn, lscan, n, nl,
                                             c->d_node_leaf0, c->d_node_leaf1, c->d_leaf_node);
    k_pan_leaf<<<nblk(nl, 128), 128, 0, s>>>(c->d_leaf_node, c->d_node_start, c->d_node_end, nl, c->d_pan_leaf);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    c->order_valid = true;
}

// ---------------------------------------------------------------- geometry
// World-frame panel geometry in sorted order and the K-point quadrature nodes
// y = c + sum_a mu_a (v_a - c), weights w_m A (Section 3.1).
__global__ void k_geometry(const double* vb, const int32_t* tris, const int32_t* perm, const int32_t* pan_body,
                           const double* pose, int64_t n, Rules r, double* V, double* C, double* Nn, double* A,
                           double* Y, double* W, int32_t* pbody) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t g = perm[i];
    int b = pan_body[g];
    pbody[i] = b;
    const double* P = pose + 12 * b;
    double v[3][3];
    for (int k = 0; k < 3; ++k) rigid(P, vb + 3 * (int64_t)tris[3 * g + k], v[k]);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = __ddiv_rn(dadd(dadd(v[0][a], v[1][a]), v[2][a]), 3.0);
    double e1[3], e2[3], cr[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = v[1][a] - v[0][a];
        e2[a] = v[2][a] - v[0][a];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nr = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) V[9 * i + 3 * k + a] = v[k][a];
    for (int a = 0; a < 3; ++a) {
        C[3 * i + a] = c[a];
        Nn[3 * i + a] = cr[a] / nr;
    }
    double area = 0.5 * nr;
    A[i] = area;
    for (int m = 0; m < r.K; ++m) {
        for (int a = 0; a < 3; ++a)
            Y[3 * (i * r.K + m) + a] =
                c[a] + ((r.mu[m][0] * (v[0][a] - c[a]) + r.mu[m][1] * (v[1][a] - c[a])) + r.mu[m][2] * (v[2][a] - c[a]));
        W[i * r.K + m] = r.w[m] * area;
    }
}

// Node centre (cube cell centre, world frame), radius^2 over its quadrature
// nodes, centroid box and max 8*A of its panels.  One block per node.
__global__ void k_node_geometry(const int32_t* nstart, const int32_t* nend, const int32_t* nlevel,
                                const int32_t* nbody, const int32_t* qcell, BodyFrame f, const double* ext,
                                const double* pose, const double* Y, const double* C, const double* A, int K,
                                double* center, double* r2, double* clo, double* chi, double* a8) {
    __shared__ double cw[3];
    int nd = blockIdx.x;
    int64_t s = nstart[nd], e = nend[nd];
    int b = nbody[nd], l = nlevel[nd];
    if (threadIdx.x == 0) {
        double h = ldexp(ext[b], -(l + 1));
        double cb[3];
        for (int a = 0; a < 3; ++a) {
            int cell = qcell[3 * s + a] >> (10 - l);
            cb[a] = dadd(f.lo[b][a], dmul(h, (double)(2 * cell + 1)));
        }
        rigid(pose + 12 * b, cb, cw);
        for (int a = 0; a < 3; ++a) center[3 * nd + a] = cw[a];
    }
    __syncthreads();
    __shared__ double sred[7][32];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, am = 0;
    for (int64_t p = s + threadIdx.x; p < e; p += blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], C[3 * p + a]);
            hi[a] = fmax(hi[a], C[3 * p + a]);
        }
        am = fmax(am, 8.0 * A[p]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    if ((threadIdx.x & 31) == 0) {
        int wi = threadIdx.x >> 5;
        for (int a = 0; a < 3; ++a) {
            sred[a][wi] = lo[a];
            sred[3 + a][wi] = hi[a];
        }
        sred[6][wi] = am;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            for (int a = 0; a < 3; ++a) {
                lo[a] = fmin(lo[a], sred[a][k]);
                hi[a] = fmax(hi[a], sred[3 + a][k]);
            }
            am = fmax(am, sred[6][k]);
        }
        for (int a = 0; a < 3; ++a) {
            clo[3 * nd + a] = lo[a];
            chi[3 * nd + a] = hi[a];
        }
        a8[nd] = am;
    }
}

// Node radius^2 = max over the node's quadrature nodes of |y - c|^2 (unfused
// FP64).  Nodes are cut into chunks of R2_CHUNK points, one block per chunk;
// chunk maxima combine by an integer atomicMax on the bit pattern (valid for
// non-negative doubles, and order-independent).
#define R2_CHUNK 4096
__global__ void k_chunk_count(const int32_t* nstart, const int32_t* nend, int64_t nn, int K, int64_t* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nn) cnt[i] = ((int64_t)(nend[i] - nstart[i]) * K + R2_CHUNK - 1) / R2_CHUNK;
}
__global__ void k_node_r2(const int32_t* nstart, const int32_t* nend, int64_t nn, const int64_t* coff,
                          const double* center, const double* Y, int K, unsigned long long* r2bits) {
    __shared__ double sh[32];
    __shared__ int64_t s_nd;
    const int64_t chunk = blockIdx.x;
    if (threadIdx.x == 0) {  // node owning this chunk: last coff <= chunk
        int64_t lo = 0, hi = nn;
        while (hi - lo > 1) {
            int64_t m = (lo + hi) >> 1;
            if (coff[m] <= chunk) lo = m;
            else hi = m;
        }
        while (lo + 1 < nn && coff[lo + 1] <= chunk) ++lo;
        s_nd = lo;
    }
    __syncthreads();
    const int64_t nd = s_nd;
    const int64_t p0 = (int64_t)nstart[nd] * K + (chunk - coff[nd]) * R2_CHUNK;
    const int64_t p1 = min((int64_t)nend[nd] * K, p0 + R2_CHUNK);
    const double c0 = center[3 * nd], c1 = center[3 * nd + 1], c2 = center[3 * nd + 2];
    double m = 0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        double dx = dsub(Y[3 * p], c0), dy = dsub(Y[3 * p + 1], c1), dz = dsub(Y[3 * p + 2], c2);
        m = fmax(m, dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, sh[k]);
        atomicMax(r2bits + nd, (unsigned long long)__double_as_longlong(m));
    }
}

// Target groups: consecutive runs of group_size panels (key order) per body.
__global__ void k_groups(const int32_t* gstart, const int32_t* gend, int64_t ng, const double* C, double* glo,
                         double* ghi, double* gcen) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t p = gstart[g]; p < gend[g]; ++p)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], C[3 * p + a]);
            hi[a] = fmax(hi[a], C[3 * p + a]);
        }
    for (int a = 0; a < 3; ++a) {
        glo[3 * g + a] = lo[a];
        ghi[3 * g + a] = hi[a];
        gcen[3 * g + a] = 0.5 * (lo[a] + hi[a]);
    }
}

__global__ void k_rel_targets(const int32_t* gstart, const int32_t* gend, int64_t ng, const double* C,
                              const double* gcen, float4* x32, dbl4* x64) {
    int64_t g = blockIdx.x;
    if (g >= ng) return;
    for (int64_t p = gstart[g] + threadIdx.x; p < gend[g]; p += blockDim.x) {
        double dx = C[3 * p] - gcen[3 * g], dy = C[3 * p + 1] - gcen[3 * g + 1], dz = C[3 * p + 2] - gcen[3 * g + 2];
        x32[p] = make_float4((float)dx, (float)dy, (float)dz, 0.f);
        x64[p] = dbl4{dx, dy, dz, 0.0};
    }
}

__global__ void k_rel_sources(const int32_t* pan_leaf, const int32_t* leaf_node, const double* ncen, int64_t n, int K,
                              const double* Y, const double* W, float4* y32, dbl4* y64) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n * K) return;
    int64_t i = p / K;
    int nd = leaf_node[pan_leaf[i]];
    double dx = Y[3 * p] - ncen[3 * nd], dy = Y[3 * p + 1] - ncen[3 * nd + 1], dz = Y[3 * p + 2] - ncen[3 * nd + 2];
    y32[p] = make_float4((float)dx, (float)dy, (float)dz, (float)W[p]);
    y64[p] = dbl4{dx, dy, dz, W[p]};
}

void build_geometry(pgb_ctx* c) {
    cudaStream_t s = c->stream;
    int64_t n = c->n_pan;
    int K = c->p.K;
    Rules r = make_rules(K, c->p.K_near, c->p.n_edge);
    // poses
    std::vector<double> pose(12 * c->bodies.size());
    for (size_t b = 0; b < c->bodies.size(); ++b) {
        for (int a = 0; a < 9; ++a) pose[12 * b + a] = c->bodies[b].R[a];
        for (int a = 0; a < 3; ++a) pose[12 * b + 9 + a] = c->bodies[b].t[a];
    }
    PGB_CUDA(cudaMemcpyAsync(c->d_pose.p, pose.data(), 8 * pose.size(), cudaMemcpyHostToDevice, s));
    c->d_v.resize(9 * n); c->d_c.resize(3 * n); c->d_n.resize(3 * n); c->d_A.resize(n);
    c->d_y.resize(3 * n * K); c->d_w.resize(n * K); c->d_pbody.resize(n);
    k_geometry<<<nblk(n, 128), 128, 0, s>>>(c->d_vb, c->d_tris, c->d_perm, c->d_pan_body, c->d_pose, n, r, c->d_v,
                                            c->d_c, c->d_n, c->d_A, c->d_y, c->d_w, c->d_pbody);
    PGB_CUDA(cudaGetLastError());
    // charges in the world frame
    if (c->n_q) {
        std::vector<double> qw(3 * c->n_q);
        for (auto& b : c->bodies) {
            for (int64_t k = 0; k < b.nq; ++k) {
                const double* v = &b.qxyz[3 * k];
                for (int a = 0; a < 3; ++a)
                    qw[3 * (b.q_off + k) + a] = ((b.R[3 * a] * v[0] + b.R[3 * a + 1] * v[1]) + b.R[3 * a + 2] * v[2]) + b.t[a];
            }
        }
        PGB_CUDA(cudaMemcpyAsync(c->d_qxyz.p, qw.data(), 8 * qw.size(), cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaStreamSynchronize(s));
    }
    BodyFrame f;
    std::vector<double> ext(c->bodies.size());
    for (size_t b = 0; b < c->bodies.size(); ++b) {
        for (int a = 0; a < 3; ++a) f.lo[b][a] = c->bodies[b].lo[a];
        f.scale[b] = 1024.0 / c->bodies[b].ext;
        ext[b] = c->bodies[b].ext;
    }
    DBuf<double> d_ext;
    d_ext.resize(ext.size());
    PGB_CUDA(cudaMemcpyAsync(d_ext.p, ext.data(), 8 * ext.size(), cudaMemcpyHostToDevice, s));
    int64_t nn = c->n_nodes;
    c->d_node_center.resize(3 * nn); c->d_node_r2.resize(nn); c->d_node_clo.resize(3 * nn);
    c->d_node_chi.resize(3 * nn); c->d_node_a8.resize(nn);
    k_node_geometry<<<(int)nn, 128, 0, s>>>(c->d_node_start, c->d_node_end, c->d_node_level, c->d_node_body,
                                            c->d_qcell, f, d_ext, c->d_pose, c->d_y, c->d_c, c->d_A, K,
                                            c->d_node_center, c->d_node_r2, c->d_node_clo, c->d_node_chi,
                                            c->d_node_a8);
    PGB_CUDA(cudaGetLastError());
    {
        DBuf<int64_t> cnt, coff;
        cnt.resize(nn);
        coff.resize(nn);
        k_chunk_count<<<nblk(nn, 256), 256, 0, s>>>(c->d_node_start, c->d_node_end, nn, K, cnt);
        int64_t nchunks = 0;
        exclusive_scan_i64(cnt, coff, nn, s, &nchunks);
        PGB_CUDA(cudaMemsetAsync(c->d_node_r2.p, 0, 8 * nn, s));
        k_node_r2<<<(unsigned)nchunks, 256, 0, s>>>(c->d_node_start, c->d_node_end, nn, coff, c->d_node_center,
                                                    c->d_y, K, (unsigned long long*)c->d_node_r2.p);
        PGB_CUDA(cudaGetLastError());
        PGB_CUDA(cudaStreamSynchronize(s));
    }
    // target groups
    std::vector<int32_t> gs, ge, gb;
    int G = c->p.group_size;
    for (size_t b = 0; b < c->bodies.size(); ++b) {
        auto& bd = c->bodies[b];
        for (int64_t o = 0; o < bd.N; o += G) {
            gs.push_back((int32_t)(bd.pan_off + o));
            ge.push_back((int32_t)(bd.pan_off + std::min<int64_t>(bd.N, o + G)));
            gb.push_back((int32_t)b);
        }
    }
    int64_t ng = (int64_t)gs.size();
    c->n_groups = ng;
    c->group_begin.assign(c->bodies.size() + 1, 0);
    for (int64_t k = 0; k < ng; ++k) c->group_begin[gb[k] + 1] = k + 1;
    for (size_t b = 1; b <= c->bodies.size(); ++b)
        c->group_begin[b] = std::max(c->group_begin[b], c->group_begin[b - 1]);
    c->adj_valid = false;
    c->d_group_start.resize(ng); c->d_group_end.resize(ng); c->d_group_body.resize(ng);
    c->d_group_lo.resize(3 * ng); c->d_group_hi.resize(3 * ng); c->d_group_center.resize(3 * ng);
    PGB_CUDA(cudaMemcpyAsync(c->d_group_start.p, gs.data(), 4 * ng, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(c->d_group_end.p, ge.data(), 4 * ng, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(c->d_group_body.p, gb.data(), 4 * ng, cudaMemcpyHostToDevice, s));
    k_groups<<<nblk(ng, 128), 128, 0, s>>>(c->d_group_start, c->d_group_end, ng, c->d_c, c->d_group_lo,
                                           c->d_group_hi, c->d_group_center);
    c->d_x32.resize(n);
    c->d_x64.resize(n);
    k_rel_targets<<<(int)ng, 32, 0, s>>>(c->d_group_start, c->d_group_end, ng, c->d_c, c->d_group_center, c->d_x32,
                                         c->d_x64);
    c->d_y32.resize(n * K);
    c->d_y64.resize(n * K);
    k_rel_sources<<<nblk(n * K, 256), 256, 0, s>>>(c->d_pan_leaf, c->d_leaf_node, c->d_node_center, n, K, c->d_y,
                                                   c->d_w, c->d_y32, c->d_y64);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- lists
// Acceptance: node far for a group when theta > 0 and r_b^2 <= theta^2 d^2,
// d = distance from the node centre to the group's box (Section 3.2).
__device__ __forceinline__ bool mac_far(double theta2, double r2, const double* cc, const double* lo, const double* hi) {
    double d2 = 0;
    double e[3];
    for (int a = 0; a < 3; ++a) {
        double u = fmax(fmax(dsub(lo[a], cc[a]), dsub(cc[a], hi[a])), 0.0);
        e[a] = u;
    }
    d2 = dadd(dadd(dmul(e[0], e[0]), dmul(e[1], e[1])), dmul(e[2], e[2]));
    return r2 <= dmul(theta2, d2);
}

struct ListArgs {
    const int32_t *nchild, *child, *nstart, *nend, *nbody, *gstart, *gend, *gbody;
    const double *center, *r2, *glo, *ghi;
    int n_bodies;
    int kind[PGB_MAX_BODIES];
    int prob[PGB_MAX_BODIES];  // problem of each body (no lists across problems)
    double theta, theta2;
    int K;
};

// count (fill == false) or write the near/far lists of each group; depth
// first, children in key order, bodies in order.  One warp per group: when a
// node is opened its children are classified (far / near leaf / to open) by
// one lane each, then pushed on the warp's stack in reverse order with their
// class, so the entries come out in the sequential depth-first order.
#define LIST_WARPS 4
// The counting pass (fill == false) also keeps the first capn near and capf
// far entries of each group in tmpn / tmpf (rows of capn / capf) and raises
// *ovf when a group has more, so that the fill pass is needed only then.
#define LIST_CAPN 256
#define LIST_CAPF 512
__global__ void __launch_bounds__(32 * LIST_WARPS) k_lists(ListArgs a, int64_t ng, bool fill, int64_t* ncnt,
                                                            int64_t* fcnt, const int64_t* noff, const int64_t* foff,
                                                            int32_t* nearl, int32_t* farl, unsigned long long* stats,
                                                            int32_t* tmpn, int32_t* tmpf, int* ovf) {
    __shared__ int32_t st_node[LIST_WARPS][PGB_LIST_STACK];
    __shared__ int8_t st_cls[LIST_WARPS][PGB_LIST_STACK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * LIST_WARPS + w;
    if (g >= ng) return;
    int64_t nn = 0, nf = 0;
    int64_t wn = fill ? noff[g] : 0, wf = fill ? foff[g] : 0;
    double lo[3], hi[3];
    for (int q = 0; q < 3; ++q) {
        lo[q] = a.glo[3 * g + q];
        hi[q] = a.ghi[3 * g + q];
    }
    const int gb = a.gbody[g];
    const int64_t gsize = a.gend[g] - a.gstart[g];
    unsigned long long p2p = 0, p2pl = 0, m2p = 0, m2pl = 0;
    bool overflow = false;
    // class of a node: 0 far, 1 near leaf, 2 open
    auto classify = [&](int nd) -> int {
        if (a.theta > 0 && mac_far(a.theta2, a.r2[nd], a.center + 3 * nd, lo, hi)) return 0;
        return a.nchild[nd] == 0 ? 1 : 2;
    };
    for (int b = 0; b < a.n_bodies; ++b) {
        if (a.prob[b] != a.prob[gb]) continue;
        const bool lap = (b == gb) && a.kind[b] == PGB_DIELECTRIC;
        int sp = 0;
        if (lane == 0) {
            st_node[w][0] = b;  // roots are nodes 0..n_bodies-1
            st_cls[w][0] = (int8_t)classify(b);
        }
        sp = 1;
        __syncwarp();
        while (sp > 0) {
            --sp;
            const int nd = st_node[w][sp];
            const int cls = st_cls[w][sp];
            __syncwarp();
            if (cls == 0) {
                if (fill && lane == 0) farl[wf] = nd;
                if (!fill && lane == 0 && nf < LIST_CAPF) tmpf[g * LIST_CAPF + nf] = nd;
                ++wf;
                ++nf;
                m2p += gsize;
                if (lap) m2pl += gsize;
            } else if (cls == 1) {
                if (fill && lane == 0) nearl[wn] = nd;
                if (!fill && lane == 0 && nn < LIST_CAPN) tmpn[g * LIST_CAPN + nn] = nd;
                ++wn;
                ++nn;
                const unsigned long long pts = (unsigned long long)(a.nend[nd] - a.nstart[nd]) * a.K;
                p2p += pts * gsize;
                if (lap) p2pl += pts * gsize;
            } else {
                const int fc = a.child[nd], k = a.nchild[nd];
                if (sp + k > PGB_LIST_STACK) {
                    overflow = true;
                    continue;
                }
                if (lane < k) {  // child `lane` goes to stack slot sp + (k - 1 - lane)
                    const int ch = fc + lane;
                    st_node[w][sp + k - 1 - lane] = ch;
                    st_cls[w][sp + k - 1 - lane] = (int8_t)classify(ch);
                }
                __syncwarp();
                sp += k;
            }
        }
    }
    if (lane != 0) return;
    if (overflow) atomicAdd(&stats[4], 1ull);  // cannot happen for depth <= 10
    if (!fill) {
        ncnt[g] = nn;
        fcnt[g] = nf;
        if (nn > LIST_CAPN || nf > LIST_CAPF) atomicOr(ovf, 1);
        atomicAdd(&stats[0], p2p);
        atomicAdd(&stats[1], p2pl);
        atomicAdd(&stats[2], m2p);
        atomicAdd(&stats[3], m2pl);
    }
}

// Lists from the entries kept by the counting pass (no group overflowed);
// one warp per group.
__global__ void k_lists_compact(int64_t ng, const int64_t* noff, const int64_t* foff, const int32_t* tmpn,
                                const int32_t* tmpf, int32_t* nearl, int32_t* farl) {
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    for (int64_t e = noff[g] + lane; e < noff[g + 1]; e += 32) nearl[e] = tmpn[g * LIST_CAPN + (e - noff[g])];
    for (int64_t e = foff[g] + lane; e < foff[g + 1]; e += 32) farl[e] = tmpf[g * LIST_CAPF + (e - foff[g])];
}

// FP32 offset of every list entry: node centre - group centre (FP64
// difference, rounded once), with the node id in the .w bits.
__global__ void k_list_offsets(int64_t ng, const int64_t* off, const int32_t* ids, const double* ncen,
                               const double* gcen, float4* out) {
    int64_t g = blockIdx.x;
    if (g >= ng) return;
    for (int64_t e = off[g] + threadIdx.x; e < off[g + 1]; e += blockDim.x) {
        int nd = ids[e];
        out[e] = make_float4((float)(ncen[3 * nd] - gcen[3 * g]), (float)(ncen[3 * nd + 1] - gcen[3 * g + 1]),
                             (float)(ncen[3 * nd + 2] - gcen[3 * g + 2]), __int_as_float(nd));
    }
}

// P2P tiles: every near leaf of a group cut into runs of at most 32
// quadrature points; descriptor = (leaf centre - group centre in FP32, first
// point) and (leaf, count, flags: 1 Laplace pair, 2 leaf holds group targets, body).
// One warp per group; the lanes take its near entries 32 at a time.
__global__ void k_tile_count(int64_t ng, const int64_t* noff, const int32_t* nearl, const int32_t* nstart,
                             const int32_t* nend, int K, int64_t* cnt) {
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    int64_t c = 0;
    for (int64_t e = noff[g] + lane; e < noff[g + 1]; e += 32) {
        const int nd = nearl[e];
        c += ((int64_t)(nend[nd] - nstart[nd]) * K + 31) / 32;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[g] = c;
}
// Tiles in entry order: a warp scan of the lanes' tile counts places each
// entry's run after those of the entries before it.
__global__ void k_tile_fill(int64_t ng, const int64_t* noff, const int32_t* nearl, const float4* near4,
                            const int32_t* nstart, const int32_t* nend, const int32_t* nbody, const int32_t* gstart,
                            const int32_t* gend, const int32_t* gbody, BodyDev bd, int K, const int64_t* toff,
                            float4* td, int4* tm) {
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    int64_t w = toff[g];
    const int gb = gbody[g];
    const int64_t e1 = noff[g + 1];
    for (int64_t e0 = noff[g]; e0 < e1; e0 += 32) {
        const int64_t e = e0 + lane;
        int nd = 0;
        int64_t s0 = 0, s1 = 0, nt = 0;
        if (e < e1) {
            nd = nearl[e];
            s0 = (int64_t)nstart[nd] * K;
            s1 = (int64_t)nend[nd] * K;
            nt = (s1 - s0 + 31) / 32;
        }
        int64_t incl = nt;  // inclusive scan over the lanes
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (e < e1) {
            const int nb = nbody[nd];
            const int flags = ((nb == gb && bd.kind[gb] == PGB_DIELECTRIC) ? 1 : 0) |
                              ((nstart[nd] < gend[g] && nend[nd] > gstart[g]) ? 2 : 0);
            const float4 o = near4[e];
            int64_t t = w + incl - nt;
            for (int64_t q = s0; q < s1; q += 32, ++t) {
                td[t] = make_float4(o.x, o.y, o.z, __int_as_float((int)q));
                tm[t] = make_int4(nd, (int)min((int64_t)32, s1 - q), flags, nb);
            }
        }
        w += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Work items per group: ceil(tiles / p2p_item) for P2P and
// ceil(far entries / m2p_item) for M2P.
__global__ void k_item_count(int64_t ng, const int64_t* toff, const int64_t* foff, int pi, int fi, int64_t* pc,
                             int64_t* fc) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    pc[g] = (toff[g + 1] - toff[g] + pi - 1) / pi;
    fc[g] = (foff[g + 1] - foff[g] + fi - 1) / fi;
}
__global__ void k_item_fill(int64_t ng, const int64_t* poff, const int64_t* foff, const int32_t* gstart,
                            const int32_t* gend, int32_t* pg, int32_t* fg, int32_t* pan_group) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    for (int64_t i = poff[g]; i < poff[g + 1]; ++i) pg[i] = (int32_t)g;
    for (int64_t i = foff[g]; i < foff[g + 1]; ++i) fg[i] = (int32_t)g;
    for (int32_t p = gstart[g]; p < gend[g]; ++p) pan_group[p] = (int32_t)g;
}

void make_lists(pgb_ctx* c, const double* r2, const double* glo, const double* ghi, DBuf<int64_t>& noff,
                DBuf<int32_t>& nearl, DBuf<int64_t>& foff, DBuf<int32_t>& farl, DBuf<float4>& near4,
                DBuf<float4>& far4, int64_t& n_near, int64_t& n_far, unsigned long long* stats4) {
    cudaStream_t s = c->stream;
    int64_t ng = c->n_groups;
    ListArgs a;
    a.nchild = c->d_node_nchild; a.child = c->d_node_child; a.nstart = c->d_node_start; a.nend = c->d_node_end;
    a.nbody = c->d_node_body; a.gstart = c->d_group_start; a.gend = c->d_group_end; a.gbody = c->d_group_body;
    a.center = c->d_node_center; a.r2 = r2; a.glo = glo; a.ghi = ghi;
    a.n_bodies = (int)c->bodies.size();
    for (int b = 0; b < a.n_bodies; ++b) {
        a.kind[b] = c->bodies[b].kind;
        a.prob[b] = c->bodies[b].prob;
    }
    a.theta = c->p.theta;
    a.theta2 = c->p.theta * c->p.theta;
    a.K = c->p.K;
    DBuf<int64_t> nc, fc;
    nc.resize(ng); fc.resize(ng);
    noff.resize(ng + 1);
    foff.resize(ng + 1);
    DBuf<unsigned long long> st;
    st.resize(6);
    PGB_CUDA(cudaMemsetAsync(st.p, 0, 48, s));
    int* ovf = (int*)(st.p + 5);
    c->d_list_tmp.resize((size_t)ng * (LIST_CAPN + LIST_CAPF));
    int32_t* tmpn = c->d_list_tmp.p;
    int32_t* tmpf = c->d_list_tmp.p + (size_t)ng * LIST_CAPN;
    k_lists<<<nblk(ng, LIST_WARPS), 32 * LIST_WARPS, 0, s>>>(a, ng, false, nc, fc, nullptr, nullptr, nullptr, nullptr,
                                                              st, tmpn, tmpf, ovf);
    PGB_CUDA(cudaGetLastError());
    unsigned long long h[6];
    PGB_CUDA(cudaMemcpyAsync(h, st.p, 48, cudaMemcpyDeviceToHost, s));
    int64_t tn = 0, tf = 0;
    exclusive_scan_i64(nc, noff, ng, s, &tn);
    exclusive_scan_i64(fc, foff, ng, s, &tf);
    PGB_CUDA(cudaMemcpyAsync(noff.p + ng, &tn, 8, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(foff.p + ng, &tf, 8, cudaMemcpyHostToDevice, s));
    n_near = tn;
    n_far = tf;
    nearl.resize(tn);
    farl.resize(tf);
    // the scans synchronised the stream: h (counts' statistics, overflow) is valid
    if (((int*)(h + 5))[0])
        k_lists<<<nblk(ng, LIST_WARPS), 32 * LIST_WARPS, 0, s>>>(a, ng, true, nullptr, nullptr, noff, foff, nearl,
                                                                  farl, st, nullptr, nullptr, nullptr);
    else
        k_lists_compact<<<nblk(32 * ng, 128), 128, 0, s>>>(ng, noff, foff, tmpn, tmpf, nearl, farl);
    PGB_CUDA(cudaGetLastError());
    near4.resize(tn);
    far4.resize(tf);
    k_list_offsets<<<(unsigned)ng, 64, 0, s>>>(ng, noff, nearl, c->d_node_center, c->d_group_center, near4);
    k_list_offsets<<<(unsigned)ng, 64, 0, s>>>(ng, foff, farl, c->d_node_center, c->d_group_center, far4);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    if (h[4]) fail(PGB_EINVAL, "octree traversal stack overflow");
    if (stats4)
        for (int k = 0; k < 4; ++k) stats4[k] = h[k];
    PGB_LAUNCHED(c, 6);
}

void build_lists(pgb_ctx* c) {
    cudaStream_t s = c->stream;
    int64_t ng = c->n_groups;
    unsigned long long h[4];
    make_lists(c, c->d_node_r2, c->d_group_lo, c->d_group_hi, c->d_near_off, c->d_near, c->d_far_off, c->d_far,
               c->d_near4, c->d_far4, c->n_near, c->n_far, h);
    c->p2p_pairs = (int64_t)h[0];
    c->p2p_lap = (int64_t)h[1];
    c->m2p_pairs = (int64_t)h[2];
    c->m2p_lap = (int64_t)h[3];
    {
        DBuf<int64_t> tc;
        tc.resize(ng);
        c->d_tile_off.resize(ng + 1);
        k_tile_count<<<nblk(32 * ng, 128), 128, 0, s>>>(ng, c->d_near_off, c->d_near, c->d_node_start, c->d_node_end,
                                                   c->p.K, tc);
        int64_t nt = 0;
        exclusive_scan_i64(tc, c->d_tile_off, ng, s, &nt);
        PGB_CUDA(cudaMemcpyAsync(c->d_tile_off.p + ng, &nt, 8, cudaMemcpyHostToDevice, s));
        c->n_tiles = nt;
        c->d_tile_d.resize(nt);
        c->d_tile_m.resize(nt);
        k_tile_fill<<<nblk(32 * ng, 128), 128, 0, s>>>(ng, c->d_near_off, c->d_near, c->d_near4, c->d_node_start,
                                                  c->d_node_end, c->d_node_body, c->d_group_start, c->d_group_end,
                                                  c->d_group_body, body_dev(c), c->p.K, c->d_tile_off, c->d_tile_d,
                                                  c->d_tile_m);
        PGB_CUDA(cudaGetLastError());
    }
    {
        DBuf<int64_t> pc, fc;
        pc.resize(ng);
        fc.resize(ng);
        c->d_pitem_off.resize(ng + 1);
        c->d_fitem_off.resize(ng + 1);
        k_item_count<<<nblk(ng, 128), 128, 0, s>>>(ng, c->d_tile_off, c->d_far_off, c->p.p2p_item, c->p.m2p_item,
                                                   pc, fc);
        int64_t np = 0, nf = 0;
        exclusive_scan_i64(pc, c->d_pitem_off, ng, s, &np);
        exclusive_scan_i64(fc, c->d_fitem_off, ng, s, &nf);
        PGB_CUDA(cudaMemcpyAsync(c->d_pitem_off.p + ng, &np, 8, cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(c->d_fitem_off.p + ng, &nf, 8, cudaMemcpyHostToDevice, s));
        c->n_pitems = np;
        c->n_fitems = nf;
        c->d_pitem_group.resize(std::max<int64_t>(np, 1));
        c->d_fitem_group.resize(std::max<int64_t>(nf, 1));
        c->d_pan_group.resize(c->n_pan);
        k_item_fill<<<nblk(ng, 128), 128, 0, s>>>(ng, c->d_pitem_off, c->d_fitem_off, c->d_group_start,
                                                  c->d_group_end, c->d_pitem_group, c->d_fitem_group, c->d_pan_group);
        PGB_CUDA(cudaGetLastError());
        PGB_CUDA(cudaStreamSynchronize(s));
    }
    PGB_LAUNCHED(c, 4);
    c->lists_valid = true;
}

// Offsets of the kept list entries and P2P tiles after the node and group
// centres moved (pgb_tree_refresh): entries, tiles and work items stay.
void refresh_lists(pgb_ctx* c) {
    cudaStream_t s = c->stream;
    const int64_t ng = c->n_groups;
    if (ng == 0) return;
    k_list_offsets<<<(unsigned)ng, 64, 0, s>>>(ng, c->d_near_off, c->d_near, c->d_node_center, c->d_group_center,
                                               c->d_near4);
    k_list_offsets<<<(unsigned)ng, 64, 0, s>>>(ng, c->d_far_off, c->d_far, c->d_node_center, c->d_group_center,
                                               c->d_far4);
    k_tile_fill<<<nblk(32 * ng, 128), 128, 0, s>>>(ng, c->d_near_off, c->d_near, c->d_near4, c->d_node_start,
                                                   c->d_node_end, c->d_node_body, c->d_group_start, c->d_group_end,
                                                   c->d_group_body, body_dev(c), c->p.K, c->d_tile_off, c->d_tile_d,
                                                   c->d_tile_m);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    PGB_LAUNCHED(c, 3);
}

// ---------------------------------------------------------------- corrections
struct CorrArgs {
    const int32_t *nchild, *child, *nstart, *nend;
    const double *clo, *chi, *a8, *C, *A;
    // FP32 copies for the prefilters: per panel (centroid, sqrt(8 A)), per
    // node (box low corner, sqrt(a8)) and (box high corner, 0); delta bounds
    // the error of a difference of two FP32-rounded coordinates
    const float4 *pf4, *nlo4, *nhi4;
    float delta;
    int n_bodies;
    int prob[PGB_MAX_BODIES];    // problem of each body (no entries across problems)
    int in_set[PGB_MAX_BODIES];  // bodies taking part (targets and sources; a region's boundary)
};

// candidates j of target i: |c_i - c_j|^2 < 8 A_j (|x - c_j| < 2 L_j), or j == i;
// cross == false: sources of the target's own body, true: of the other bodies
// The counting pass also keeps the first `cap` candidates of each target in
// tmp (row i at tmp + i * cap) and raises *overflow when a target has more,
// so that the fill pass is needed only then.
// One warp per 32 consecutive targets (sorted order, so they lie close
// together): the warp walks the union of the nodes its targets need (a node
// is opened when any lane's target is within its reach, the FP64 test of the
// per-target walk), and at a leaf every lane tests its own target against
// the leaf's panels.  The panel test is prefiltered in FP32 on the FP64
// differences (a panel is skipped only when its squared distance exceeds
// 8 A_j by more than 1e-5 relative, far above the FP32 rounding of the
// squares) and decided in FP64 as the oracle does, so each row holds the
// per-target walk's entries in the same depth-first order.
#define CORR_WARPS 4
__global__ void __launch_bounds__(32 * CORR_WARPS) k_corr_find(CorrArgs a, int64_t n, bool fill, bool cross,
                                                               const int32_t* pbody, int64_t* cnt,
                                                               const int64_t* off, int32_t* cj, int32_t* tmp,
                                                               int cap, int* overflow) {
    __shared__ int32_t stack[CORR_WARPS][PGB_LIST_STACK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * CORR_WARPS + w) * 32;
    if (i0 >= n) return;  // warp-uniform
    const int64_t i = i0 + lane;
    const bool valid = i < n;
    const int64_t ii = valid ? i : i0;
    const double x[3] = {a.C[3 * ii], a.C[3 * ii + 1], a.C[3 * ii + 2]};
    const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    int64_t k = 0, wr = fill && valid ? off[i] : 0;
    const int ib = pbody[ii];
    for (int b = 0; b < a.n_bodies; ++b) {
        const bool mine = valid && a.in_set[ib] && ((b != ib) == cross) && a.prob[b] == a.prob[ib] && a.in_set[b];
        if (!__any_sync(0xffffffffu, mine)) continue;
        int sp = 0;
        if (lane == 0) stack[w][0] = b;
        sp = 1;
        __syncwarp();
        while (sp > 0) {
            const int nd = stack[w][--sp];
            __syncwarp();
            bool need = false;
            if (mine) {
                // conservative FP32 form of the FP64 test d2 < a8 (or d2 = 0):
                // a node it passes may still hold no candidate (the panel test
                // below decides), a node it fails holds none
                const float4 lo = a.nlo4[nd], hi = a.nhi4[nd];
                const float ux = fmaxf(fmaxf(lo.x - xf[0], xf[0] - hi.x), 0.f);
                const float uy = fmaxf(fmaxf(lo.y - xf[1], xf[1] - hi.y), 0.f);
                const float uz = fmaxf(fmaxf(lo.z - xf[2], xf[2] - hi.z), 0.f);
                const float d2 = ux * ux + uy * uy + uz * uz;
                const float reach = lo.w + a.delta;
                need = d2 < reach * reach * 1.000004f || d2 == 0.f;
            }
            if (!__any_sync(0xffffffffu, need)) continue;
            if (a.nchild[nd] == 0) {
                if (need) {
                    for (int64_t j = a.nstart[nd]; j < a.nend[nd]; ++j) {
                        // FP32 distance of the rounded centroids, off by at most
                        // delta: clearly outside or inside 2L is decided here,
                        // the band between goes to the FP64 test of the oracle
                        const float4 pj = a.pf4[j];
                        const float fx = xf[0] - pj.x, fy = xf[1] - pj.y, fz = xf[2] - pj.z;
                        const float fd = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, fz * fz));
                        const float up = pj.w + a.delta, dn = pj.w - a.delta;
                        bool near = j == ii;
                        if (!near) {
                            if (fd > up * up * 1.000004f) continue;
                            if (dn > 0.5f * pj.w && fd < dn * dn * 0.999996f) {
                                near = true;
                            } else {
                                const double dx = x[0] - a.C[3 * j], dy = x[1] - a.C[3 * j + 1],
                                             dz = x[2] - a.C[3 * j + 2];
                                const double dd = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
                                near = dd < 8.0 * a.A[j];
                            }
                        }
                        if (near) {
                            if (fill) cj[wr++] = (int32_t)j;
                            else if (k < cap) tmp[ii * cap + k] = (int32_t)j;
                            ++k;
                        }
                    }
                }
            } else {
                const int fc = a.child[nd], m = a.nchild[nd];
                if (sp + m > PGB_LIST_STACK) continue;
                if (lane == 0)
                    for (int q = m - 1; q >= 0; --q) stack[w][sp + (m - 1 - q)] = fc + q;
                sp += m;
                __syncwarp();
            }
        }
    }
    if (!fill && valid) {
        cnt[i] = k;
        if (k > cap) atomicOr(overflow, 1);
    }
}

// FP32 prefilter data of the near-field search (CorrArgs).
__global__ void k_corr_prefilter(int64_t n, int64_t nn, const double* C, const double* A, const double* clo,
                                 const double* chi, const double* a8, float4* pf4, float4* nlo4, float4* nhi4) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n)
        pf4[t] = make_float4((float)C[3 * t], (float)C[3 * t + 1], (float)C[3 * t + 2], sqrtf((float)(8.0 * A[t])));
    if (t < nn) {
        nlo4[t] = make_float4((float)clo[3 * t], (float)clo[3 * t + 1], (float)clo[3 * t + 2], sqrtf((float)a8[t]));
        nhi4[t] = make_float4((float)chi[3 * t], (float)chi[3 * t + 1], (float)chi[3 * t + 2], 0.f);
    }
}

// CSR rows from the candidates kept by the counting pass (no row overflowed).
__global__ void k_corr_compact(int64_t n, const int64_t* off, const int32_t* tmp, int cap, int32_t* cj) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off[i], e = off[i + 1];
    for (int64_t k = b; k < e; ++k) cj[k] = tmp[i * cap + (k - b)];
}

// Fine-rule (19- or 37-point) nodes of every panel, mapped like the K-point nodes.
__global__ void k_fine_nodes(int64_t n, const double* V, const double* C, Rules r, double* YF) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * r.Kn) return;
    const int64_t j = t / r.Kn;
    const int m = (int)(t - j * r.Kn);
    const double* v = V + 9 * j;
    const double* cjp = C + 3 * j;
    for (int a = 0; a < 3; ++a)
        YF[3 * t + a] = cjp[a] + ((r.mun[m][0] * (v[a] - cjp[a]) + r.mun[m][1] * (v[3 + a] - cjp[a])) +
                                  r.mun[m][2] * (v[6 + a] - cjp[a]));
}

// Quadrature nodes (3 doubles each) split into double-single once per build.
__global__ void k_nodes_to_ds(const double* __restrict__ in, ds* __restrict__ out, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = ds_from_double(in[t]);
}

// Kernel values at a target x from a source point y with normal n (no 1/4pi)
// in double-single arithmetic (about 48 significant bits, on the FP32 pipe):
// V_L, K_L (with LAP), V_Y, K_Y weighted by w.
template <bool LAP>
__device__ __forceinline__ void kern4_ds(const ds* x, const ds* y, const ds* n, ds kappa, ds w, ds& vl, ds& kl,
                                         ds& vy, ds& ky) {
    const ds dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    const ds r2 = ds_fma(dx, dx, ds_fma(dy, dy, dz * dz));
    if (!(r2.hi > 0.f)) return;
    const ds ri = ds_rsqrt(r2);
    const ds r = r2 * ri;
    const ds nd = ds_fma(n[0], dx, ds_fma(n[1], dy, n[2] * dz));
    const ds kr = kappa * r;
    const ds e = ds_exp(-kr);
    const ds ri3 = (ri * ri) * ri;
    const ds wn = w * nd;
    if (LAP) {
        vl = ds_fma(w, ri, vl);
        kl = ds_fma(wn, ri3, kl);
    }
    vy = ds_fma(w * e, ri, vy);
    ky = ds_fma((wn * (kr + ds(1))) * e, ri3, ky);
}

template <bool LAP>
__device__ __forceinline__ void corr_sums_ds(const ds* x, const ds* nj, int64_t j, const ds* YF, const ds* Y,
                                             const double* W, double Aj, const Rules& r, ds kappa, ds* tv, ds* kv) {
    for (int m = 0; m < r.Kn; ++m)
        kern4_ds<LAP>(x, YF + 3 * (j * r.Kn + m), nj, kappa, ds_from_double(r.wn[m] * Aj), tv[0], tv[1], tv[2],
                      tv[3]);
    for (int m = 0; m < r.K; ++m)
        kern4_ds<LAP>(x, Y + 3 * (j * r.K + m), nj, kappa, ds_from_double(W[j * r.K + m]), kv[0], kv[1], kv[2],
                      kv[3]);
}

__device__ __forceinline__ int64_t owner_row(const int64_t* off, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n;  // last row with off[row] <= e
    while (hi - lo > 1) {
        const int64_t m = (lo + hi) >> 1;
        if (off[m] <= e) lo = m;
        else hi = m;
    }
    return lo;
}

// Correction entries (i, j), j != i: fine rule minus the K-point sum,
// for V_L, K_L, V_Y, K_Y (Section 3.1), one thread per entry, in
// double-single arithmetic from the nodes split once per build (YF, Y); the
// Laplace pair only where it enters a row (same dielectric body).  The
// semi-analytical self entries stay FP64 (k_corr_self).
__global__ void k_corr_values(int64_t n, int64_t tot, const int64_t* off, const int32_t* cj, const ds* YF,
                              const double* C, const double* Nn, const double* A, const ds* Y, const double* W,
                              const int32_t* pbody, BodyDev bd, Rules r, double kappa, dbl4* out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const int64_t i = owner_row(off, n, e);
    const int64_t j = cj[e];
    if (j == i) return;  // self entries: k_corr_self
    const ds x[3] = {ds_from_double(C[3 * i]), ds_from_double(C[3 * i + 1]), ds_from_double(C[3 * i + 2])};
    const ds nj[3] = {ds_from_double(Nn[3 * j]), ds_from_double(Nn[3 * j + 1]), ds_from_double(Nn[3 * j + 2])};
    const int bi = pbody[i], bj = pbody[j];
    const bool lap = bi == bj && bd.kind[bi] == PGB_DIELECTRIC;
    const ds kp = ds_from_double(kappa);
    ds tv[4] = {ds(0), ds(0), ds(0), ds(0)}, kv[4] = {ds(0), ds(0), ds(0), ds(0)};
    if (lap) corr_sums_ds<true>(x, nj, j, YF, Y, W, A[j], r, kp, tv, kv);
    else corr_sums_ds<false>(x, nj, j, YF, Y, W, A[j], r, kp, tv, kv);
    double d[4];
    for (int q = 0; q < 4; ++q) d[q] = ds_to_double(tv[q] - kv[q]) / PGB_FOUR_PI;
    out[e] = dbl4{d[0], d[1], d[2], d[3]};
}

// Self entries: the whole semi-analytical single layer (the treecode sums
// leave out the target's own panel): three sub-triangles about the centroid,
// radial integral in closed form, n_edge Gauss points along each edge; K_ii = 0.
// One thread per target; the self entry is located by its column.
__global__ void k_corr_self(int64_t n, const int64_t* off, const int32_t* cj, const double* V, const double* C,
                            const int32_t* pbody, BodyDev bd, Rules r, double kappa, dbl4* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t e = -1;
    for (int64_t k = off[i]; k < off[i + 1]; ++k)
        if (cj[k] == i) e = k;
    if (e < 0) return;
    const double* x = C + 3 * i;
    const double* v = V + 9 * i;
    // square roots and reciprocals by rsqrt_nr<2> (FP64 rounding, common.cuh):
    // the FP64 pipe runs at 1/64 of the FP32 rate and the library's sqrt and
    // division cost several times as much
    const double inv_kappa = kappa > 0 ? 1.0 / kappa : 0.0;
    double vl = 0, vy = 0;
    for (int ed = 0; ed < 3; ++ed) {
        const double* pa = v + 3 * ed;
        const double* pb = v + 3 * ((ed + 1) % 3);
        double ev[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double ell2 = ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2];
        const double il = rsqrt_nr<2>(ell2);
        const double ell = ell2 * il;
        double u[3] = {ev[0] * il, ev[1] * il, ev[2] * il};
        double cpa[3] = {x[0] - pa[0], x[1] - pa[1], x[2] - pa[2]};
        double proj = cpa[0] * u[0] + cpa[1] * u[1] + cpa[2] * u[2];
        double hv[3] = {cpa[0] - proj * u[0], cpa[1] - proj * u[1], cpa[2] - proj * u[2]};
        const double h2 = hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2];
        const double h = h2 * rsqrt_nr<2>(h2);
        for (int g = 0; g < r.ne; ++g) {
            double sg = r.ex[g] * ell;
            double p[3] = {pa[0] + sg * u[0] - x[0], pa[1] + sg * u[1] - x[1], pa[2] + sg * u[2] - x[2]};
            const double rho2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
            const double ri = rsqrt_nr<2>(rho2);
            const double rho = rho2 * ri;
            double jac = h * (ri * ri) * ell * r.ew[g];
            vl += rho * jac;
            vy += (kappa > 0 ? (1.0 - exp(-kappa * rho)) * inv_kappa : rho) * jac;
        }
    }
    const int bi = pbody[i];
    const bool lap = bd.kind[bi] == PGB_DIELECTRIC;
    out[e] = dbl4{lap ? vl / PGB_FOUR_PI : 0.0, 0.0, vy / PGB_FOUR_PI, 0.0};
}

BodyDev body_dev(const pgb_ctx* c) {
    BodyDev b;
    memset(&b, 0, sizeof(b));
    b.n_bodies = (int)c->bodies.size();
    for (int i = 0; i < b.n_bodies; ++i) {
        const auto& bb = c->bodies[i];
        b.kind[i] = bb.kind;
        b.eps_ratio[i] = bb.eps_in / c->eps_out;
        b.bc[i] = bb.bc;
        b.pan_off[i] = bb.pan_off;
        b.unk_off[i] = bb.unk_off;
        b.parent[i] = bb.parent;
    }
    b.pan_off[b.n_bodies] = c->n_pan;
    return b;
}

__global__ void k_dbl4_to_f4(const dbl4* a, float4* b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const dbl4 v = a[i];
        b[i] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
    }
}

// in_set (host, per body; nullptr: all bodies) restricts targets and sources
// to a region's boundary; kappa is the screening of the Yukawa values.
static void build_corr_part(pgb_ctx* c, bool cross, DBuf<int64_t>& off, DBuf<int32_t>& cj, DBuf<dbl4>& val,
                            DBuf<float4>& val32, int64_t& count, const int* in_set, double kappa) {
    cudaStream_t s = c->stream;
    int64_t n = c->n_pan;
    CorrArgs a;
    a.nchild = c->d_node_nchild; a.child = c->d_node_child; a.nstart = c->d_node_start; a.nend = c->d_node_end;
    a.clo = c->d_node_clo; a.chi = c->d_node_chi; a.a8 = c->d_node_a8; a.C = c->d_c; a.A = c->d_A;
    a.n_bodies = (int)c->bodies.size();
    for (int b = 0; b < a.n_bodies; ++b) {
        a.prob[b] = c->bodies[b].prob;
        a.in_set[b] = in_set ? in_set[b] : 1;
    }
    {
        // prefilter copies, and delta from the largest coordinate of the body
        // boxes (a difference of two FP32-rounded coordinates of size <= m
        // is off by at most 2^-23 m per axis; sqrt(3) for the distance, with
        // a factor 2 of room)
        const int64_t nn = c->n_nodes;
        c->d_corr_pf4.resize(n);
        c->d_corr_nlo4.resize(nn);
        c->d_corr_nhi4.resize(nn);
        k_corr_prefilter<<<nblk(std::max(n, nn), 256), 256, 0, s>>>(n, nn, c->d_c, c->d_A, c->d_node_clo,
                                                                    c->d_node_chi, c->d_node_a8, c->d_corr_pf4,
                                                                    c->d_corr_nlo4, c->d_corr_nhi4);
        const int nb = (int)c->bodies.size();
        std::vector<double> lo(3 * nb), hi(3 * nb);
        PGB_CUDA(cudaMemcpyAsync(lo.data(), c->d_node_clo.p, 24 * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(hi.data(), c->d_node_chi.p, 24 * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        double m = 0;
        for (int q = 0; q < 3 * nb; ++q) m = std::max(m, std::max(fabs(lo[q]), fabs(hi[q])));
        a.delta = (float)(2.0 * 1.7320508075688772 * ldexp(m, -23)) + 1e-30f;
        a.pf4 = c->d_corr_pf4;
        a.nlo4 = c->d_corr_nlo4;
        a.nhi4 = c->d_corr_nhi4;
    }
    DBuf<int64_t> cnt;
    cnt.resize(n);
    off.resize(n + 1);
    const int cap = PGB_CORR_CAP;
    c->d_corr_tmp.resize((size_t)n * cap + 1);
    int* ovf = (int*)(c->d_corr_tmp.p + (size_t)n * cap);
    PGB_CUDA(cudaMemsetAsync(ovf, 0, 4, s));
    k_corr_find<<<nblk(n, 32 * CORR_WARPS), 32 * CORR_WARPS, 0, s>>>(a, n, false, cross, c->d_pbody, cnt, nullptr,
                                                                     nullptr, c->d_corr_tmp, cap,
                                           ovf);
    PGB_CUDA(cudaGetLastError());
    int h_ovf = 0;
    PGB_CUDA(cudaMemcpyAsync(&h_ovf, ovf, 4, cudaMemcpyDeviceToHost, s));
    int64_t tot = 0;
    exclusive_scan_i64(cnt, off, n, s, &tot);  // synchronises: h_ovf is valid
    PGB_CUDA(cudaMemcpyAsync(off.p + n, &tot, 8, cudaMemcpyHostToDevice, s));
    count = tot;
    cj.resize(tot);
    val.resize(tot);
    if (tot) {
        if (h_ovf)
            k_corr_find<<<nblk(n, 32 * CORR_WARPS), 32 * CORR_WARPS, 0, s>>>(a, n, true, cross, c->d_pbody, nullptr,
                                                                             off, cj, nullptr, 0, nullptr);
        else
            k_corr_compact<<<nblk(n, 128), 128, 0, s>>>(n, off, c->d_corr_tmp, cap, cj);
        Rules r = make_rules(c->p.K, c->p.K_near, c->p.n_edge);
        c->d_yfine.resize(3 * n * r.Kn);
        k_fine_nodes<<<nblk(n * r.Kn, 256), 256, 0, s>>>(n, c->d_v, c->d_c, r, c->d_yfine);
        // both node sets split into double-single (8 bytes a value, as doubles)
        c->d_yfine_ds.resize(3 * n * r.Kn);
        c->d_y_ds.resize(3 * n * r.K);
        k_nodes_to_ds<<<nblk(3 * n * r.Kn, 256), 256, 0, s>>>(c->d_yfine, (ds*)c->d_yfine_ds.p, 3 * n * r.Kn);
        k_nodes_to_ds<<<nblk(3 * n * r.K, 256), 256, 0, s>>>(c->d_y, (ds*)c->d_y_ds.p, 3 * n * r.K);
        k_corr_values<<<nblk(tot, 128), 128, 0, s>>>(n, tot, off, cj, (const ds*)c->d_yfine_ds.p, c->d_c, c->d_n,
                                                     c->d_A, (const ds*)c->d_y_ds.p, c->d_w, c->d_pbody, body_dev(c),
                                                     r, kappa, val);
        if (!cross)
            k_corr_self<<<nblk(n, 128), 128, 0, s>>>(n, off, cj, c->d_v, c->d_c, c->d_pbody, body_dev(c), r,
                                                     kappa, val);
    }
    val32.resize(std::max<int64_t>(tot, 1));
    if (tot) k_dbl4_to_f4<<<nblk(tot, 256), 256, 0, s>>>(val, val32, tot);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    PGB_LAUNCHED(c, tot ? 7 : 2);
}

// Regions of a nested system (the solvent, then the interior of every
// dielectric body) with the bodies bounding each, and each region's
// near-field corrections at its own screening, among its boundary bodies.
static void build_regions(pgb_ctx* c) {
    const int nb = (int)c->bodies.size();
    c->regions.clear();
    for (int R = 0; R <= nb; ++R) {
        if (R > 0 && c->bodies[R - 1].kind != PGB_DIELECTRIC) continue;
        auto reg = std::make_unique<pgb_ctx::Region>();
        RegionDev& d = reg->dev;
        memset(&d, 0, sizeof(d));
        const double epsR = R == 0 ? c->eps_out : c->bodies[R - 1].eps_in;
        d.kappa = R == 0 ? c->kappa : c->bodies[R - 1].kappa_in;
        int in_set[PGB_MAX_BODIES] = {0};
        bool any = false;
        for (int b = 0; b < nb; ++b) {
            const auto& bb = c->bodies[b];
            const int outer = bb.parent < 0 ? 0 : bb.parent + 1;
            const int inner = bb.kind == PGB_DIELECTRIC ? b + 1 : -1;
            const int sg = inner == R ? 1 : (outer == R ? -1 : 0);
            d.sign[b] = sg;
            if (!sg) continue;
            any = true;
            in_set[b] = 1;
            d.fac[b] = sg > 0 ? 1.0 : (bb.kind == PGB_DIELECTRIC ? bb.eps_in / epsR : 1.0);
            d.psi_known[b] = bb.kind == PGB_SET_CHARGE ? -bb.bc / epsR : 0.0;
        }
        if (!any) continue;
        build_corr_part(c, false, reg->corr_off, reg->corr_j, reg->corr_val, reg->corr_val32, reg->n_corr, in_set,
                        d.kappa);
        build_corr_part(c, true, reg->xcorr_off, reg->xcorr_j, reg->xcorr_val, reg->xcorr_val32, reg->n_xcorr, in_set,
                        d.kappa);
        c->regions.push_back(std::move(reg));
    }
}

void build_corrections(pgb_ctx* c) {
    if (nested(c)) build_regions(c);
    else c->regions.clear();
    if (!c->intra_valid) {
        build_corr_part(c, false, c->d_corr_off, c->d_corr_j, c->d_corr_val, c->d_corr_val32, c->n_corr, nullptr,
                        c->kappa);
        c->intra_valid = true;
    }
    // cross-body entries: none when every pair of bodies of one problem is
    // farther apart (centroid boxes of the roots) than the larger 2L reach
    // (a8) of the two
    const int nb = (int)c->bodies.size();
    bool reach = false;
    if (nb > 1) {
        std::vector<double> lo(3 * nb), hi(3 * nb), a8(nb);
        cudaStream_t s = c->stream;
        PGB_CUDA(cudaMemcpyAsync(lo.data(), c->d_node_clo.p, 24 * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(hi.data(), c->d_node_chi.p, 24 * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(a8.data(), c->d_node_a8.p, 8 * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        for (int a = 0; a < nb && !reach; ++a)
            for (int b = a + 1; b < nb && !reach; ++b) {
                if (c->bodies[a].prob != c->bodies[b].prob) continue;
                double d2 = 0;
                for (int q = 0; q < 3; ++q) {
                    const double u = std::max(std::max(lo[3 * a + q] - hi[3 * b + q], lo[3 * b + q] - hi[3 * a + q]), 0.0);
                    d2 += u * u;
                }
                // the traversal's test is d2 < a8 with d2 >= this box distance
                reach = !(d2 >= std::max(a8[a], a8[b]) * 1.000001);
            }
    }
    if (reach) {
        build_corr_part(c, true, c->d_xcorr_off, c->d_xcorr_j, c->d_xcorr_val, c->d_xcorr_val32, c->n_xcorr, nullptr,
                        c->kappa);
    } else {
        c->d_xcorr_off.resize(c->n_pan + 1);
        PGB_CUDA(cudaMemsetAsync(c->d_xcorr_off.p, 0, 8 * (c->n_pan + 1), c->stream));
        c->d_xcorr_j.resize(1);
        c->d_xcorr_val.resize(1);
        c->d_xcorr_val32.resize(1);
        c->n_xcorr = 0;
    }
}

Geo geo(const pgb_ctx* c) {
    Geo g;
    g.n_pan = c->n_pan;
    g.n_src = c->n_pan * c->p.K;
    g.K = c->p.K;
    g.perm = c->d_perm; g.pbody = c->d_pbody; g.v = c->d_v; g.c = c->d_c; g.n = c->d_n; g.A = c->d_A;
    g.pleaf = c->d_pan_leaf; g.y = c->d_y; g.w = c->d_w;
    return g;
}

}  // namespace pgb
