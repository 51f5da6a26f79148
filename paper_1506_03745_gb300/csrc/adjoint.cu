// Adjoint gradients of the total energy: transposed treecode, adjoint GMRES
// and the parameter derivatives (charges, imposed sigma0 / phi0, rigid
// translation of each body).  The paper has no gradient; the method is the
// discrete adjoint of Eq. 6 / Eq. 7 with the energies of Eq. 11-16.
#include <math.h>

#include <algorithm>
#include <vector>

#include "adjoint.cuh"

namespace pgb {

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------- set-up
// Unit normals and centroids relative to their leaf centre.
__global__ void k_adj_panels(int64_t n, const double* C, const double* Nn, const int32_t* pan_leaf,
                             const int32_t* leaf_node, const double* ncen, float4* n32, dbl4* n64, float4* c32,
                             dbl4* c64) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nd = leaf_node[pan_leaf[i]];
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = C[3 * i + a] - ncen[3 * nd + a];
    n32[i] = make_float4((float)Nn[3 * i], (float)Nn[3 * i + 1], (float)Nn[3 * i + 2], 0.f);
    n64[i] = dbl4{Nn[3 * i], Nn[3 * i + 1], Nn[3 * i + 2], 0.0};
    c32[i] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
    c64[i] = dbl4{d[0], d[1], d[2], 0.0};
}

// Transposed near-field corrections: CSR by source panel j, entries sorted by i.
__global__ void k_ct_count(int64_t n, const int64_t* off, const int32_t* cj, unsigned long long* cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) atomicAdd(cnt + cj[e], 1ull);
}
__global__ void k_ct_fill(int64_t n, const int64_t* off, const int32_t* cj, const dbl4* val, const int64_t* toff,
                          unsigned long long* cur, int32_t* ti, dbl4* tval) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        const int64_t j = cj[e];
        const int64_t pos = toff[j] + (int64_t)atomicAdd(cur + j, 1ull);
        ti[pos] = (int32_t)i;
        tval[pos] = val[e];
    }
}
__global__ void k_ct_sort(int64_t n, const int64_t* toff, int32_t* ti, dbl4* tval) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int64_t a = toff[j] + 1; a < toff[j + 1]; ++a) {
        const int32_t ki = ti[a];
        const dbl4 kv = tval[a];
        int64_t b = a - 1;
        while (b >= toff[j] && ti[b] > ki) {
            ti[b + 1] = ti[b];
            tval[b + 1] = tval[b];
            --b;
        }
        ti[b + 1] = ki;
        tval[b + 1] = kv;
    }
}
__global__ void k_i64_from_u64(const unsigned long long* a, int64_t* b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int64_t)a[i];
}

// group of every forward near entry
__global__ void k_entry_group(int64_t ng, const int64_t* noff, int32_t* eg) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    for (int64_t e = noff[g]; e < noff[g + 1]; ++e) eg[e] = (int32_t)g;
}
__global__ void k_tn_count(int64_t ne, const int32_t* nearl, unsigned long long* cnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < ne) atomicAdd(cnt + nearl[e], 1ull);
}
__global__ void k_tn_fill(int64_t ne, const int32_t* nearl, const int64_t* toff, unsigned long long* cur,
                          int64_t* te) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int nd = nearl[e];
    te[toff[nd] + (int64_t)atomicAdd(cur + nd, 1ull)] = e;
}
__global__ void k_tn_sort(int64_t nn, const int64_t* toff, int64_t* te) {  // insertion sort per node
    const int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (nd >= nn) return;
    for (int64_t a = toff[nd] + 1; a < toff[nd + 1]; ++a) {
        const int64_t v = te[a];
        int64_t b = a - 1;
        while (b >= toff[nd] && te[b] > v) {
            te[b + 1] = te[b];
            --b;
        }
        te[b + 1] = v;
    }
}

static void build_adjoint(pgb_ctx* c) {
    if (c->adj_valid) return;
    cudaStream_t s = c->stream;
    const int64_t n = c->n_pan, ng = c->n_groups;
    c->d_n32.resize(n); c->d_n64.resize(n); c->d_cT32.resize(n); c->d_cT64.resize(n);
    k_adj_panels<<<nblk(n, 128), 128, 0, s>>>(n, c->d_c, c->d_n, c->d_pan_leaf, c->d_leaf_node, c->d_node_center,
                                             c->d_n32, c->d_n64, c->d_cT32, c->d_cT64);
    PGB_CUDA(cudaGetLastError());
    // the forward near lists by source leaf: for every leaf node, the forward
    // near entries (group, leaf) that hold it, in entry (= group) order
    {
        const int64_t nn = c->n_nodes, ne = c->n_near;
        c->d_near_group.resize(std::max<int64_t>(ne, 1));
        k_entry_group<<<nblk(ng, 128), 128, 0, s>>>(ng, c->d_near_off, c->d_near_group);
        DBuf<unsigned long long> tcnt, tcur;
        tcnt.resize(nn);
        tcur.resize(nn);
        PGB_CUDA(cudaMemsetAsync(tcnt.p, 0, 8 * nn, s));
        PGB_CUDA(cudaMemsetAsync(tcur.p, 0, 8 * nn, s));
        k_tn_count<<<nblk(ne, 256), 256, 0, s>>>(ne, c->d_near, tcnt);
        DBuf<int64_t> t64;
        t64.resize(nn);
        k_i64_from_u64<<<nblk(nn, 256), 256, 0, s>>>(tcnt, t64, nn);
        c->d_tn_off.resize(nn + 1);
        int64_t tot_tn = 0;
        exclusive_scan_i64(t64, c->d_tn_off, nn, s, &tot_tn);
        PGB_CUDA(cudaMemcpyAsync(c->d_tn_off.p + nn, &tot_tn, 8, cudaMemcpyHostToDevice, s));
        if (tot_tn != ne) fail(PGB_EINVAL, "transposed near-list count mismatch");
        c->d_tn_e.resize(std::max<int64_t>(ne, 1));
        k_tn_fill<<<nblk(ne, 256), 256, 0, s>>>(ne, c->d_near, c->d_tn_off, tcur, c->d_tn_e);
        k_tn_sort<<<nblk(nn, 128), 128, 0, s>>>(nn, c->d_tn_off, c->d_tn_e);
        PGB_CUDA(cudaGetLastError());
    }
    // transpose the near-field corrections (intra + cross)
    const int64_t tot = c->n_corr + c->n_xcorr;
    DBuf<unsigned long long> cnt, cur;
    cnt.resize(n);
    cur.resize(n);
    PGB_CUDA(cudaMemsetAsync(cnt.p, 0, 8 * n, s));
    PGB_CUDA(cudaMemsetAsync(cur.p, 0, 8 * n, s));
    if (c->n_corr) k_ct_count<<<nblk(n, 128), 128, 0, s>>>(n, c->d_corr_off, c->d_corr_j, cnt);
    if (c->n_xcorr) k_ct_count<<<nblk(n, 128), 128, 0, s>>>(n, c->d_xcorr_off, c->d_xcorr_j, cnt);
    DBuf<int64_t> cnt64;
    cnt64.resize(n);
    k_i64_from_u64<<<nblk(n, 256), 256, 0, s>>>(cnt, cnt64, n);
    c->d_ct_off.resize(n + 1);
    int64_t t2 = 0;
    exclusive_scan_i64(cnt64, c->d_ct_off, n, s, &t2);
    PGB_CUDA(cudaMemcpyAsync(c->d_ct_off.p + n, &t2, 8, cudaMemcpyHostToDevice, s));
    if (t2 != tot) fail(PGB_EINVAL, "transposed correction count mismatch");
    c->d_ct_i.resize(tot);
    c->d_ct_val.resize(tot);
    if (c->n_corr)
        k_ct_fill<<<nblk(n, 128), 128, 0, s>>>(n, c->d_corr_off, c->d_corr_j, c->d_corr_val, c->d_ct_off, cur,
                                               c->d_ct_i, c->d_ct_val);
    if (c->n_xcorr)
        k_ct_fill<<<nblk(n, 128), 128, 0, s>>>(n, c->d_xcorr_off, c->d_xcorr_j, c->d_xcorr_val, c->d_ct_off, cur,
                                               c->d_ct_i, c->d_ct_val);
    k_ct_sort<<<nblk(n, 128), 128, 0, s>>>(n, c->d_ct_off, c->d_ct_i, c->d_ct_val);
    PGB_CUDA(cudaGetLastError());
    PGB_CUDA(cudaStreamSynchronize(s));
    PGB_LAUNCHED(c, 10);
    c->adj_valid = true;
}

// ---------------------------------------------------------------- A^T lam
// Per panel j: the K nodes' potentials and normal derivatives weighted by w_s
// (the transposed V and K products), the transposed near-field corrections,
// then the columns of A^T lam in the caller's layout.
__global__ void k_assemble_T(Geo g, BodyDev bd, const double* __restrict__ out4, const double* __restrict__ sT,
                             const int64_t* __restrict__ toff, const int32_t* __restrict__ ti,
                             const dbl4* __restrict__ tval, const double* __restrict__ lam, double* __restrict__ y) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= g.n_pan) return;
    double vl = 0, kl = 0, vy = 0, ky = 0;
    for (int m = 0; m < g.K; ++m) {
        const int64_t q = j * g.K + m;
        const double w = g.w[q];
        vl += w * out4[4 * q];
        kl += w * out4[4 * q + 1];
        vy += w * out4[4 * q + 2];
        ky += w * out4[4 * q + 3];
    }
    const double inv4pi = 1.0 / PGB_FOUR_PI;
    vl *= inv4pi;
    kl *= inv4pi;
    vy *= inv4pi;
    ky *= inv4pi;
    for (int64_t e = toff[j]; e < toff[j + 1]; ++e) {
        const int64_t i = ti[e];
        const dbl4 d = tval[e];
        vl += d.x * sT[2 * i];
        kl += d.y * sT[2 * i];
        vy += d.z * sT[2 * i + 1];
        ky += d.w * sT[2 * i + 1];
    }
    const int b = g.pbody[j];
    const int64_t loc = g.perm[j] - bd.pan_off[b], N = bd.pan_off[b + 1] - bd.pan_off[b], o = bd.unk_off[b];
    if (bd.kind[b] == PGB_DIELECTRIC) {
        const double l1 = lam[o + loc], l2 = lam[o + N + loc];
        y[o + loc] = 0.5 * l1 + kl + 0.5 * l2 - ky;
        y[o + N + loc] = -vl + bd.eps_ratio[b] * vy;
    } else if (bd.kind[b] == PGB_SET_CHARGE) {
        y[o + loc] = -ky + 0.5 * lam[o + loc];
    } else {
        y[o + loc] = vy;
    }
}

template <typename real, int P>
static void launch_T(pgb_ctx* c, const TArgs& ta0, const void* xrel, const void* yrel, const void* nrm, void* L) {
    using v4 = typename V4<real>::t;
    constexpr int T = MI<P>::T;
    constexpr int NW = 4;
    cudaStream_t s = c->stream;
    TArgs ta = ta0;
    PGB_CUDA(cudaMemsetAsync(L, 0, sizeof(real) * (size_t)c->n_nodes * 2 * T, s));
    k_p2p_T<real><<<(unsigned)std::max<int64_t>(ta.n_leaves, 1), 256, 0, s>>>(ta, (const v4*)xrel, c->d_sT,
                                                                                (const v4*)yrel, (const v4*)nrm);
    if (ta.n_fitems > 0)
        k_m2p_T<real, P, NW><<<(unsigned)ta.n_fitems, NW * 32, 0, s>>>(ta, (const v4*)xrel, c->d_sT, (real*)L);
    int launches = 3;
    for (size_t l = 0; l + 2 < c->level_begin.size(); ++l) {  // parents at level l push to level l + 1
        ta.lvl_begin = c->level_begin[l];
        ta.lvl_end = c->level_begin[l + 1];
        if (ta.lvl_end > ta.lvl_begin) {
            k_l2l_level<real, P><<<(unsigned)(ta.lvl_end - ta.lvl_begin), 256, 0, s>>>(ta, (real*)L);
            ++launches;
        }
    }
    k_l2p<real, P><<<(unsigned)std::max<int64_t>(ta.n_leaves, 1), 128, 0, s>>>(ta, (const v4*)yrel, (const v4*)nrm,
                                                                               (const real*)L);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, launches);
}

template <typename real>
static void dispatch_T(pgb_ctx* c, const TArgs& ta, const void* xrel, const void* yrel, const void* nrm, void* L) {
    switch (c->p.P) {
        case 0: launch_T<real, 0>(c, ta, xrel, yrel, nrm, L); break;
        case 1: launch_T<real, 1>(c, ta, xrel, yrel, nrm, L); break;
        case 2: launch_T<real, 2>(c, ta, xrel, yrel, nrm, L); break;
        case 3: launch_T<real, 3>(c, ta, xrel, yrel, nrm, L); break;
        case 4: launch_T<real, 4>(c, ta, xrel, yrel, nrm, L); break;
        case 5: launch_T<real, 5>(c, ta, xrel, yrel, nrm, L); break;
        case 6: launch_T<real, 6>(c, ta, xrel, yrel, nrm, L); break;
        case 7: launch_T<real, 7>(c, ta, xrel, yrel, nrm, L); break;
        case 8: launch_T<real, 8>(c, ta, xrel, yrel, nrm, L); break;
        default: fail(PGB_EINVAL, "the transposed treecode takes P in 0..8");
    }
}

// Row weights of the transposed product: s_L = lam of the interior (Laplace)
// row of a molecule panel, s_Y = lam of its exterior row or of a surface row.
__global__ void k_sT(Geo g, BodyDev bd, const double* __restrict__ lam, double* __restrict__ sT) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b], N = bd.pan_off[b + 1] - bd.pan_off[b], o = bd.unk_off[b];
    double sL = 0, sY;
    if (bd.kind[b] == PGB_DIELECTRIC) {
        sL = lam[o + loc];
        sY = lam[o + N + loc];
    } else {
        sY = lam[o + loc];
    }
    sT[2 * i] = sL;
    sT[2 * i + 1] = sY;
}

void apply_transpose(pgb_ctx* c, const double* lam, double* y, int precision) {
    if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
    build_adjoint(c);
    cudaStream_t s = c->stream;
    Geo g = geo(c);
    BodyDev bd = body_dev(c);
    const int64_t n = c->n_pan, K = c->p.K;
    const int T = n_terms(c->p.P);
    TArgs ta;
    ta.n_groups = c->n_groups;
    ta.gstart = c->d_group_start; ta.gend = c->d_group_end; ta.gbody = c->d_group_body;
    ta.gcenter = c->d_group_center; ta.ncenter = c->d_node_center;
    ta.nstart = c->d_node_start; ta.nend = c->d_node_end; ta.nbody = c->d_node_body;
    ta.nchild = c->d_node_nchild; ta.child = c->d_node_child;
    ta.K = (int)K;
    ta.kappa = c->kappa;
    for (int b = 0; b < PGB_MAX_BODIES; ++b) ta.lap_body[b] = 0;
    for (size_t b = 0; b < c->bodies.size(); ++b) ta.lap_body[b] = c->bodies[b].kind == PGB_DIELECTRIC;
    ta.n_fitems = c->n_fitems;
    ta.far_off = c->d_far_off; ta.fitem_off = c->d_fitem_off; ta.far_l = c->d_far; ta.fitem_group = c->d_fitem_group;
    ta.far4 = c->d_far4;
    ta.m2p_item = c->p.m2p_item;
    ta.tn_off = c->d_tn_off; ta.tn_e = c->d_tn_e; ta.near_group = c->d_near_group; ta.near4 = c->d_near4;
    ta.near_l = c->d_near;
    ta.n_leaves = c->n_leaves;
    ta.leaf_node = c->d_leaf_node;
    ta.lvl_begin = ta.lvl_end = 0;
    c->d_Tout.resize(4 * n * K);
    ta.out = c->d_Tout;
    c->d_sT.resize(2 * n);
    k_sT<<<nblk(n, 128), 128, 0, s>>>(g, bd, lam, c->d_sT);
    if (precision == PGB_FP32) {
        c->d_momT32.resize((size_t)c->n_nodes * 2 * T);
        dispatch_T<float>(c, ta, c->d_x32, c->d_y32, c->d_n32, c->d_momT32);
    } else {
        c->d_momT64.resize((size_t)c->n_nodes * 2 * T);
        dispatch_T<double>(c, ta, c->d_x64, c->d_y64, c->d_n64, c->d_momT64);
    }
    k_assemble_T<<<nblk(n, 128), 128, 0, s>>>(g, bd, c->d_Tout, c->d_sT, c->d_ct_off, c->d_ct_i, c->d_ct_val, lam, y);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 2);
}

// ---------------------------------------------------------------- dF/dx
// g = dF/dx: molecule panel j: -1/2 sum_k q_k K_L,kj on phi, 1/2 sum_k q_k V_L,kj on
// dphi (the charge rows of Eq. 13, three tiers); surface panel: 1/2 beta A_j,
// beta = sigma0 or eps_out phi0.  One block per panel.
__global__ void k_dFdx(Geo g, BodyDev bd, Rules r, const double* qxyz, const double* qv, const int64_t* qoff,
                       double eps_out, double* gx) {
    __shared__ double sh[32];
    const int64_t j = blockIdx.x;
    if (j >= g.n_pan) return;
    const int b = g.pbody[j];
    const int64_t loc = g.perm[j] - bd.pan_off[b], N = bd.pan_off[b + 1] - bd.pan_off[b], o = bd.unk_off[b];
    if (bd.kind[b] != PGB_DIELECTRIC) {
        if (threadIdx.x == 0) {
            const double beta = bd.kind[b] == PGB_SET_CHARGE ? bd.bc[b] : eps_out * bd.bc[b];
            gx[o + loc] = 0.5 * beta * g.A[j];
        }
        return;
    }
    const double* cj = g.c + 3 * j;
    const double* nj = g.n + 3 * j;
    const double* v = g.v + 9 * j;
    double sv = 0, sk = 0;
    for (int64_t k = qoff[b] + threadIdx.x; k < qoff[b + 1]; k += blockDim.x) {
        const double* xq = qxyz + 3 * k;
        double dx = xq[0] - cj[0], dy = xq[1] - cj[1], dz = xq[2] - cj[2];
        double vl = 0, kl = 0;
        const bool near = dx * dx + dy * dy + dz * dz < 8.0 * g.A[j];
        const int M = near ? r.Kn : g.K;
        for (int m = 0; m < M; ++m) {
            double y[3], w;
            if (near) {
                for (int a = 0; a < 3; ++a)
                    y[a] = cj[a] + ((r.mun[m][0] * (v[a] - cj[a]) + r.mun[m][1] * (v[3 + a] - cj[a])) +
                                    r.mun[m][2] * (v[6 + a] - cj[a]));
                w = r.wn[m] * g.A[j];
            } else {
                for (int a = 0; a < 3; ++a) y[a] = g.y[3 * (j * g.K + m) + a];
                w = g.w[j * g.K + m];
            }
            double ex = xq[0] - y[0], ey = xq[1] - y[1], ez = xq[2] - y[2];
            double rr = sqrt(ex * ex + ey * ey + ez * ez), ri = 1.0 / rr;
            vl += w * ri;
            kl += w * (nj[0] * ex + nj[1] * ey + nj[2] * ez) * ri * ri * ri;
        }
        sv += qv[k] * vl;
        sk += qv[k] * kl;
    }
    sv = block_sum(sv, sh);
    sk = block_sum(sk, sh);
    if (threadIdx.x == 0) {
        gx[o + loc] = -0.5 * sk / PGB_FOUR_PI;
        gx[o + N + loc] = 0.5 * sv / PGB_FOUR_PI;
    }
}

// dF/dq_k (internal units): Coulomb potential of the body's other charges +
// 1/2 phi_reac(r_k) + (1/eps_in) sum_i lam_i / (4 pi |c_i - r_k|) over the
// interior rows.  One block per charge.
__global__ void k_dq(Geo g, BodyDev bd, const double* qxyz, const double* qv, const int32_t* qbody,
                     const int64_t* qoff, const double* eps_in, const double* phir, const double* lam, double* dq) {
    __shared__ double sh[32];
    const int64_t k = blockIdx.x;
    const int b = qbody[k];
    const double* xk = qxyz + 3 * k;
    double s_coul = 0, s_lam = 0;
    for (int64_t l = qoff[b] + threadIdx.x; l < qoff[b + 1]; l += blockDim.x) {
        if (l == k) continue;
        double dx = xk[0] - qxyz[3 * l], dy = xk[1] - qxyz[3 * l + 1], dz = xk[2] - qxyz[3 * l + 2];
        s_coul += qv[l] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    const int64_t p0 = bd.pan_off[b], p1 = bd.pan_off[b + 1], o = bd.unk_off[b];
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        const double lam1 = lam[o + (g.perm[i] - p0)];
        double dx = g.c[3 * i] - xk[0], dy = g.c[3 * i + 1] - xk[1], dz = g.c[3 * i + 2] - xk[2];
        s_lam += lam1 / sqrt(dx * dx + dy * dy + dz * dz);
    }
    s_coul = block_sum(s_coul, sh);
    s_lam = block_sum(s_lam, sh);
    if (threadIdx.x == 0)
        dq[k] = (s_coul + s_lam) / (PGB_FOUR_PI * eps_in[b]) + 0.5 * phir[k];
}

// ---------------------------------------------------------------- dF/dt
// Full Yukawa densities of every panel (imposed parts included) as per-node
// source terms {w psi_Y, w phi_Y n}, and the adjoint weight of each panel's
// Yukawa row.
__global__ void k_full_src(Geo g, BodyDev bd, const double* x, const double* lam, double eps_out, float4* fsrc,
                           double* lamY) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n_pan) return;
    const int b = g.pbody[i];
    const int64_t loc = g.perm[i] - bd.pan_off[b], N = bd.pan_off[b + 1] - bd.pan_off[b], o = bd.unk_off[b];
    double psi, phi;
    if (bd.kind[b] == PGB_DIELECTRIC) {
        phi = x[o + loc];
        psi = bd.eps_ratio[b] * x[o + N + loc];
        lamY[i] = lam[o + N + loc];
    } else if (bd.kind[b] == PGB_SET_CHARGE) {
        phi = x[o + loc];
        psi = -bd.bc[b] / eps_out;
        lamY[i] = lam[o + loc];
    } else {
        psi = x[o + loc];
        phi = bd.bc[b];
        lamY[i] = lam[o + loc];
    }
    for (int m = 0; m < g.K; ++m) {
        const int64_t p = i * g.K + m;
        const double w = g.w[p];
        fsrc[p] = make_float4((float)(w * psi), (float)(w * phi * g.n[3 * i]), (float)(w * phi * g.n[3 * i + 1]),
                              (float)(w * phi * g.n[3 * i + 2]));
    }
}

// sum over the targets i of one group (body a) of lamY_i grad U^(b)(c_i), with
// U^(b) the Yukawa potential of body b's full densities (K-point rule; the
// bodies are farther apart than 2L).  grad of G_Y = -(1 + k r) e d / r^3 and of
// p.grad_y G_Y = (1 + k r) e p / r^3 - (k^2 r^2 + 3 k r + 3) e (p.d) d / r^5,
// d = x - y (without 1/4pi).  8 warps share the source tiles; FP32 with FP64
// offsets per point.
__global__ void __launch_bounds__(256) k_cross_grad(Geo g, const float4* __restrict__ xrel,
                                                    const double* __restrict__ gcen, const int32_t* __restrict__ gstart,
                                                    const int32_t* __restrict__ gend, int64_t g0, int64_t src0,
                                                    int64_t src1, const float4* __restrict__ fsrc,
                                                    const double* __restrict__ lamY, double kappa, double* out3) {
    __shared__ float4 sP[8][32], sQ[8][32];
    __shared__ double red[8][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gi = g0 + blockIdx.x;
    const int64_t p0 = gstart[gi], p1 = gend[gi];
    const int64_t p = p0 + lane;
    const bool active = p < p1;
    const float4 x = xrel[active ? p : p0];
    const double c0 = gcen[3 * gi], c1 = gcen[3 * gi + 1], c2 = gcen[3 * gi + 2];
    const float k = (float)kappa;
    float acc[3] = {0, 0, 0}, cmp[3] = {0, 0, 0};
    for (int64_t t = src0 + 32 * w; t < src1; t += 32 * 8) {
        const int cnt = (int)min((int64_t)32, src1 - t);
        __syncwarp();
        if (lane < cnt) {
            const int64_t q = t + lane;
            sP[w][lane] = make_float4((float)(g.y[3 * q] - c0), (float)(g.y[3 * q + 1] - c1),
                                      (float)(g.y[3 * q + 2] - c2), 0.f);
            sQ[w][lane] = fsrc[q];
        }
        __syncwarp();
        float tg[3] = {0, 0, 0};
        for (int j = 0; j < cnt; ++j) {
            const float4 Y = sP[w][j], S = sQ[w][j];
            const float dx = x.x - Y.x, dy = x.y - Y.y, dz = x.z - Y.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float ri = rsqrt_fast(r2);
            const float r = r2 * ri;
            const float ex = exp2_(-k * r * 1.4426950408889634f);
            const float ri3 = ri * ri * ri;
            const float a1 = (1.f + k * r) * ex * ri3;                       // (1 + k r) e / r^3
            const float a2 = (k * k * r2 + 3.f * k * r + 3.f) * ex * ri3 * ri * ri;
            const float pd = S.y * dx + S.z * dy + S.w * dz;
            // grad U = -q a1 d - (a1 p - a2 (p.d) d)
            const float cd = -S.x * a1 + a2 * pd;
            tg[0] += cd * dx - a1 * S.y;
            tg[1] += cd * dy - a1 * S.z;
            tg[2] += cd * dz - a1 * S.w;
        }
        for (int a = 0; a < 3; ++a) kadd(acc[a], cmp[a], tg[a]);
    }
    const double lw = active ? lamY[p] : 0.0;
    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = lw * ((double)acc[a] + (double)cmp[a]);
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) red[w][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int q = 0; q < 8; ++q) s += red[q][threadIdx.x];
        atomicAdd(out3 + threadIdx.x, s / PGB_FOUR_PI);
    }
}

// ---------------------------------------------------------------- driver
void grad(pgb_ctx* c, const double* x, int precision, double tol, int max_iter, int restart, double* dq, double* dbc,
          double* dt, pgb_solve_stats* st) {
    if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
    if (c->n_xcorr) fail(PGB_EINVAL, "gradients need the bodies farther apart than 2L (cross-body near entries exist)");
    if (precision != PGB_FP32 && precision != PGB_FP64) fail(PGB_EINVAL, "precision must be PGB_FP32 or PGB_FP64");
    cudaStream_t s = c->stream;
    const int64_t n = c->n_unk, np = c->n_pan;
    const int nb = (int)c->bodies.size();
    Geo g = geo(c);
    BodyDev bd = body_dev(c);
    Rules r = make_rules(c->p.K, c->p.K_near, c->p.n_edge);
    std::vector<int64_t> qo(nb + 1);
    std::vector<double> eps(nb);
    for (int b = 0; b < nb; ++b) {
        qo[b] = c->bodies[b].q_off;
        eps[b] = c->bodies[b].eps_in;
    }
    qo[nb] = c->n_q;
    DBuf<int64_t> qoff;
    DBuf<double> deps;
    qoff.resize(nb + 1);
    deps.resize(nb);
    PGB_CUDA(cudaMemcpyAsync(qoff.p, qo.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(deps.p, eps.data(), 8 * nb, cudaMemcpyHostToDevice, s));
    // adjoint system A^T lam = dF/dx
    c->d_gx.resize(n);
    c->d_lam.resize(n);
    k_dFdx<<<(unsigned)np, 128, 0, s>>>(g, bd, r, c->d_qxyz, c->d_qval, qoff, c->eps_out, c->d_gx);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, 1);
    c->d_V.resize((size_t)(restart + 1) * n);
    c->d_red.resize((size_t)304 * (restart + 1));
    PGB_CUDA(cudaMemsetAsync(c->d_lam.p, 0, 8 * n, s));
    precond_prepare(c);
    double gnorm = sqrt(vec_dot(c, c->d_gx, c->d_gx));
    pgb_solve_stats z{};
    if (gnorm > 0) {
        int mv = 0;
        z.iterations = gmres_op(c, precision, true, c->d_gx, c->d_lam, tol * gnorm, max_iter, restart, &mv, nullptr, true);
        z.matvecs = mv;
        z.matvecs_fp64 = precision == PGB_FP64 ? mv : 0;
        // true residual of the adjoint system
        c->d_r.resize(n);
        apply_transpose(c, c->d_lam, c->d_r, precision);
        ++z.matvecs;
        if (precision == PGB_FP64) ++z.matvecs_fp64;
        std::vector<double> hr(n), hg(n);
        PGB_CUDA(cudaMemcpyAsync(hr.data(), c->d_r.p, 8 * n, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(hg.data(), c->d_gx.p, 8 * n, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        double rr = 0;
        for (int64_t i = 0; i < n; ++i) rr += (hg[i] - hr[i]) * (hg[i] - hr[i]);
        z.rel_residual = sqrt(rr) / gnorm;
    }
    z.outer_steps = 1;
    if (st) *st = z;
    const double U = energy_unit_kcal();
    // charges
    if (dq && c->n_q) {
        DBuf<double> phir, d;
        phir.resize(c->n_q);
        d.resize(c->n_q);
        phi_reac(c, x, phir);
        k_dq<<<(unsigned)c->n_q, 128, 0, s>>>(g, bd, c->d_qxyz, c->d_qval, c->d_q_body, qoff, deps, phir, c->d_lam, d);
        PGB_CUDA(cudaGetLastError());
        PGB_LAUNCHED(c, 1);
        std::vector<double> hq(c->n_q);
        PGB_CUDA(cudaMemcpyAsync(hq.data(), d.p, 8 * c->n_q, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        for (auto& b : c->bodies)
            for (int64_t k = 0; k < b.nq; ++k) dq[b.q_off + k] = hq[b.q_off + k] * U;
    }
    // imposed sigma0 / phi0: 1/2 fac sum A u + lam . b_known(bc = 1)
    if (dbc) {
        DBuf<double> sums;
        std::vector<double> h(3 * nb);
        for (int b = 0; b < nb; ++b) {
            dbc[b] = 0.0;
            if (c->bodies[b].kind == PGB_DIELECTRIC) continue;
            int mask[PGB_MAX_BODIES] = {0};
            mask[b] = 1;
            const double saved = c->bodies[b].bc;
            c->bodies[b].bc = 1.0;
            c->d_bu.resize(n);
            PGB_CUDA(cudaMemsetAsync(c->d_bu.p, 0, 8 * n, s));
            try {
                apply_operator(c, nullptr, c->d_bu, precision, true, mask);
            } catch (...) {
                c->bodies[b].bc = saved;
                throw;
            }
            c->bodies[b].bc = saved;
            const double lb = vec_dot(c, c->d_lam, c->d_bu);
            // sum_j A_j u_j for this surface
            std::vector<double> hx(c->bodies[b].N), hA(np);
            PGB_CUDA(cudaMemcpyAsync(hx.data(), x + c->bodies[b].unk_off, 8 * c->bodies[b].N, cudaMemcpyDeviceToHost, s));
            std::vector<int32_t> hperm(np);
            PGB_CUDA(cudaMemcpyAsync(hA.data(), c->d_A.p, 8 * np, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaMemcpyAsync(hperm.data(), c->d_perm.p, 4 * np, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            double su = 0;
            for (int64_t i = c->bodies[b].pan_off; i < c->bodies[b].pan_off + c->bodies[b].N; ++i)
                su += hA[i] * hx[hperm[i] - c->bodies[b].pan_off];
            const double fac = c->bodies[b].kind == PGB_SET_CHARGE ? 1.0 : c->eps_out;
            const double e = 1.602176634e-19, eps0 = 8.8541878128e-12;
            const double conv = c->bodies[b].kind == PGB_SET_CHARGE ? 1e-20 / e : eps0 * 1e-10 / e;
            dbc[b] = (0.5 * fac * su + lb) * conv * U;
        }
    }
    // translations
    if (dt) {
        DBuf<float4> fsrc;
        DBuf<double> lamY, acc;
        fsrc.resize(np * c->p.K);
        lamY.resize(np);
        acc.resize(3 * nb * nb);
        PGB_CUDA(cudaMemsetAsync(acc.p, 0, 8 * 3 * nb * nb, s));
        k_full_src<<<nblk(np, 128), 128, 0, s>>>(g, bd, x, c->d_lam, c->eps_out, fsrc, lamY);
        for (int a = 0; a < nb; ++a)
            for (int b = 0; b < nb; ++b) {
                if (a == b) continue;
                const int64_t g0 = c->group_begin[a], g1 = c->group_begin[a + 1];
                if (g1 <= g0) continue;
                k_cross_grad<<<(unsigned)(g1 - g0), 256, 0, s>>>(
                    g, c->d_x32, c->d_group_center, c->d_group_start, c->d_group_end, g0,
                    c->bodies[b].pan_off * c->p.K, (c->bodies[b].pan_off + c->bodies[b].N) * c->p.K, fsrc, lamY,
                    c->kappa, acc.p + 3 * (a * nb + b));
                PGB_LAUNCHED(c, 1);
            }
        PGB_CUDA(cudaGetLastError());
        std::vector<double> h(3 * nb * nb);
        PGB_CUDA(cudaMemcpyAsync(h.data(), acc.p, 8 * 3 * nb * nb, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        for (int m = 0; m < nb; ++m)
            for (int ax = 0; ax < 3; ++ax) {
                double v = 0;
                for (int b = 0; b < nb; ++b)
                    if (b != m) v -= h[3 * (m * nb + b) + ax];
                for (int a = 0; a < nb; ++a)
                    if (a != m) v += h[3 * (a * nb + m) + ax];
                dt[3 * m + ax] = v * U;
            }
    }
    PGB_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pgb
