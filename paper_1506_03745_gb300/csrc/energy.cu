// Energies of Section 3.3 (Eq. 11-16) from a solution vector, FP64.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "pgb_internal.cuh"

namespace pgb {

// V_L and K_L (without the 1/4pi) of panel j (sorted index) at the point xq:
// the 19-point rule when |xq - c_j| < 2 L_j, else the K-point rule; 1/r by
// two Newton steps.
__device__ __forceinline__ void panel_vk(const Geo& g, const Rules& r, const double* xq, int64_t j, double& vl,
                                         double& kl) {
    const double* cj = g.c + 3 * j;
    const double* nj = g.n + 3 * j;
    double dx = xq[0] - cj[0], dy = xq[1] - cj[1], dz = xq[2] - cj[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    vl = 0;
    kl = 0;
    if (d2 < 8.0 * g.A[j]) {
        const double* v = g.v + 9 * j;
        for (int m = 0; m < r.Kn; ++m) {
            double y[3];
            for (int a = 0; a < 3; ++a)
                y[a] = cj[a] + ((r.mun[m][0] * (v[a] - cj[a]) + r.mun[m][1] * (v[3 + a] - cj[a])) +
                                r.mun[m][2] * (v[6 + a] - cj[a]));
            double ex = xq[0] - y[0], ey = xq[1] - y[1], ez = xq[2] - y[2];
            double ri = rsqrt_nr<2>(ex * ex + ey * ey + ez * ez);
            double w = r.wn[m] * g.A[j];
            vl += w * ri;
            kl += w * (nj[0] * ex + nj[1] * ey + nj[2] * ez) * ri * ri * ri;
        }
    } else {
        for (int m = 0; m < g.K; ++m) {
            const double* y = g.y + 3 * (j * g.K + m);
            double ex = xq[0] - y[0], ey = xq[1] - y[1], ez = xq[2] - y[2];
            double ri = rsqrt_nr<2>(ex * ex + ey * ey + ez * ez);
            double w = g.w[j * g.K + m];
            vl += w * ri;
            kl += w * (nj[0] * ex + nj[1] * ey + nj[2] * ez) * ri * ri * ri;
        }
    }
}

// Contribution of panel j (sorted index) of body b to phi_reac at xq
// (without the 1/4pi): -K_L phi + V_L dphi.
__device__ __forceinline__ double phi_panel(const Geo& g, const BodyDev& bd, const Rules& r, const double* xq,
                                            const double* x, int b, int64_t j) {
    const int64_t s0 = bd.pan_off[b], N = bd.pan_off[b + 1] - s0, o = bd.unk_off[b];
    const int64_t loc = g.perm[j] - s0;
    const double phi = x[o + loc], dphi = x[o + N + loc];
    double vl, kl;
    panel_vk(g, r, xq, j, vl, kl);
    return vl * dphi - kl * phi;
}

// Charge weights of every panel j of a dielectric body b (Eq. 13 summed over
// the charges first): sum_k q_k phi_reac(r_k) = sum_j (wV_j dphi_j - wK_j
// phi_j) with wV_j = sum_k q_k V_L(r_k, j), wK_j = sum_k q_k K_L(r_k, j)
// (without the 1/4pi), each pair with the rule of phi_panel.  The weights
// depend on the body's own mesh and charges only, so they hold for every
// rigid pose.  With nested interfaces a panel also bounds the interior of the
// body enclosing it (a cavity's panels bound the molecule's interior): its
// second pair of weights takes that body's charges.  One warp per panel,
// lanes over the charges.  w[j] = {wV own, wK own, wV enclosing, wK enclosing}.
// The same weights with one thread per panel over all its charges in order,
// for bodies of fewer than 32 charges (a warp per panel would leave most
// lanes idle, and the FP64 pipe takes whole warps).
__global__ void k_charge_weights_1t(Geo g, BodyDev bd, Rules r, const double* qxyz, const double* qv,
                                    const int64_t* qoff, dbl4* w) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= g.n_pan) return;
    const int b = g.pbody[j];
    double sv[2] = {0, 0}, sk[2] = {0, 0};
    for (int side = 0; side < 2; ++side) {
        const int src = side == 0 ? (bd.kind[b] == PGB_DIELECTRIC ? b : -1) : bd.parent[b];
        if (src < 0) continue;
        for (int64_t k = qoff[src]; k < qoff[src + 1]; ++k) {
            const double xq[3] = {qxyz[3 * k], qxyz[3 * k + 1], qxyz[3 * k + 2]};
            double vl, kl;
            panel_vk(g, r, xq, j, vl, kl);
            sv[side] += qv[k] * vl;
            sk[side] += qv[k] * kl;
        }
    }
    w[j] = dbl4{sv[0], sk[0], sv[1], sk[1]};
}

__global__ void k_charge_weights(Geo g, BodyDev bd, Rules r, const double* qxyz, const double* qv,
                                 const int64_t* qoff, dbl4* w) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= g.n_pan) return;
    const int b = g.pbody[j];
    double sv[2] = {0, 0}, sk[2] = {0, 0};
    for (int side = 0; side < 2; ++side) {
        const int src = side == 0 ? (bd.kind[b] == PGB_DIELECTRIC ? b : -1) : bd.parent[b];
        if (src < 0) continue;
        for (int64_t k = qoff[src] + lane; k < qoff[src + 1]; k += 32) {
            const double xq[3] = {qxyz[3 * k], qxyz[3 * k + 1], qxyz[3 * k + 2]};
            double vl, kl;
            panel_vk(g, r, xq, j, vl, kl);
            sv[side] += qv[k] * vl;
            sk[side] += qv[k] * kl;
        }
    }
    for (int side = 0; side < 2; ++side) {
        sv[side] = warp_sum(sv[side]);
        sk[side] = warp_sum(sk[side]);
    }
    if (lane == 0) w[j] = dbl4{sv[0], sk[0], sv[1], sk[1]};
}

// phi_reac(r_k) = -K_L(phi) + V_L(dphi) at each charge of a dielectric body
// (Eq. 13), three-tier rule with r_k as target: 19-point rule when
// |r_k - c_j| < 2 L_j, the K-point rule otherwise.  One block per charge.
__global__ void k_phi_reac(Geo g, BodyDev bd, Rules r, const double* qxyz, const int32_t* qbody, const double* x,
                           double* out) {
    __shared__ double sh[32];
    const int64_t k = blockIdx.x;
    const int b = qbody[k];
    const double xq[3] = {qxyz[3 * k], qxyz[3 * k + 1], qxyz[3 * k + 2]};
    double acc = 0;
    for (int64_t j = bd.pan_off[b] + threadIdx.x; j < bd.pan_off[b + 1]; j += blockDim.x)
        acc += phi_panel(g, bd, r, xq, x, b, j);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[k] = acc / PGB_FOUR_PI;
}

// The same sums split over blocks of PHI_CHUNK panels (grid: chunks x
// charges) for few charges: part[k * nch + chunk], reduced in chunk order by
// k_phi_reduce.
#define PHI_CHUNK 256
__global__ void __launch_bounds__(PHI_CHUNK) k_phi_reac_part(Geo g, BodyDev bd, Rules r, const double* qxyz,
                                                            const int32_t* qbody, const double* x, int nch,
                                                            double* part) {
    __shared__ double sh[32];
    const int64_t k = blockIdx.y;
    const int b = qbody[k];
    const double xq[3] = {qxyz[3 * k], qxyz[3 * k + 1], qxyz[3 * k + 2]};
    const int64_t j = bd.pan_off[b] + (int64_t)blockIdx.x * PHI_CHUNK + threadIdx.x;
    double acc = j < bd.pan_off[b + 1] ? phi_panel(g, bd, r, xq, x, b, j) : 0.0;
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[k * nch + blockIdx.x] = acc;
}
__global__ void k_phi_reduce(int64_t nq, int nch, const double* part, double* out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nq) return;
    double acc = 0;
    for (int i = 0; i < nch; ++i) acc += part[k * nch + i];
    out[k] = acc / PGB_FOUR_PI;
}

// phi_reac at every charge into out (device, n_q): the chunked kernels when
// the charges alone would not fill the GPU, else one block per charge.
static void launch_phi_reac(pgb_ctx* c, const Rules& r, const double* x, double* out) {
    int64_t nmax = 0;
    for (auto& b : c->bodies) nmax = std::max<int64_t>(nmax, b.N);
    const int nch = (int)std::max<int64_t>(1, (nmax + PHI_CHUNK - 1) / PHI_CHUNK);
    if (c->n_q < 1024 && c->n_q * nch <= ((int64_t)1 << 22)) {
        c->d_phi_part.resize((size_t)c->n_q * nch);
        k_phi_reac_part<<<dim3((unsigned)nch, (unsigned)c->n_q), PHI_CHUNK, 0, c->stream>>>(
            geo(c), body_dev(c), r, c->d_qxyz, c->d_q_body, x, nch, c->d_phi_part);
        k_phi_reduce<<<(unsigned)((c->n_q + 127) / 128), 128, 0, c->stream>>>(c->n_q, nch, c->d_phi_part, out);
        PGB_LAUNCHED(c, 1);
    } else {
        k_phi_reac<<<(unsigned)c->n_q, 128, 0, c->stream>>>(geo(c), body_dev(c), r, c->d_qxyz, c->d_q_body, x, out);
    }
    PGB_CUDA(cudaGetLastError());
}

// per-body sums: [0] sum q phi_reac over the body's own charges (from phir
// at the charges, or, when w is given, from the charge weights of the
// body's panels), [1] the part of the enclosing body's sum that this body's
// panels carry (nested interfaces; added to the enclosing body on the host),
// [2] sum_j u_j A_j (surfaces).  One block per body.  The Coulomb pair sum is
// k_coulomb_pairs (which overwrites [1] afterwards; energies() keeps [1]
// first).
__global__ void k_body_sums(Geo g, BodyDev bd, const double* qxyz, const double* qv, const int64_t* qoff,
                            const double* phir, const dbl4* w, const double* x, double* out) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    double s0 = 0, s1 = 0, s2 = 0;
    const int64_t p0 = bd.pan_off[b], p1 = bd.pan_off[b + 1], N = p1 - p0, o = bd.unk_off[b];
    if (!w) {
        for (int64_t k = qoff[b] + threadIdx.x; k < qoff[b + 1]; k += blockDim.x) s0 += qv[k] * phir[k];
    } else if (bd.kind[b] == PGB_DIELECTRIC) {
        // the enclosing body's interior sees this body from outside: sign -1
        // and the flux-scaled density (eps_in(b) / eps_in(parent)) dphi
        const int pb = bd.parent[b];
        const double f = pb >= 0 ? bd.eps_ratio[b] / bd.eps_ratio[pb] : 0.0;
        for (int64_t j = p0 + threadIdx.x; j < p1; j += blockDim.x) {
            const int64_t loc = g.perm[j] - p0;
            const double phi = x[o + loc], dphi = x[o + N + loc];
            s0 += w[j].x * dphi - w[j].y * phi;
            if (pb >= 0) s1 -= w[j].z * f * dphi - w[j].w * phi;
        }
        s0 *= 1.0 / PGB_FOUR_PI;
        s1 *= 1.0 / PGB_FOUR_PI;
    }
    if (bd.kind[b] != PGB_DIELECTRIC)
        for (int64_t j = p0 + threadIdx.x; j < p1; j += blockDim.x) s2 += x[o + (g.perm[j] - p0)] * g.A[j];
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        out[3 * b] = s0;
        out[3 * b + 1] = s1;
        out[3 * b + 2] = s2;
    }
}

// k_body_sums over BODY_PARTS blocks per body (blockIdx.y = body, blockIdx.x
// = part, panels strided over the parts), partial sums part[(b * BODY_PARTS +
// x) * 3 + {0, 1, 2}] reduced in part order by k_body_sums_final; the
// charge-weight path only (energies()).
#define BODY_PARTS 64
__global__ void k_body_sums_part(Geo g, BodyDev bd, const dbl4* w, const double* x, double* part) {
    __shared__ double sh[32];
    const int b = blockIdx.y;
    double s0 = 0, s1 = 0, s2 = 0;
    const int64_t p0 = bd.pan_off[b], p1 = bd.pan_off[b + 1], N = p1 - p0, o = bd.unk_off[b];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w && bd.kind[b] == PGB_DIELECTRIC) {
        const int pb = bd.parent[b];
        const double f = pb >= 0 ? bd.eps_ratio[b] / bd.eps_ratio[pb] : 0.0;
        for (int64_t j = first; j < p1; j += stride) {
            const int64_t loc = g.perm[j] - p0;
            const double phi = x[o + loc], dphi = x[o + N + loc];
            s0 += w[j].x * dphi - w[j].y * phi;
            if (pb >= 0) s1 -= w[j].z * f * dphi - w[j].w * phi;
        }
    }
    if (bd.kind[b] != PGB_DIELECTRIC)
        for (int64_t j = first; j < p1; j += stride) s2 += x[o + (g.perm[j] - p0)] * g.A[j];
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        double* q = part + 3 * ((int64_t)b * gridDim.x + blockIdx.x);
        q[0] = s0;
        q[1] = s1;
        q[2] = s2;
    }
}
__global__ void k_body_sums_final(const double* part, int nparts, double* out) {
    if (threadIdx.x >= 3) return;
    const int b = blockIdx.x;
    double t = 0;
    for (int k = 0; k < nparts; ++k) t += part[3 * ((int64_t)b * nparts + k) + threadIdx.x];
    // the charge-weight sums carry the 1/4pi of phi_reac (Eq. 13)
    out[3 * b + threadIdx.x] = threadIdx.x < 2 ? t * (1.0 / PGB_FOUR_PI) : t;
}

// Coulomb sum_{l>k} q_k q_l / r_kl of each body: one block per charge k,
// partial sums pair[k], then a per-body reduction.
__global__ void k_coulomb_pairs(const double* qxyz, const double* qv, const int32_t* qbody, const int64_t* qoff,
                                double* pair) {
    __shared__ double sh[32];
    const int64_t k = blockIdx.x;
    const int b = qbody[k];
    double s = 0;
    for (int64_t l = k + 1 + threadIdx.x; l < qoff[b + 1]; l += blockDim.x) {
        double dx = qxyz[3 * k] - qxyz[3 * l], dy = qxyz[3 * k + 1] - qxyz[3 * l + 1], dz = qxyz[3 * k + 2] - qxyz[3 * l + 2];
        s += qv[l] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) pair[k] = qv[k] * s;
}
__global__ void k_coulomb_reduce(const int64_t* qoff, const double* pair, double* out) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    double s = 0;
    for (int64_t k = qoff[b] + threadIdx.x; k < qoff[b + 1]; k += blockDim.x) s += pair[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[3 * b + 1] = s;
}

// e^2/(eps0 Angstrom) in kcal/mol from CODATA 2018
double energy_unit_kcal() {
    const double e = 1.602176634e-19, eps0 = 8.8541878128e-12, NA = 6.02214076e23;
    return e * e / (eps0 * 1e-10) * NA / 4184.0;
}

void energies(pgb_ctx* c, const double* x, pgb_energies* e, pgb_energies* per_body) {
    if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
    cudaStream_t s = c->stream;
    const int nb = (int)c->bodies.size();
    DBuf<double> sums;
    DBuf<int64_t> qoff;
    sums.resize(3 * nb);
    std::vector<int64_t> qo(nb + 1);
    for (int b = 0; b < nb; ++b) qo[b] = c->bodies[b].q_off;
    qo[nb] = c->n_q;
    qoff.resize(nb + 1);
    PGB_CUDA(cudaMemcpyAsync(qoff.p, qo.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    Rules r = make_rules(c->p.K, c->p.K_near, c->p.n_edge);
    // charge weights of the panels: computed once per tree, charges and rule,
    // then every solution costs one pass over the panels
    if (c->n_q) {
        const uint64_t key[4] = {c->tree_gen, c->config_gen, (uint64_t)c->p.K, (uint64_t)c->p.K_near};
        if (memcmp(key, c->qw_key, sizeof(key))) {
            c->d_qw.resize(c->n_pan);
            int64_t qmax = 0;
            for (const auto& bo : c->bodies) qmax = std::max<int64_t>(qmax, bo.nq);
            if (qmax < 32)
                k_charge_weights_1t<<<(unsigned)((c->n_pan + 127) / 128), 128, 0, s>>>(
                    geo(c), body_dev(c), r, c->d_qxyz, c->d_qval, qoff, c->d_qw);
            else
                k_charge_weights<<<(unsigned)((c->n_pan * 32 + 127) / 128), 128, 0, s>>>(
                    geo(c), body_dev(c), r, c->d_qxyz, c->d_qval, qoff, c->d_qw);
            PGB_CUDA(cudaGetLastError());
            PGB_LAUNCHED(c, 1);
            memcpy(c->qw_key, key, sizeof(key));
        }
    }
    {
        DBuf<double> part;
        part.resize((size_t)3 * BODY_PARTS * nb);
        k_body_sums_part<<<dim3(BODY_PARTS, nb), 128, 0, s>>>(geo(c), body_dev(c), c->n_q ? c->d_qw.p : nullptr, x,
                                                             part);
        k_body_sums_final<<<nb, 32, 0, s>>>(part, BODY_PARTS, sums);
        PGB_LAUNCHED(c, 1);
    }
    // the cavities' share of each body's reaction potential, before the
    // Coulomb reduction reuses slot [1]
    DBuf<double> inner;
    inner.resize(nb);
    PGB_CUDA(cudaMemcpy2DAsync(inner.p, 8, sums.p + 1, 24, 8, nb, cudaMemcpyDeviceToDevice, s));
    {
        DBuf<double> pair;
        pair.resize(std::max<int64_t>(1, c->n_q));
        if (c->n_q)
            k_coulomb_pairs<<<(unsigned)c->n_q, 128, 0, s>>>(c->d_qxyz, c->d_qval, c->d_q_body, qoff, pair);
        else
            PGB_CUDA(cudaMemsetAsync(pair.p, 0, 8, s));
        k_coulomb_reduce<<<nb, 128, 0, s>>>(qoff, pair, sums);
        PGB_CUDA(cudaGetLastError());
        PGB_CUDA(cudaStreamSynchronize(s));
    }
    PGB_LAUNCHED(c, c->n_q ? 3 : 2);
    std::vector<double> h(3 * nb), hin(nb);
    PGB_CUDA(cudaMemcpyAsync(h.data(), sums.p, 8 * 3 * nb, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(hin.data(), inner.p, 8 * nb, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    // each body's reaction-potential sum includes what its cavities carry
    for (int b = 0; b < nb; ++b)
        if (c->bodies[b].parent >= 0) h[3 * c->bodies[b].parent] += hin[b];
    const double U = energy_unit_kcal();
    pgb_energies tot{0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
        const auto& bd = c->bodies[b];
        pgb_energies eb{0, 0, 0, 0};
        if (bd.kind == PGB_DIELECTRIC) {
            eb.solvation = 0.5 * h[3 * b] * U;
            eb.coulomb = h[3 * b + 1] / (PGB_FOUR_PI * bd.eps_in) * U;
        } else if (bd.kind == PGB_SET_CHARGE) {
            eb.surface = 0.5 * bd.bc * h[3 * b + 2] * U;  // 1/2 sum phi_j sigma0 A_j
        } else {
            // -1/2 sum phi0 sigma_j A_j with sigma_j = -eps_out dphi_j
            eb.surface = 0.5 * c->eps_out * bd.bc * h[3 * b + 2] * U;
        }
        eb.total = eb.coulomb + eb.solvation + eb.surface;
        tot.coulomb += eb.coulomb;
        tot.solvation += eb.solvation;
        tot.surface += eb.surface;
        tot.total += eb.total;
        if (per_body) per_body[b] = eb;
    }
    if (e) *e = tot;
}

// ---------------------------------------------------------------- no-alloc path
// Scratch of pgb_energy_noalloc: reaction potentials at up to
// PGB_NOALLOC_MAX_CHARGES charges, then 3 sums per body, then the body charge
// offsets (PGB_MAX_BODIES + 1 int64 in double-sized slots).  Shared by every
// call in the process; held by every device that loads the library.
#define PGB_NOALLOC_SCRATCH (PGB_NOALLOC_MAX_CHARGES + 4 * PGB_MAX_BODIES + 1)
static __device__ __align__(256) double g_energy_scratch[PGB_NOALLOC_SCRATCH];

static std::mutex g_scratch_mu;
static double* g_scratch_ptr[64];
static bool g_scratch_ready[64];

// Device address of g_energy_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself: it names a host stand-in).
static double* energy_scratch() {
    int dev = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(PGB_EINVAL, "device ordinal out of range for the no-alloc scratch table");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ready[dev]) {
        double* p = nullptr;
        cudaError_t err = cudaGetSymbolAddress((void**)&p, g_energy_scratch);
        if (err != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            fail(PGB_ECUDA, std::string("cudaGetSymbolAddress(g_energy_scratch): ") + cudaGetErrorString(err));
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ready[dev] = true;
    }
    return g_scratch_ptr[dev];
}

// The solvation energy is summed per charge here (phi_reac at every charge,
// k_phi_reac, then the per-body sums), whereas energies() sums over the
// per-panel charge weights it caches; the two orders agree to rounding.
// Every buffer is either the context's or the static scratch, and the host
// side uses only stack arrays.
void energies_noalloc(pgb_ctx* c, const double* x, pgb_energies* e) {
    if (!c->tree_valid) fail(PGB_ESTATE, "pgb_tree_build has not run");
    if (c->n_q > PGB_NOALLOC_MAX_CHARGES)
        fail(PGB_EINVAL, "pgb_energy_noalloc handles at most " + std::to_string(PGB_NOALLOC_MAX_CHARGES) +
                             " charges; this context has " + std::to_string(c->n_q));
    double* scratch = energy_scratch();
    double* phir = scratch;
    double* sums = scratch + PGB_NOALLOC_MAX_CHARGES;
    cudaStream_t s = c->stream;
    const int nb = (int)c->bodies.size();
    int64_t qo[PGB_MAX_BODIES + 1];
    for (int b = 0; b < nb; ++b) qo[b] = c->bodies[b].q_off;
    qo[nb] = c->n_q;
    // the body charge offsets follow the sums (written before the kernels
    // read them, on the same stream)
    static_assert(sizeof(int64_t) == sizeof(double), "layout");
    int64_t* qoff = reinterpret_cast<int64_t*>(sums + 3 * PGB_MAX_BODIES);
    PGB_CUDA(cudaMemcpyAsync(qoff, qo, 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    Rules r = make_rules(c->p.K, c->p.K_near, c->p.n_edge);
    if (c->n_q) k_phi_reac<<<(unsigned)c->n_q, 128, 0, s>>>(geo(c), body_dev(c), r, c->d_qxyz, c->d_q_body, x, phir);
    k_body_sums<<<nb, 128, 0, s>>>(geo(c), body_dev(c), c->d_qxyz, c->d_qval, qoff, phir, nullptr, x, sums);
    PGB_CUDA(cudaGetLastError());
    // Coulomb pair sums, one block per charge, accumulated into the scratch
    // after the per-body sums (pair sums reuse the reaction-potential slots
    // only after k_body_sums has read them: same stream, in order)
    if (c->n_q) {
        k_coulomb_pairs<<<(unsigned)c->n_q, 128, 0, s>>>(c->d_qxyz, c->d_qval, c->d_q_body, qoff, phir);
    }
    k_coulomb_reduce<<<nb, 128, 0, s>>>(qoff, phir, sums);
    PGB_CUDA(cudaGetLastError());
    PGB_LAUNCHED(c, c->n_q ? 4 : 2);
    double h[3 * PGB_MAX_BODIES];
    PGB_CUDA(cudaMemcpyAsync(h, sums, 8 * 3 * nb, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    const double U = energy_unit_kcal();
    pgb_energies tot{0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
        const auto& bd = c->bodies[b];
        pgb_energies eb{0, 0, 0, 0};
        if (bd.kind == PGB_DIELECTRIC) {
            eb.solvation = 0.5 * h[3 * b] * U;
            eb.coulomb = h[3 * b + 1] / (PGB_FOUR_PI * bd.eps_in) * U;
        } else if (bd.kind == PGB_SET_CHARGE) {
            eb.surface = 0.5 * bd.bc * h[3 * b + 2] * U;
        } else {
            eb.surface = 0.5 * c->eps_out * bd.bc * h[3 * b + 2] * U;
        }
        eb.total = eb.coulomb + eb.solvation + eb.surface;
        tot.coulomb += eb.coulomb;
        tot.solvation += eb.solvation;
        tot.surface += eb.surface;
        tot.total += eb.total;
    }
    *e = tot;
}

// phi_reac (Eq. 13) at every charge into device doubles `out` (n_q entries).
void phi_reac(pgb_ctx* c, const double* x, double* out) {
    if (!c->n_q) return;
    Rules r = make_rules(c->p.K, c->p.K_near, c->p.n_edge);
    launch_phi_reac(c, r, x, out);
    PGB_LAUNCHED(c, 1);
}

}  // namespace pgb
