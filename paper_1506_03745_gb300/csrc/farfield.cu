// Far-field coefficient tables of the M2P evaluation (Section 3.2: Cartesian
// Taylor expansion of order P about a node centre).
//
// The far field of a node is U(R) = sum_{|k|<=P} G_k(R) M_k with
// G_k = d^k G / k! and the node's moments M_k.  Per degree n the terms form
// mu_n(grad) G with the homogeneous polynomial mu_n(s) = sum_{|k|=n} M_k s^k / k!.
// Write mu_n = sum_m |s|^{2m} h_{n,m}(s) with harmonic h_{n,m} of degree
// n - 2m (Gauss decomposition).  Away from the source G satisfies
// Laplace(G) = kappa^2 G, so |grad|^{2m} acts as kappa^{2m}, and a harmonic
// polynomial h of degree d applied to a radial function gives
// h(grad) G = h(R) D^d G with D = (1/r) d/dr (Hobson's theorem).  Hence
//   U(R) = sum_p D^p G(r) E_p(R),  E_p = sum_m kappa^{2m} h_{p+2m,m},
// and with D^p (e^{-kappa r}/r) = e^{-x} r^{-(2p+1)} g_p(x), x = kappa r,
// g_0 = 1, g_1 = -(1 + x), g_{p+2} = x^2 g_p - (2p + 3) g_{p+1}:
//   U(R) = (e^{-x} / r) sum_p g_p(x) E_p(S),  S = R / r^2.
// Laplace (kappa = 0) keeps only m = 0 and g_p = (-1)^p (2p - 1)!!, which is
// folded into its table, so that U_L(R) = (1/r) sum_j e_j S^j.
//
// The decomposition: h_{n,m} = H_{n-2m}[Lap^m mu_n] / (2^m m! prod_{i=1..m}
// (2(n-2m) + 2i + 1)), with the harmonic projection of a homogeneous f of
// degree d H_d[f] = sum_j c_j |s|^{2j} Lap^j f, c_j = (-1)^j (2d-2j-1)!! /
// (2^j j! (2d-1)!!).  (Lap^m (|s|^{2m} h) = 2^m m! prod_i (2i + 2d + 1) h for
// harmonic h of degree d, and the other parts of mu_n project to zero.)
//
// Table layout (T = (P+1)(P+2)(P+3)/6): rows = output coefficients in the
// evaluation order (a = 0..P, b = 0..P-a, c = 0..P-a-b for S^(a,b,c)), columns
// = moments in the graded order of the upward pass (degree, then kx and ky
// descending); the Yukawa table (T x T) then the Laplace table (T x T).
#include <math.h>

#include <map>
#include <vector>

#include "pgb_internal.cuh"

namespace pgb {

namespace {

// position of (a, b, d-a-b) among the degree-d monomials (kx, then ky descending)
inline int pos(int d, int a, int b) { return (d - a) * (d - a + 1) / 2 + (d - a - b); }
inline int n_deg(int d) { return (d + 1) * (d + 2) / 2; }

using Poly = std::vector<double>;  // homogeneous polynomial of one degree, by pos()

Poly laplacian(int d, const Poly& f) {
    Poly out(d >= 2 ? n_deg(d - 2) : 0, 0.0);
    if (d < 2) return out;
    for (int a = 0; a <= d; ++a)
        for (int b = 0; b <= d - a; ++b) {
            const int c = d - a - b;
            const double v = f[pos(d, a, b)];
            if (v == 0.0) continue;
            if (a >= 2) out[pos(d - 2, a - 2, b)] += v * a * (a - 1);
            if (b >= 2) out[pos(d - 2, a, b - 2)] += v * b * (b - 1);
            if (c >= 2) out[pos(d - 2, a, b)] += v * c * (c - 1);
        }
    return out;
}

Poly times_r2(int d, const Poly& f) {
    Poly out(n_deg(d + 2), 0.0);
    for (int a = 0; a <= d; ++a)
        for (int b = 0; b <= d - a; ++b) {
            const double v = f[pos(d, a, b)];
            if (v == 0.0) continue;
            out[pos(d + 2, a + 2, b)] += v;
            out[pos(d + 2, a, b + 2)] += v;
            out[pos(d + 2, a, b)] += v;
        }
    return out;
}

double dfact(int n) {
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

double fact(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

// harmonic projection of the degree-d polynomial f
Poly harmonic(int d, const Poly& f) {
    Poly out = f;
    Poly g = f;
    for (int j = 1; 2 * j <= d; ++j) {
        g = laplacian(d - 2 * (j - 1), g);  // Lap^j f, degree d - 2j
        const double cj = ((j & 1) ? -1.0 : 1.0) * dfact(2 * d - 2 * j - 1) / (pow(2.0, j) * fact(j) * dfact(2 * d - 1));
        Poly t = g;
        for (int i = 0; i < j; ++i) t = times_r2(d - 2 * j + 2 * i, t);
        for (size_t q = 0; q < out.size(); ++q) out[q] += cj * t[q];
    }
    return out;
}

}  // namespace

void far_tables(int P, double kappa, std::vector<double>& tab) {
    const int T = n_terms(P);
    // evaluation-order index of every (a, b, c)
    std::vector<int> ev((P + 1) * (P + 1) * (P + 1), -1);
    int e = 0;
    for (int a = 0; a <= P; ++a)
        for (int b = 0; b <= P - a; ++b)
            for (int c = 0; c <= P - a - b; ++c) ev[(a * (P + 1) + b) * (P + 1) + c] = e++;
    tab.assign(2 * (size_t)T * T, 0.0);
    double* Y = tab.data();
    double* L = tab.data() + (size_t)T * T;
    for (int n = 0; n <= P; ++n) {
        for (int a = 0; a <= n; ++a)
            for (int b = 0; b <= n - a; ++b) {
                const int c = n - a - b;
                const int col = (n == 0 ? 0 : n_terms(n - 1)) + pos(n, a, b);
                Poly f(n_deg(n), 0.0);
                f[pos(n, a, b)] = 1.0 / (fact(a) * fact(b) * fact(c));
                for (int m = 0; 2 * m <= n; ++m) {
                    if (m > 0) f = laplacian(n - 2 * (m - 1), f);
                    const int d = n - 2 * m;
                    const Poly h = harmonic(d, f);
                    double norm = pow(2.0, m) * fact(m);
                    for (int i = 1; i <= m; ++i) norm *= 2 * i + 2 * d + 1;
                    const double ky = pow(kappa, 2 * m) / norm;
                    const double kl = ((d & 1) ? -1.0 : 1.0) * dfact(2 * d - 1) / norm;
                    for (int aa = 0; aa <= d; ++aa)
                        for (int bb = 0; bb <= d - aa; ++bb) {
                            const double v = h[pos(d, aa, bb)];
                            if (v == 0.0) continue;
                            const int row = ev[(aa * (P + 1) + bb) * (P + 1) + (d - aa - bb)];
                            Y[(size_t)row * T + col] += ky * v;
                            if (m == 0) L[(size_t)row * T + col] += kl * v;
                        }
                }
            }
    }
}

// Device copy of the tables for the context's P and the screening kappa
// (one per kappa: the solvent, and each region of a nested system), in FP64,
// double-single and FP32 (transposed dense, and packed for orders above 8).
const FarTab& far_table(pgb_ctx* c, double kappa) {
    for (const auto& t : c->far_tabs)
        if (t->P == c->p.P && t->kappa == kappa) return *t;
    std::vector<double> rowmajor;
    far_tables(c->p.P, kappa, rowmajor);
    // device layout: packed rows in the graded order of the moments, per row
    // the Yukawa entries over the moment degrees p, p + 2, ..., P then the
    // Laplace entries over degree p (k_far_coef)
    const int P = c->p.P, T = n_terms(P);
    std::vector<int> ev((P + 1) * (P + 1) * (P + 1), -1);
    {
        int e = 0;
        for (int a = 0; a <= P; ++a)
            for (int b = 0; b <= P - a; ++b)
                for (int cc = 0; cc <= P - a - b; ++cc) ev[(a * (P + 1) + b) * (P + 1) + cc] = e++;
    }
    std::vector<double> h;
    for (int n = 0; n <= P; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                const int row = ev[(a * (P + 1) + b) * (P + 1) + (n - a - b)];
                for (int q = n; q <= P; q += 2)
                    for (int k = (q > 0 ? n_terms(q - 1) : 0); k < n_terms(q); ++k)
                        h.push_back(rowmajor[(size_t)row * T + k]);
                for (int k = (n > 0 ? n_terms(n - 1) : 0); k < n_terms(n); ++k)
                    h.push_back(rowmajor[(size_t)T * T + (size_t)row * T + k]);
            }
    // FP32 layout: each table transposed, tab[k][j] with rows of far_tr(P)
    // columns (k_far_f32), Yukawa then Laplace
    const int TR = (((T + 3) & ~3) + 31) & ~31;
    std::vector<float> hf(2 * (size_t)T * TR, 0.f);
    for (int q = 0; q < 2; ++q)
        for (int j = 0; j < T; ++j)
            for (int k = 0; k < T; ++k)
                hf[(size_t)q * T * TR + (size_t)k * TR + j] = (float)rowmajor[(size_t)q * T * T + (size_t)j * T + k];
    auto t = std::make_unique<FarTab>();
    t->P = c->p.P;
    t->kappa = kappa;
    // double-single: hi = the FP32 rounding, lo = the FP32 rounding of the rest
    std::vector<float> hds(2 * h.size());
    for (size_t q = 0; q < h.size(); ++q) {
        const float hi = (float)h[q];
        hds[2 * q] = hi;
        hds[2 * q + 1] = (float)(h[q] - (double)hi);
    }
    std::vector<float> hp(h.size());
    for (size_t q = 0; q < h.size(); ++q) hp[q] = (float)h[q];
    t->t64.resize(h.size());
    t->t32.resize(hf.size());
    t->tds.resize(h.size());
    t->t32p.resize(hp.size());
    PGB_CUDA(cudaMemcpyAsync(t->t64.p, h.data(), 8 * h.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA(cudaMemcpyAsync(t->t32.p, hf.data(), 4 * hf.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA(cudaMemcpyAsync(t->tds.p, hds.data(), 4 * hds.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA(cudaMemcpyAsync(t->t32p.p, hp.data(), 4 * hp.size(), cudaMemcpyHostToDevice, c->stream));
    PGB_CUDA(cudaStreamSynchronize(c->stream));
    c->far_tabs.push_back(std::move(t));
    return *c->far_tabs.back();
}

}  // namespace pgb

extern "C" int pgb_far_table(int32_t P, double kappa, double* out, int64_t n) {
    if (P < 0 || P > PGB_MAX_P || !(kappa >= 0) || !out) return PGB_EINVAL;
    const int T = pgb::n_terms(P);
    if (n != 2 * (int64_t)T * T) return PGB_EINVAL;
    std::vector<double> tab;
    pgb::far_tables(P, kappa, tab);
    for (size_t i = 0; i < tab.size(); ++i) out[i] = tab[i];
    return PGB_OK;
}
