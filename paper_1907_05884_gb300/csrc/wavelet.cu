// wavelet.cu -- the multiwavelet spaces W_{s,q} of the per-column basis choice of Algorithm 1
// (Sec. 4.2, Fig. 3): host construction of the basis, its conversion to local Legendre
// expansions on the finest cells, and the design matrix of the fit on the grid nodes.
//
// W_{s,q} holds the piecewise polynomials of degree <= q on the 2^s equal cells of [-1, 1].
// Its orthonormal basis (inner product <f, g> = 1/2 int f g dt): the Legendre functions
// phi_0 .. phi_q (phi_n = sqrt(2n+1) L_n) on the whole interval, and for each level
// l = 0 .. s-1 and cell c of that level the wavelets psi_{l,c,i}(t) = 2^{l/2} psi_i(u),
// u = 2^l (t + 1) - 2c - 1, i = 0 .. q.  The mother wavelets psi_i are piecewise polynomials
// of degree <= q on the two halves of [-1, 1], orthogonal to every polynomial of degree <= q:
// sgn(t) phi_i(t), i = 0 .. q in order, orthogonalised against phi_0 .. phi_q and the earlier
// psi and normalised.  Function index: n for phi_n, (q+1)(2^l + c) + i for psi_{l,c,i}.
//
// A coordinate lies in finest cell f when f interior boundaries lo + ((hi - lo) c) 2^-s
// (c = 1 .. 2^s - 1) are at or below it (exact comparisons); the cell of level l is
// f >> (s - l) and the half of its level-l cell is bit s - l - 1 of f.
#include <math.h>

#include <vector>

#include "fst_internal.cuh"

namespace fst {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on L_n from the Chebyshev guesses).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 0 ? 1.0 : p1, pm = n == 0 ? 0.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// phi_0 .. phi_q at t (orthonormal Legendre functions)
static void legendre_ortho(double t, int q, double* out) {
    double Lm = 1.0, L = t;
    for (int n = 0; n <= q; ++n) {
        double v;
        if (n == 0) {
            v = 1.0;
        } else if (n == 1) {
            v = t;
        } else {
            v = ((2.0 * n - 1.0) * t * L - (n - 1.0) * Lm) / n;
            Lm = L;
            L = v;
        }
        out[n] = v * sqrt(2.0 * n + 1.0);
    }
}

// a[(i * 2 + h) * (q + 1) + m]: psi_i(t) = sum_m a phi_m(tau) on half h (h = 0: t < 0,
// tau = 2t + 1; h = 1: tau = 2t - 1).  Coordinates in the orthonormal basis
// sqrt(2) phi_m(tau) of each half, by Gauss-Legendre quadrature.
std::vector<double> mother_wavelets(int q) {
    const int nq = q + 1, G = q + 2, D = 2 * nq;
    std::vector<double> xg, wg;
    gauss_legendre(G, xg, wg);
    std::vector<double> ph(nq), pt(nq);
    // coordinates of f (values at the nodes of both halves) in that basis
    auto coords = [&](auto&& f) {
        std::vector<double> c(D, 0.0);
        for (int h = 0; h < 2; ++h)
            for (int g = 0; g < G; ++g) {
                const double t = h == 0 ? (xg[g] - 1.0) / 2.0 : (xg[g] + 1.0) / 2.0;
                legendre_ortho(xg[g], q, ph.data());
                const double fv = f(t);
                for (int m = 0; m < nq; ++m) c[h * nq + m] += sqrt(2.0) / 4.0 * wg[g] * fv * ph[m];
            }
        return c;
    };
    std::vector<std::vector<double>> basis;
    for (int n = 0; n < nq; ++n)
        basis.push_back(coords([&](double t) {
            legendre_ortho(t, q, pt.data());
            return pt[n];
        }));
    std::vector<double> a((size_t)nq * D, 0.0);
    for (int i = 0; i < nq; ++i) {
        std::vector<double> v = coords([&](double t) {
            legendre_ortho(t, q, pt.data());
            return (t < 0.0 ? -1.0 : 1.0) * pt[i];
        });
        for (int pass = 0; pass < 2; ++pass)
            for (const auto& b : basis) {
                double d = 0.0;
                for (int e = 0; e < D; ++e) d += b[e] * v[e];
                for (int e = 0; e < D; ++e) v[e] -= d * b[e];
            }
        double nrm = 0.0;
        for (double x : v) nrm += x * x;
        nrm = sqrt(nrm);
        for (double& x : v) x /= nrm;
        basis.push_back(v);
        for (int e = 0; e < D; ++e) a[(size_t)i * D + e] = v[e] * sqrt(2.0);
    }
    return a;
}

// Function idx of W_{s,q} at t, t known to lie in finest cell f.
static double wavelet_value(int s, int q, const std::vector<double>& mw, int idx, double t, int f) {
    const int nq = q + 1;
    std::vector<double> ph(nq);
    if (idx < nq) {
        legendre_ortho(t, q, ph.data());
        return ph[idx];
    }
    const int blk = idx / nq, i = idx % nq;   // blk = 2^l + c
    int l = 0;
    while ((2 << l) <= blk) ++l;
    const int c = blk - (1 << l);
    if ((f >> (s - l)) != c) return 0.0;
    const double u = ldexp(t + 1.0, l) - 2.0 * c - 1.0;
    const int h = (f >> (s - l - 1)) & 1;
    const double tau = h ? 2.0 * u - 1.0 : 2.0 * u + 1.0;
    legendre_ortho(tau, q, ph.data());
    double v = 0.0;
    for (int m = 0; m < nq; ++m) v += mw[((size_t)i * 2 + h) * nq + m] * ph[m];
    return v * pow(2.0, 0.5 * l);
}

// out[f * (q+1) + n]: function idx of W_{s,q} on finest cell f as sum_n out phi_n(tau),
// tau = 2^s (t + 1) - 2f - 1 (projection by Gauss-Legendre quadrature, exact here).
void wavelet_piecewise(int s, int q, int idx, const std::vector<double>& mw, std::vector<double>& out) {
    const int nq = q + 1, cells = 1 << s, G = q + 2;
    std::vector<double> xg, wg, ph(nq);
    gauss_legendre(G, xg, wg);
    out.assign((size_t)cells * nq, 0.0);
    for (int f = 0; f < cells; ++f)
        for (int g = 0; g < G; ++g) {
            const double t = ldexp(xg[g] + 2.0 * f + 1.0, -s) - 1.0;
            const double v = wavelet_value(s, q, mw, idx, t, f);
            if (v == 0.0) continue;
            legendre_ortho(xg[g], q, ph.data());
            for (int n = 0; n < nq; ++n) out[(size_t)f * nq + n] += 0.5 * wg[g] * v * ph[n];
        }
}

// Every function of W_{s,q} at the points t of [-1, 1]: B[i][idx] (row-major), the cells
// decided by comparing t with the boundaries -1 + (2 c) 2^-s.
void wavelet_design(const std::vector<double>& t, int s, int q, std::vector<double>& B) {
    const int nq = q + 1, P = nq << s, cells = 1 << s;
    const std::vector<double> mw = mother_wavelets(q);
    B.assign(t.size() * P, 0.0);
    for (size_t i = 0; i < t.size(); ++i) {
        int f = 0;
        for (int c = 1; c < cells; ++c) f += t[i] >= -1.0 + ldexp(2.0 * c, -s) ? 1 : 0;
        for (int idx = 0; idx < P; ++idx) B[i * P + idx] = wavelet_value(s, q, mw, idx, t[i], f);
    }
}

// Design of W_{s,q} at the grid nodes g_i = -1 + 2 i / (N - 1): Phi[i][idx] (N x (q+1) 2^s).
void wavelet_grid_design(int N, int s, int q, std::vector<double>& Phi) {
    std::vector<double> t(N);
    for (int i = 0; i < N; ++i) t[i] = -1.0 + 2.0 * i / (N - 1);
    wavelet_design(t, s, q, Phi);
}

// Columns sampled so that dot products are the inner products 1/2 int f g of the functions:
// sqrt(w / 2) f(x) at the Gauss-Legendre nodes (max(p, q) + 1 a cell) of every finest cell.
// cols[j] = (rows, values, in W_{s,q}); Legendre columns use phi_0..phi_p.  Out: column j at
// S[j * L .. j * L + L), L = 2^s (max(p, q) + 1).
void function_samples(int p, int s, int q, const std::vector<const int32_t*>& rows, const std::vector<const double*>& vals,
                      const std::vector<int>& len, const std::vector<uint8_t>& is_wav, std::vector<double>& S, int& L) {
    const int cells = 1 << s, G = (p > q ? p : q) + 1;
    std::vector<double> xg, wg;
    gauss_legendre(G, xg, wg);
    std::vector<double> t, wt;
    for (int c = 0; c < cells; ++c)
        for (int g = 0; g < G; ++g) {
            t.push_back(-1.0 + (2.0 * c + 1.0 + xg[g]) / cells);
            wt.push_back(wg[g] / cells);
        }
    L = (int)t.size();
    std::vector<double> B;
    wavelet_design(t, s, q, B);
    const int P = (q + 1) << s;
    std::vector<double> ph(p + 1);
    S.assign((size_t)L * rows.size(), 0.0);
    for (size_t j = 0; j < rows.size(); ++j)
        for (int i = 0; i < L; ++i) {
            double v = 0.0;
            if (is_wav[j]) {
                for (int e = 0; e < len[j]; ++e) v += vals[j][e] * B[(size_t)i * P + rows[j][e]];
            } else {
                legendre_ortho(t[i], p, ph.data());
                for (int e = 0; e < len[j]; ++e) v += vals[j][e] * ph[rows[j][e]];
            }
            S[j * L + i] = v * sqrt(wt[i] / 2.0);
        }
}

}  // namespace fst
