/*
 * fst_oracle.c -- plain FP64 CPU oracle for functional sparse Tucker evaluation
 * and the randomized least-squares core refit.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the CUDA library, with which it shares
 * no code.
 *
 * Each routine writes the paper's definition out in FP64 with no blocking,
 * fusion or reordering beyond what the definition states:
 *   Sec. 2, eq. func_tuck  u~(y) = sum_{j1,j2,j3} alpha_{j1 j2 j3} w1_{j1}(y1) w2_{j2}(y2) w3_{j3}(y3)
 *   Sec. 2, eq. sparse     w_j(y) = sum_i W_{i,j} phi_i(y) with an orthonormal basis phi
 *   Sec. 5, eq. rand_core  alpha^ = argmin || u - W alpha ||_2^2, W_{q,j} = w_j(y^q)
 *   Algorithm 2            uniform sampling of S > R rows, then the sampled LS solve
 * OpenMP, when enabled, only splits independent outer loops (points, rows of G)
 * across threads; every sum is still taken in its defining order.
 */
#include "fst_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int max_rank(const fst_oracle_model* M) {
    int m = M->r[0];
    if (M->r[1] > m) m = M->r[1];
    if (M->r[2] > m) m = M->r[2];
    return m;
}

static int max_degree(const fst_oracle_model* M) {
    int m = M->p[0];
    if (M->p[1] > m) m = M->p[1];
    if (M->p[2] > m) m = M->p[2];
    return m;
}

/* Bonnet's recurrence: (n+1) L_{n+1}(t) = (2n+1) t L_n(t) - n L_{n-1}(t), L_0 = 1, L_1 = t. */
void fst_oracle_legendre(double t, int32_t p, double* L) {
    L[0] = 1.0;
    if (p >= 1) L[1] = t;
    for (int n = 1; n < p; ++n)
        L[n + 1] = ((2.0 * n + 1.0) * t * L[n] - (double)n * L[n - 1]) / (n + 1.0);
}

/* eq. sparse with phi_n = sqrt(2n+1) L_n, orthonormal for the measure dt/2 on [-1,1] (Sec. 2). */
static void factor_values_scratch(const fst_oracle_model* M, int k, double yk, double* w,
                                  double* L) {
    double t = 2.0 * (yk - M->lo[k]) / (M->hi[k] - M->lo[k]) - 1.0;
    fst_oracle_legendre(t, M->p[k], L);
    for (int j = 0; j < M->r[k]; ++j) {
        double s = 0.0;
        for (int e = M->colptr[k][j]; e < M->colptr[k][j + 1]; ++e) {
            int n = M->rowidx[k][e];
            s += M->val[k][e] * sqrt(2.0 * n + 1.0) * L[n];
        }
        w[j] = s;
    }
}

void fst_oracle_factor_values(const fst_oracle_model* M, int32_t k, double yk, double* w) {
    double* L = (double*)malloc(sizeof(double) * (size_t)(M->p[k] + 1));
    factor_values_scratch(M, k, yk, w, L);
    free(L);
}

/* eq. func_tuck: the triple sum over the core. */
static double eval_point_scratch(const fst_oracle_model* M, double y1, double y2, double y3,
                                 double* w1, double* w2, double* w3, double* L) {
    factor_values_scratch(M, 0, y1, w1, L);
    factor_values_scratch(M, 1, y2, w2, L);
    factor_values_scratch(M, 2, y3, w3, L);
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    double f = 0.0;
    for (int j1 = 0; j1 < r1; ++j1)
        for (int j2 = 0; j2 < r2; ++j2)
            for (int j3 = 0; j3 < r3; ++j3)
                f += M->alpha[((size_t)j1 * r2 + j2) * r3 + j3] * w1[j1] * w2[j2] * w3[j3];
    return f;
}

double fst_oracle_eval_point(const fst_oracle_model* M, double y1, double y2, double y3) {
    int rm = max_rank(M), pm = max_degree(M);
    double* buf = (double*)malloc(sizeof(double) * (size_t)(3 * rm + pm + 1));
    double f = eval_point_scratch(M, y1, y2, y3, buf, buf + rm, buf + 2 * rm, buf + 3 * rm);
    free(buf);
    return f;
}

void fst_oracle_eval(const fst_oracle_model* M, const double* y, int64_t n, double* out,
                     int32_t nthreads) {
    int rm = max_rank(M), pm = max_degree(M);
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        double* buf = (double*)malloc(sizeof(double) * (size_t)(3 * rm + pm + 1));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t q = 0; q < n; ++q)
            out[q] = eval_point_scratch(M, y[q], y[n + q], y[2 * n + q], buf, buf + rm,
                                        buf + 2 * rm, buf + 3 * rm);
        free(buf);
    }
}

/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014): state advances by the golden-ratio
 * increment; each output is the state passed through the variant-13 finaliser. */
uint64_t fst_oracle_key(uint64_t seed, uint64_t q) {
    uint64_t z = seed + (q + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key; int64_t row; } keyed_row;

static int cmp_key(const void* a, const void* b) {
    const keyed_row* x = (const keyed_row*)a;
    const keyed_row* y = (const keyed_row*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->row < y->row ? -1 : (x->row > y->row);
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y);
}

/* Uniform sampling without replacement by random sort keys: attach an independent
 * uniform key to every row and keep the m rows whose keys are smallest. */
void fst_oracle_sample(uint64_t seed, int64_t Q, int64_t m, int64_t* idx) {
    if (m >= Q) {
        for (int64_t q = 0; q < Q; ++q) idx[q] = q;
        return;
    }
    keyed_row* kr = (keyed_row*)malloc(sizeof(keyed_row) * (size_t)Q);
    for (int64_t q = 0; q < Q; ++q) {
        kr[q].key = fst_oracle_key(seed, (uint64_t)q);
        kr[q].row = q;
    }
    qsort(kr, (size_t)Q, sizeof(keyed_row), cmp_key);
    for (int64_t s = 0; s < m; ++s) idx[s] = kr[s].row;
    free(kr);
    qsort(idx, (size_t)m, sizeof(int64_t), cmp_i64);
}

/* Row of the measurement matrix W of eq. rand_core, j = (j1, j2, j3) flattened C-order. */
void fst_oracle_design_row(const fst_oracle_model* M, double y1, double y2, double y3, double* a) {
    int rm = max_rank(M), pm = max_degree(M);
    double* buf = (double*)malloc(sizeof(double) * (size_t)(3 * rm + pm + 1));
    double *w1 = buf, *w2 = buf + rm, *w3 = buf + 2 * rm, *L = buf + 3 * rm;
    factor_values_scratch(M, 0, y1, w1, L);
    factor_values_scratch(M, 1, y2, w2, L);
    factor_values_scratch(M, 2, y3, w3, L);
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    for (int j1 = 0; j1 < r1; ++j1)
        for (int j2 = 0; j2 < r2; ++j2)
            for (int j3 = 0; j3 < r3; ++j3)
                a[((size_t)j1 * r2 + j2) * r3 + j3] = w1[j1] * w2[j2] * w3[j3];
    free(buf);
}

void fst_oracle_design_matrix(const fst_oracle_model* M, const double* y, int64_t Q,
                              const int64_t* idx, int64_t m, double* A) {
    const size_t R = (size_t)M->r[0] * M->r[1] * M->r[2];
    for (int64_t s = 0; s < m; ++s) {
        int64_t q = idx[s];
        fst_oracle_design_row(M, y[q], y[Q + q], y[2 * Q + q], A + (size_t)s * R);
    }
}

void fst_oracle_normal_equations(const fst_oracle_model* M, const double* y, const double* u,
                                 int64_t Q, const int64_t* idx, int64_t m,
                                 double* G, double* h, double* btb, int32_t nthreads) {
    const int64_t R = (int64_t)M->r[0] * M->r[1] * M->r[2];
    double* A = (double*)malloc(sizeof(double) * (size_t)(m * R));
    fst_oracle_design_matrix(M, y, Q, idx, m, A);
    double bb = 0.0;
    for (int64_t s = 0; s < m; ++s) bb += u[idx[s]] * u[idx[s]];
    *btb = bb;
    (void)nthreads;
    /* G_{ab} = sum_s A_{s a} A_{s b}; h_a = sum_s A_{s a} b_s.  Rows a are independent. */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t a = 0; a < R; ++a) {
        double* Ga = G + (size_t)a * R;
        for (int64_t b = 0; b <= a; ++b) Ga[b] = 0.0;
        double ha = 0.0;
        for (int64_t s = 0; s < m; ++s) {
            const double* As = A + (size_t)s * R;
            const double x = As[a];
            for (int64_t b = 0; b <= a; ++b) Ga[b] += x * As[b];
            ha += x * u[idx[s]];
        }
        h[a] = ha;
    }
    for (int64_t a = 0; a < R; ++a)
        for (int64_t b = a + 1; b < R; ++b) G[(size_t)a * R + b] = G[(size_t)b * R + a];
    free(A);
}

/* Cholesky-Crout, column by column: L_jj = sqrt(G_jj - sum_k L_jk^2),
 * L_ij = (G_ij - sum_k L_ik L_jk) / L_jj for i > j. */
int32_t fst_oracle_cholesky(double* G, int32_t R, int32_t nthreads) {
    (void)nthreads;
    for (int32_t j = 0; j < R; ++j) {
        double d = G[(size_t)j * R + j];
        for (int32_t k = 0; k < j; ++k) d -= G[(size_t)j * R + k] * G[(size_t)j * R + k];
        if (!(d > 0.0)) return -(j + 1);
        const double Ljj = sqrt(d);
        G[(size_t)j * R + j] = Ljj;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (int32_t i = j + 1; i < R; ++i) {
            double s = G[(size_t)i * R + j];
            for (int32_t k = 0; k < j; ++k) s -= G[(size_t)i * R + k] * G[(size_t)j * R + k];
            G[(size_t)i * R + j] = s / Ljj;
        }
    }
    for (int32_t i = 0; i < R; ++i)
        for (int32_t j = i + 1; j < R; ++j) G[(size_t)i * R + j] = 0.0;
    return 0;
}

void fst_oracle_cholesky_solve(const double* L, int32_t R, const double* h, double* x) {
    double* z = (double*)malloc(sizeof(double) * (size_t)R);
    for (int32_t i = 0; i < R; ++i) {          /* L z = h */
        double s = h[i];
        for (int32_t k = 0; k < i; ++k) s -= L[(size_t)i * R + k] * z[k];
        z[i] = s / L[(size_t)i * R + i];
    }
    for (int32_t i = R - 1; i >= 0; --i) {     /* L^T x = z */
        double s = z[i];
        for (int32_t k = i + 1; k < R; ++k) s -= L[(size_t)k * R + i] * x[k];
        x[i] = s / L[(size_t)i * R + i];
    }
    free(z);
}

/* Householder QR: for each column j reflect rows j..m-1 so that column j below the
 * diagonal vanishes; apply the same reflections to b; then back-substitute R x = Q^T b. */
int32_t fst_oracle_lsq_qr(double* A, int64_t m, int32_t R, double* b, double* x) {
    if ((int64_t)R > m) return -1;
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    for (int32_t j = 0; j < R; ++j) {
        double nrm = 0.0;
        for (int64_t i = j; i < m; ++i) nrm += A[(size_t)i * R + j] * A[(size_t)i * R + j];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { free(v); return -(j + 2); }
        const double ajj = A[(size_t)j * R + j];
        const double alpha = ajj > 0.0 ? -nrm : nrm;      /* avoid cancellation */
        double vnorm2 = 0.0;
        for (int64_t i = j; i < m; ++i) v[i] = A[(size_t)i * R + j];
        v[j] -= alpha;
        for (int64_t i = j; i < m; ++i) vnorm2 += v[i] * v[i];
        /* H = I - 2 v v^T / (v^T v) applied to columns j..R-1 and to b */
        for (int32_t c = j; c < R; ++c) {
            double dot = 0.0;
            for (int64_t i = j; i < m; ++i) dot += v[i] * A[(size_t)i * R + c];
            const double f = 2.0 * dot / vnorm2;
            for (int64_t i = j; i < m; ++i) A[(size_t)i * R + c] -= f * v[i];
        }
        double dotb = 0.0;
        for (int64_t i = j; i < m; ++i) dotb += v[i] * b[i];
        const double fb = 2.0 * dotb / vnorm2;
        for (int64_t i = j; i < m; ++i) b[i] -= fb * v[i];
    }
    for (int32_t i = R - 1; i >= 0; --i) {
        double s = b[i];
        for (int32_t k = i + 1; k < R; ++k) s -= A[(size_t)i * R + k] * x[k];
        x[i] = s / A[(size_t)i * R + i];
    }
    free(v);
    return 0;
}

int32_t fst_oracle_refit(const fst_oracle_model* M, const double* y, const double* u, int64_t Q,
                         const int64_t* idx, int64_t m, double* alpha_out, int32_t nthreads) {
    const int64_t R = (int64_t)M->r[0] * M->r[1] * M->r[2];
    double* G = (double*)malloc(sizeof(double) * (size_t)(R * R));
    double* h = (double*)malloc(sizeof(double) * (size_t)R);
    double btb;
    fst_oracle_normal_equations(M, y, u, Q, idx, m, G, h, &btb, nthreads);
    int32_t rc = fst_oracle_cholesky(G, (int32_t)R, nthreads);
    if (rc == 0) {
        fst_oracle_cholesky_solve(G, (int32_t)R, h, alpha_out);
    } else {
        double* A = (double*)malloc(sizeof(double) * (size_t)(m * R));
        double* b = (double*)malloc(sizeof(double) * (size_t)m);
        fst_oracle_design_matrix(M, y, Q, idx, m, A);
        for (int64_t s = 0; s < m; ++s) b[s] = u[idx[s]];
        rc = fst_oracle_lsq_qr(A, m, (int32_t)R, b, alpha_out);
        rc = rc == 0 ? 1 : rc;
        free(A);
        free(b);
    }
    free(G);
    free(h);
    return rc;
}

void fst_oracle_normal_residual(const fst_oracle_model* M, const double* y, const double* u,
                                int64_t Q, const int64_t* idx, int64_t m, const double* alpha,
                                double* g, int32_t nthreads) {
    const int64_t R = (int64_t)M->r[0] * M->r[1] * M->r[2];
    memset(g, 0, sizeof(double) * (size_t)R);
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        double* a = (double*)malloc(sizeof(double) * (size_t)R);
        double* gl = (double*)calloc((size_t)R, sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < m; ++s) {
            const int64_t q = idx[s];
            fst_oracle_design_row(M, y[q], y[Q + q], y[2 * Q + q], a);
            double pred = 0.0;
            for (int64_t j = 0; j < R; ++j) pred += a[j] * alpha[j];
            const double res = u[q] - pred;
            for (int64_t j = 0; j < R; ++j) gl[j] += res * a[j];
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int64_t j = 0; j < R; ++j) g[j] += gl[j];
        free(a);
        free(gl);
    }
}
