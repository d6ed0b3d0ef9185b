/*
 * fst_oracle.h -- plain FP64 CPU oracle for the functional sparse Tucker (FST)
 * evaluation and the randomized least-squares refit of its core.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The CUDA library never
 * links, includes or calls this code, and the two share no source.
 *
 * Paper: P. Rai, H. Kolla, L. Cannada, A. Gorodetsky, "Randomized Functional
 * Sparse Tucker Tensor for Compression and Fast Visualization of Scientific
 * Data" (arXiv 1907.05884).
 */
#ifndef FST_ORACLE_H
#define FST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A functional sparse Tucker model with d = 3 (Sec. 2, eq. func_tuck and eq. sparse).
 * Column j of mode k stores the nonzero coefficients W^k_{n,j} of the orthonormal
 * Legendre functions phi_n(t) = sqrt(2n+1) L_n(t), n <= p[k], in CSC form.
 * The core alpha is C-ordered [j1][j2][j3].  Coordinate y_k is mapped to
 * t = 2 (y_k - lo[k]) / (hi[k] - lo[k]) - 1. */
typedef struct {
    int32_t r[3];
    int32_t p[3];
    double lo[3];
    double hi[3];
    const int32_t* colptr[3];   /* r[k] + 1 entries */
    const int32_t* rowidx[3];   /* degree n of each stored coefficient */
    const double* val[3];       /* W^k_{n,j} */
    const double* alpha;        /* r1*r2*r3 */
} fst_oracle_model;

/* Legendre polynomials L_0..L_p at t by the three-term (Bonnet) recurrence. */
void fst_oracle_legendre(double t, int32_t p, double* L);

/* Factor functions w^(k)_j(y_k), j < r[k] (eq. sparse). */
void fst_oracle_factor_values(const fst_oracle_model* M, int32_t k, double yk, double* w);

/* u~(y) at one point by the plain triple sum of eq. func_tuck. */
double fst_oracle_eval_point(const fst_oracle_model* M, double y1, double y2, double y3);

/* u~ at n points given structure-of-arrays y (y[0..n) = y1, y[n..2n) = y2, y[2n..3n) = y3). */
void fst_oracle_eval(const fst_oracle_model* M, const double* y, int64_t n, double* out,
                     int32_t nthreads);

/* Counter-based key of row q: the (q+1)-th output of a splitmix64 stream seeded with `seed`. */
uint64_t fst_oracle_key(uint64_t seed, uint64_t q);

/* Uniform sample of m distinct rows of [0,Q) without replacement: the m rows with the
 * smallest keys, returned in ascending row order (Algorithm 2, sampling step). */
void fst_oracle_sample(uint64_t seed, int64_t Q, int64_t m, int64_t* idx);

/* Row q of the measurement matrix of eq. rand_core: a[(j1 r2 + j2) r3 + j3] = prod_k w_jk(y_k). */
void fst_oracle_design_row(const fst_oracle_model* M, double y1, double y2, double y3, double* a);

/* Rows idx[0..m) of the measurement matrix, m x R row-major; y is SoA with stride Q. */
void fst_oracle_design_matrix(const fst_oracle_model* M, const double* y, int64_t Q,
                              const int64_t* idx, int64_t m, double* A);

/* Normal equations of the sampled problem: G = A^T A (R x R, both triangles),
 * h = A^T b, btb = b^T b with A the sampled design rows and b = u[idx]. */
void fst_oracle_normal_equations(const fst_oracle_model* M, const double* y, const double* u,
                                 int64_t Q, const int64_t* idx, int64_t m,
                                 double* G, double* h, double* btb, int32_t nthreads);

/* In-place Cholesky factorisation G = L L^T (lower triangle written). 0 on success,
 * -(j+1) when the pivot of column j is not positive. */
int32_t fst_oracle_cholesky(double* G, int32_t R, int32_t nthreads);

/* Solve L L^T x = h with the factor from fst_oracle_cholesky. */
void fst_oracle_cholesky_solve(const double* L, int32_t R, const double* h, double* x);

/* Least squares min ||A x - b|| by Householder QR (A m x R row-major, overwritten;
 * b overwritten).  0 on success, -1 if R > m, -(j+2) on a zero column pivot. */
int32_t fst_oracle_lsq_qr(double* A, int64_t m, int32_t R, double* b, double* x);

/* Core refit on the sampled rows (eq. rand_core, Algorithm 2 without the mixing
 * steps): normal equations + Cholesky; Householder QR when Cholesky fails.
 * Returns 0 (Cholesky), 1 (QR fallback) or a negative error. */
int32_t fst_oracle_refit(const fst_oracle_model* M, const double* y, const double* u, int64_t Q,
                         const int64_t* idx, int64_t m, double* alpha_out, int32_t nthreads);

/* g = A^T (b - A alpha) over the sampled rows (the normal-equation residual). */
void fst_oracle_normal_residual(const fst_oracle_model* M, const double* y, const double* u,
                                int64_t Q, const int64_t* idx, int64_t m, const double* alpha,
                                double* g, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
