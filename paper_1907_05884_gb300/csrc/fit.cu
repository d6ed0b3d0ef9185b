// fit.cu -- construction of a functional sparse Tucker model on the GPU (Algorithm 1)
// followed by the randomized least-squares refit of its core (Algorithm 2):
//   1. a uniform sample of a fraction of the points (the row sampler of sample.cu) is
//      splatted trilinearly onto an equispaced node grid (both ends of [-1,1] are nodes): each
//      sample adds its value to the 8 nodes of its cell with trilinear weights and a node takes
//      the weighted mean; nodes without weight are filled by Jacobi sweeps that give an empty
//      node the mean of its filled 6-neighbours of the previous sweep (Sec. 4.1);
//   2. ST-HOSVD (Sec. 4.1, Algorithm 1): modes 1, 2, 3 in order; the mode Gram matrix in FP64,
//      its eigenpairs by parallel cyclic Jacobi in one block; the kept rank is the smallest
//      r >= 1 whose discarded eigenvalues sum to at most eps^2 ||U||^2 / 3, capped (or the cap
//      itself in fixed-rank mode); each kept eigenvector's largest-magnitude entry is made
//      positive, and the tensor is multiplied by the transposed factor before the next mode;
//   3. per factor column (Sec. 3, Sec. 4.2): the Lasso-modified LARS path on the
//      orthonormal-Legendre design of the grid nodes (columns scaled to unit norm for the
//      correlations); every support the path visits is refitted by least squares and scored by
//      its exact leave-one-out error; the least error wins (ties within 1e-12 mean(y^2) go to
//      the smaller, then the earlier support) and its least-squares coefficients are stored;
//   4. a fitted factor function in the span of the earlier ones of its mode (relative
//      residual norm <= 1e-6 after in-order Gram-Schmidt on its orthonormal-Legendre
//      coefficients) is dropped, so the refit's least squares has independent columns;
//   5. the core refit of refit.cu on m = min(ceil(oversample R), Q) sampled rows (Sec. 5).
// Steps 1-3 run in FP64; the refit runs in the requested precision.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fst_internal.cuh"

namespace fst {

namespace {

constexpr int kMaxGrid = 256;
constexpr int kLarsMaxP = 64;
constexpr int kLarsMaxN = kMaxGrid;
constexpr int kLarsThreads = 256;
constexpr int kLarsMaxSeen = 8 * kLarsMaxP + 16;
constexpr int kEigThreads = 1024;
constexpr int kEigMaxSweeps = 30;
constexpr uint64_t kRefitSeedOffset = 0x632BE59BD9B4E019ull;

// ------------------------------------------------------------------ step 1: interpolation
__global__ void splat_kernel(const float* __restrict__ xyz, const float* __restrict__ u, int64_t Q,
                             const int64_t* __restrict__ idx, int64_t ns, double lo0, double lo1, double lo2,
                             double hi0, double hi1, double hi2, int I0, int I1, int I2, double* num, double* den) {
    const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    const int I[3] = {I0, I1, I2};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = idx[s];
        int c[3];
        double f[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double t = 2.0 * ((double)xyz[k * Q + q] - lo[k]) / (hi[k] - lo[k]) - 1.0;
            const double sc = (t + 1.0) / (2.0 / (I[k] - 1));
            double fl = floor(sc);
            fl = fl < 0.0 ? 0.0 : (fl > I[k] - 2 ? (double)(I[k] - 2) : fl);
            c[k] = (int)fl;
            f[k] = sc - fl;
        }
        const double val = (double)u[q];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    const double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (e ? f[2] : 1.0 - f[2]);
                    const size_t node = ((size_t)(c[0] + a) * I1 + (c[1] + b)) * I2 + (c[2] + e);
                    atomicAdd(&num[node], w * val);
                    atomicAdd(&den[node], w);
                }
    }
}

__device__ __forceinline__ void warp_count(unsigned long long v, unsigned long long* total) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// num <- num / den where den > 0 (filled), else 0; counts the empty nodes.
__global__ void node_values_kernel(double* num, const double* den, int64_t n, uint8_t* filled,
                                   unsigned long long* empty) {
    unsigned long long e = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const bool f = den[i] > 0.0;
        num[i] = f ? num[i] / den[i] : 0.0;
        filled[i] = f;
        e += !f;
    }
    warp_count(e, empty);
}

// One Jacobi fill sweep: reads (U, filled), writes (U2, filled2); counts nodes left empty.
__global__ void fill_sweep_kernel(const double* U, const uint8_t* filled, double* U2, uint8_t* filled2, int I0,
                                  int I1, int I2, unsigned long long* empty_left) {
    const int64_t n = (int64_t)I0 * I1 * I2;
    const int64_t plane = (int64_t)I1 * I2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long left = 0;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += stride) {
        if (filled[id]) {
            U2[id] = U[id];
            filled2[id] = 1;
            continue;
        }
        const int i = (int)(id / plane), j = (int)((id / I2) % I1), l = (int)(id % I2);
        const int64_t nb[6] = {i > 0 ? id - plane : -1, i + 1 < I0 ? id + plane : -1,
                               j > 0 ? id - I2 : -1,    j + 1 < I1 ? id + I2 : -1,
                               l > 0 ? id - 1 : -1,     l + 1 < I2 ? id + 1 : -1};
        double s = 0.0;
        int cnt = 0;
        for (int e = 0; e < 6; ++e)
            if (nb[e] >= 0 && filled[nb[e]]) {
                s += U[nb[e]];
                ++cnt;
            }
        U2[id] = cnt ? s / cnt : 0.0;
        filled2[id] = cnt > 0;
        left += cnt == 0;
    }
    warp_count(left, empty_left);
}

// ------------------------------------------------------------------ step 2: ST-HOSVD
__device__ double block_sum(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// deterministic sum of squares (one block of 1024 threads)
__global__ void sumsq_kernel(const double* X, int64_t n, double* out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += X[i] * X[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

// offset of entry (a, r) of the mode-k unfolding of a C-ordered n0 x n1 x n2 tensor
__device__ __forceinline__ int64_t unfold_off(int k, int a, int64_t r, int n1, int n2) {
    if (k == 0) return (int64_t)a * n1 * n2 + r;
    if (k == 1) return ((r / n2) * n1 + a) * n2 + r % n2;
    return r * n2 + a;
}

// S = X_(k) X_(k)^T (n_k x n_k), 16 x 16 output tiles, 16 x 16 threads
__global__ void mode_gram_kernel(const double* X, int k, int n0, int n1, int n2, double* S) {
    const int nk = k == 0 ? n0 : k == 1 ? n1 : n2;
    const int64_t rest = (int64_t)n0 * n1 * n2 / nk;
    __shared__ double xa[16][33], xb[16][33];
    double acc = 0.0;
    for (int64_t r0 = 0; r0 < rest; r0 += 32) {
        for (int e = threadIdx.y * 16 + threadIdx.x; e < 16 * 32; e += 256) {
            const int rr = e % 32, row = e / 32;
            const int64_t r = r0 + rr;
            const int ga = blockIdx.y * 16 + row, gb = blockIdx.x * 16 + row;
            xa[row][rr] = (ga < nk && r < rest) ? X[unfold_off(k, ga, r, n1, n2)] : 0.0;
            xb[row][rr] = (gb < nk && r < rest) ? X[unfold_off(k, gb, r, n1, n2)] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) acc += xa[threadIdx.y][rr] * xb[threadIdx.x][rr];
        __syncthreads();
    }
    const int a = blockIdx.y * 16 + threadIdx.y, b = blockIdx.x * 16 + threadIdx.x;
    if (a < nk && b < nk) S[(size_t)a * nk + b] = acc;
}

// Parallel cyclic Jacobi for the symmetric n x n matrix S (overwritten; its diagonal ends as
// the eigenvalues) with the eigenvectors accumulated in the columns of V.  Each round
// applies n/2 disjoint rotations (round-robin pairing, player 0 fixed, a dummy player when n
// is odd); a sweep is m-1 rounds for m = n rounded up to even.  Stops when the off-diagonal
// Frobenius norm is at most 1e-14 of the whole, or after max_sweeps sweeps.  Each rotation
// is the symmetric 2 x 2 Schur rotation that zeroes S_pq.
__global__ void __launch_bounds__(kEigThreads) jacobi_eig_kernel(double* S, double* V, int n, int max_sweeps,
                                                                  int* sweeps_out) {
    extern __shared__ double jsm[];
    const int m = n + (n & 1);
    double* cs = jsm;
    double* sn = jsm + m / 2;
    int* pp = reinterpret_cast<int*>(sn + m / 2);
    int* qq = pp + m / 2;
    __shared__ double red[kEigThreads];
    const int tid = threadIdx.x, B = blockDim.x;
    for (int e = tid; e < n * n; e += B) V[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += B) {
            const double v = S[e] * S[e];
            tot += v;
            if (e / n != e % n) off += v;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (!(off > 1e-28 * tot)) break;
        for (int round = 0; round + 1 < m; ++round) {
            for (int h = tid; h < m / 2; h += B) {
                const int pos_b = m - 1 - h;   // >= 1
                int p = h == 0 ? 0 : 1 + (h - 1 + round) % (m - 1);
                int q = 1 + (pos_b - 1 + round) % (m - 1);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                pp[h] = p;
                qq[h] = q;
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = S[(size_t)p * n + q];
                    if (apq != 0.0) {
                        const double theta = (S[(size_t)q * n + q] - S[(size_t)p * n + p]) / (2.0 * apq);
                        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                cs[h] = c;
                sn[h] = s;
            }
            __syncthreads();
            for (int e = tid; e < (m / 2) * n; e += B) {      // rows p, q:  S <- J^T S
                const int h = e / n, col = e % n, p = pp[h], q = qq[h];
                if (q >= n) continue;
                const double c = cs[h], s = sn[h];
                const double sp = S[(size_t)p * n + col], sq = S[(size_t)q * n + col];
                S[(size_t)p * n + col] = c * sp - s * sq;
                S[(size_t)q * n + col] = s * sp + c * sq;
            }
            __syncthreads();
            for (int e = tid; e < (m / 2) * n; e += B) {      // columns p, q:  S <- S J,  V <- V J
                const int h = e / n, row = e % n, p = pp[h], q = qq[h];
                if (q >= n) continue;
                const double c = cs[h], s = sn[h];
                const double sp = S[(size_t)row * n + p], sq = S[(size_t)row * n + q];
                S[(size_t)row * n + p] = c * sp - s * sq;
                S[(size_t)row * n + q] = s * sp + c * sq;
                const double vp = V[(size_t)row * n + p], vq = V[(size_t)row * n + q];
                V[(size_t)row * n + p] = c * vp - s * vq;
                V[(size_t)row * n + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    if (tid == 0) *sweeps_out = sw;
}

__global__ void diag_kernel(const double* S, int n, double* d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = S[(size_t)i * n + i];
}

// W[:, j] = V[:, order[j]] with its largest-magnitude entry (lowest index on ties) positive.
__global__ void select_vectors_kernel(const double* V, int n, const int* order, int r, double* W) {
    const int j = blockIdx.x;
    __shared__ int best_i;
    if (threadIdx.x == 0) {
        double best_v = -1.0;
        best_i = 0;
        for (int i = 0; i < n; ++i) {
            const double a = fabs(V[(size_t)i * n + order[j]]);
            if (a > best_v) {
                best_v = a;
                best_i = i;
            }
        }
    }
    __syncthreads();
    const double sgn = V[(size_t)best_i * n + order[j]] < 0 ? -1.0 : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) W[(size_t)i * r + j] = sgn * V[(size_t)i * n + order[j]];
}

// Y = X x_k W^T: mode k goes from n_k to r entries (W is n_k x r, row-major).
__global__ void ttm_kernel(const double* X, int k, int n0, int n1, int n2, const double* W, int r, double* Y) {
    const int nk = k == 0 ? n0 : k == 1 ? n1 : n2;
    const int m0 = k == 0 ? r : n0, m1 = k == 1 ? r : n1, m2 = k == 2 ? r : n2;
    const int64_t total = (int64_t)m0 * m1 * m2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ((int64_t)m1 * m2)), j = (int)((e / m2) % m1), l = (int)(e % m2);
        const int jj = k == 0 ? i : k == 1 ? j : l;
        double s = 0.0;
        for (int a = 0; a < nk; ++a) {
            const int64_t src = k == 0 ? ((int64_t)a * n1 + j) * n2 + l
                              : k == 1 ? ((int64_t)i * n1 + a) * n2 + l
                                       : ((int64_t)i * n1 + j) * n2 + a;
            s += W[(size_t)a * r + jj] * X[src];
        }
        Y[e] = s;
    }
}

// ------------------------------------------------------------------ step 3: sparse columns
// Phi[i][n] = sqrt(2n+1) L_n(g_i), g_i = -1 + 2 i / (N - 1), n = 0..P-1 (Bonnet recurrence)
__global__ void legendre_design_kernel(int N, int P, double* Phi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double t = -1.0 + 2.0 * i / (N - 1);
        double Lm = 1.0, L = t;
        Phi[(size_t)i * P] = 1.0;
        if (P > 1) Phi[(size_t)i * P + 1] = L * sqrt(3.0);
        for (int n = 1; n + 1 < P; ++n) {
            const double Ln = ((2.0 * n + 1.0) * t * L - n * Lm) / (n + 1.0);
            Lm = L;
            L = Ln;
            Phi[(size_t)i * P + n + 1] = Ln * sqrt(2.0 * n + 3.0);
        }
    }
}

struct LarsJob {
    const double* Phi;   // N x P row-major design of the mode
    const double* W;     // N x ldw factor matrix; the job fits column col
    int ldw, col, N, P;
};

// In-place Cholesky of the s x s row-major matrix A (leading dimension ld) by the whole
// block; returns false (on every thread) if a pivot is not positive.
__device__ bool block_cholesky(double* A, int s, int ld) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < s; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * ld + j];
            if (!(d > 0.0)) bad = 1;
            A[j * ld + j] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncthreads();
        const double piv = A[j * ld + j];
        for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) A[i * ld + j] /= piv;
        __syncthreads();
        const int t = s - j - 1;
        for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
            const int i = j + 1 + e / t, c = j + 1 + e % t;
            if (c <= i) A[i * ld + c] -= A[i * ld + j] * A[c * ld + j];
        }
        __syncthreads();
    }
    const bool ok = bad == 0;
    __syncthreads();
    return ok;
}

// x <- (L L^T)^-1 x, L lower triangular row-major; one thread
__device__ void chol_solve_1t(const double* L, int s, int ld, double* x) {
    for (int i = 0; i < s; ++i) {
        double v = x[i];
        for (int k = 0; k < i; ++k) v -= L[i * ld + k] * x[k];
        x[i] = v / L[i * ld + i];
    }
    for (int i = s - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < s; ++k) v -= L[k * ld + i] * x[k];
        x[i] = v / L[i * ld + i];
    }
}

// One block per factor column: Lasso-LARS path with leave-one-out selection (file comment).
// Dynamic shared memory: two kLarsMaxP x kLarsMaxP FP64 matrices.
__global__ void __launch_bounds__(kLarsThreads) lars_loo_kernel(const LarsJob* jobs, int32_t* rows_out,
                                                                 double* coef_out, int32_t* nnz_out, double* loo_out) {
    extern __shared__ double lsm[];
    double* G = lsm;                                  // Phi^T Phi
    double* GA = lsm + kLarsMaxP * kLarsMaxP;        // factor workspace
    __shared__ double y[kLarsMaxN], mu[kLarsMaxN], uA[kLarsMaxN];
    __shared__ double nrm[kLarsMaxP], c[kLarsMaxP], beta[kLarsMaxP], a[kLarsMaxP], bvec[kLarsMaxP];
    __shared__ double g1[kLarsMaxP], w[kLarsMaxP], sgn[kLarsMaxP], coef[kLarsMaxP], best_coef[kLarsMaxP];
    __shared__ int act[kLarsMaxP], sup[kLarsMaxP], best_rows[kLarsMaxP];
    __shared__ unsigned long long seen[kLarsMaxSeen];
    __shared__ double red[kLarsThreads];
    __shared__ double sh_C, sh_AA, sh_gamma, best_err;
    __shared__ int nact, nxt, done, best_len, nseen, skip;

    const LarsJob J = jobs[blockIdx.x];
    const int N = J.N, P = J.P, tid = threadIdx.x;
    const double* Phi = J.Phi;
    for (int i = tid; i < N; i += blockDim.x) {
        y[i] = J.W[(size_t)i * J.ldw + J.col];
        mu[i] = 0.0;
    }
    __syncthreads();
    for (int e = tid; e < P * P; e += blockDim.x) {
        const int n1 = e / P, n2 = e % P;
        double g = 0.0;
        for (int r = 0; r < N; ++r) g += Phi[(size_t)r * P + n1] * Phi[(size_t)r * P + n2];
        G[n1 * kLarsMaxP + n2] = g;
    }
    for (int n = tid; n < P; n += blockDim.x) {
        double sy = 0.0;
        for (int r = 0; r < N; ++r) sy += Phi[(size_t)r * P + n] * y[r];
        bvec[n] = sy;
        beta[n] = 0.0;
    }
    __syncthreads();
    for (int n = tid; n < P; n += blockDim.x) {
        nrm[n] = sqrt(G[n * kLarsMaxP + n]);
        c[n] = nrm[n] > 0.0 ? bvec[n] / nrm[n] : 0.0;
    }
    double yy = 0.0;
    for (int i = tid; i < N; i += blockDim.x) yy += y[i] * y[i];
    yy = block_sum(yy, red);
    const double ynorm = sqrt(yy), scale = yy / N;
    if (tid == 0) {
        nact = 0;
        nseen = 0;
        best_len = 0;
        best_err = INFINITY;
        done = ynorm == 0.0;
        int arg = 0;
        double mx = -1.0;
        for (int n = 0; n < P; ++n)
            if (fabs(c[n]) > mx) {
                mx = fabs(c[n]);
                arg = n;
            }
        nxt = arg;
    }
    __syncthreads();

    // least squares on the current active set, scored by its leave-one-out error
    auto score = [&]() {
        const int s = nact;
        if (s >= N) return;
        if (tid == 0) {
            unsigned long long mask = 0;
            for (int i = 0; i < s; ++i) {
                sup[i] = act[i];
                mask |= 1ull << act[i];
            }
            for (int i = 1; i < s; ++i)
                for (int k = i; k > 0 && sup[k - 1] > sup[k]; --k) {
                    const int t = sup[k];
                    sup[k] = sup[k - 1];
                    sup[k - 1] = t;
                }
            skip = 0;
            for (int i = 0; i < nseen; ++i) skip |= seen[i] == mask;
            if (!skip && nseen < kLarsMaxSeen) seen[nseen++] = mask;
        }
        __syncthreads();
        if (skip) return;
        for (int e = tid; e < s * s; e += blockDim.x) {
            const int i = e / s, k = e % s;
            GA[i * kLarsMaxP + k] = G[sup[i] * kLarsMaxP + sup[k]];
        }
        __syncthreads();
        const bool ok = block_cholesky(GA, s, kLarsMaxP);
        if (tid == 0) {
            for (int i = 0; i < s; ++i) coef[i] = bvec[sup[i]];
            if (ok) chol_solve_1t(GA, s, kLarsMaxP, coef);
        }
        __syncthreads();
        double acc = 0.0, lev_bad = 0.0;
        for (int r = tid; r < N; r += blockDim.x) {
            double z[kLarsMaxP];
            double pred = 0.0, h = 0.0;
            for (int i = 0; i < s; ++i) {
                double v = Phi[(size_t)r * P + sup[i]];
                pred += v * coef[i];
                for (int k = 0; k < i; ++k) v -= GA[i * kLarsMaxP + k] * z[k];
                z[i] = v / GA[i * kLarsMaxP + i];
                h += z[i] * z[i];
            }
            if (h >= 1.0 - 1e-10) lev_bad = 1.0;
            const double e = (y[r] - pred) / (1.0 - h);
            acc += e * e;
        }
        acc = block_sum(acc, red);
        lev_bad = block_sum(lev_bad, red);
        if (tid == 0) {
            const double err = (ok && lev_bad == 0.0) ? acc / N : INFINITY;
            bool take = best_len == 0;
            if (!take && err < best_err - 1e-12 * scale) take = true;
            if (!take && fabs(err - best_err) <= 1e-12 * scale && s < best_len) take = true;
            if (take) {
                best_err = err;
                best_len = s;
                for (int i = 0; i < s; ++i) {
                    best_rows[i] = sup[i];
                    best_coef[i] = coef[i];
                }
            }
        }
        __syncthreads();
    };

    const int max_steps = 8 * P + 8;
    for (int step = 0; step < max_steps && !done; ++step) {
        if (nxt >= 0) {
            if (tid == 0) act[nact++] = nxt;
            __syncthreads();
            score();
        }
        // correlations of the unit-norm columns with the residual
        for (int n = tid; n < P; n += blockDim.x) {
            double cn = 0.0;
            if (nrm[n] > 0.0) {
                for (int r = 0; r < N; ++r) cn += Phi[(size_t)r * P + n] * (y[r] - mu[r]);
                cn /= nrm[n];
            }
            c[n] = cn;
        }
        __syncthreads();
        const int s = nact;
        if (tid == 0) {
            double C = 0.0;
            for (int i = 0; i < s; ++i) {
                C = fmax(C, fabs(c[act[i]]));
                sgn[i] = c[act[i]] >= 0.0 ? 1.0 : -1.0;
            }
            sh_C = C;
            if (C <= 1e-14 * ynorm) done = 1;
        }
        __syncthreads();
        if (done) break;
        for (int e = tid; e < s * s; e += blockDim.x) {
            const int i = e / s, k = e % s;
            GA[i * kLarsMaxP + k] =
                G[act[i] * kLarsMaxP + act[k]] * sgn[i] * sgn[k] / (nrm[act[i]] * nrm[act[k]]);
        }
        __syncthreads();
        const bool ok = block_cholesky(GA, s, kLarsMaxP);
        if (tid == 0) {
            if (!ok) {
                done = 1;
            } else {
                for (int i = 0; i < s; ++i) g1[i] = 1.0;
                chol_solve_1t(GA, s, kLarsMaxP, g1);
                double den = 0.0;
                for (int i = 0; i < s; ++i) den += g1[i];
                if (!(den > 0.0)) {
                    done = 1;
                } else {
                    sh_AA = 1.0 / sqrt(den);
                    for (int i = 0; i < s; ++i) w[i] = sh_AA * g1[i];
                }
            }
        }
        __syncthreads();
        if (done) break;
        // equiangular direction u_A and the correlations a = X^T u_A
        for (int r = tid; r < N; r += blockDim.x) {
            double v = 0.0;
            for (int i = 0; i < s; ++i) v += w[i] * sgn[i] * Phi[(size_t)r * P + act[i]] / nrm[act[i]];
            uA[r] = v;
        }
        __syncthreads();
        for (int n = tid; n < P; n += blockDim.x) {
            double an = 0.0;
            if (nrm[n] > 0.0) {
                for (int r = 0; r < N; ++r) an += Phi[(size_t)r * P + n] * uA[r];
                an /= nrm[n];
            }
            a[n] = an;
        }
        __syncthreads();
        if (tid == 0) {
            const double C = sh_C, AA = sh_AA;
            double gamma_enter = C / AA;
            int j_enter = -1;
            int usable = 0;
            for (int n = 0; n < P; ++n) usable += nrm[n] > 0.0;
            if (s < min(N, usable)) {
                for (int n = 0; n < P; ++n) {
                    if (!(nrm[n] > 0.0)) continue;
                    bool in = false;
                    for (int i = 0; i < s; ++i) in |= act[i] == n;
                    if (in) continue;
                    const double c1 = AA != a[n] ? (C - c[n]) / (AA - a[n]) : INFINITY;
                    const double c2 = AA != -a[n] ? (C + c[n]) / (AA + a[n]) : INFINITY;
                    if (c1 > 1e-15 && c1 < gamma_enter) {
                        gamma_enter = c1;
                        j_enter = n;
                    }
                    if (c2 > 1e-15 && c2 < gamma_enter) {
                        gamma_enter = c2;
                        j_enter = n;
                    }
                }
            }
            double gamma_drop = INFINITY;
            int i_drop = -1;
            for (int i = 0; i < s; ++i) {
                const double d = sgn[i] * w[i];
                if (d != 0.0) {
                    const double g = -beta[act[i]] / d;
                    if (g > 1e-15 && g < gamma_drop) {
                        gamma_drop = g;
                        i_drop = i;
                    }
                }
            }
            double gamma = gamma_enter;
            if (gamma_drop < gamma_enter) gamma = gamma_drop;
            else i_drop = -1;
            sh_gamma = gamma;
            for (int i = 0; i < s; ++i) beta[act[i]] += gamma * sgn[i] * w[i];
            if (i_drop >= 0) {
                beta[act[i_drop]] = 0.0;
                for (int i = i_drop; i + 1 < s; ++i) act[i] = act[i + 1];
                --nact;
                nxt = -2;                 // the reduced set is scored next; nothing enters
            } else {
                nxt = j_enter;
                if (j_enter < 0) done = 1;  // the least-squares fit of the active set is reached
            }
        }
        __syncthreads();
        for (int r = tid; r < N; r += blockDim.x) mu[r] += sh_gamma * uA[r];
        __syncthreads();
        if (nxt == -2) {
            score();
            if (tid == 0) nxt = -1;
            __syncthreads();
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int j = blockIdx.x;
        if (best_len == 0) {            // zero column: a single zero coefficient
            rows_out[j * kLarsMaxP] = 0;
            coef_out[j * kLarsMaxP] = 0.0;
            nnz_out[j] = 1;
            loo_out[j] = 0.0;
        } else {
            for (int i = 0; i < best_len; ++i) {
                rows_out[j * kLarsMaxP + i] = best_rows[i];
                coef_out[j * kLarsMaxP + i] = best_coef[i];
            }
            nnz_out[j] = best_len;
            loo_out[j] = best_err;
        }
    }
}

__global__ void widen_kernel(const float* src, double* dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// ------------------------------------------------------------------ host side
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T> fst_status get(T** out, size_t count) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("fst_fit: cannot allocate %zu bytes of device memory", count * sizeof(T));
            return FST_ENOMEM;
        }
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return FST_OK;
    }
};

int grid_blocks(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 8));
}

struct Timer {
    cudaEvent_t e[5] = {};
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        for (auto& x : e) cudaEventCreate(&x);
    }
    ~Timer() {
        for (auto& x : e) cudaEventDestroy(x);
    }
    void mark(int i) { cudaEventRecord(e[i], s); }
    double ms(int a, int b) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[a], e[b]);
        return t;
    }
};

// Columns of the (P x r) column-major coefficient matrix C kept, in order, by modified
// Gram-Schmidt with two passes: a column goes when its squared residual against the kept
// ones is <= 1e-12 of its squared norm, or it is zero.
std::vector<int> independent_columns(const std::vector<double>& C, int P, int r) {
    std::vector<int> kept;
    std::vector<std::vector<double>> qs;
    for (int j = 0; j < r; ++j) {
        std::vector<double> v(C.begin() + (size_t)j * P, C.begin() + (size_t)(j + 1) * P);
        double n2 = 0.0;
        for (double x : v) n2 += x * x;
        for (int pass = 0; pass < 2; ++pass)
            for (const auto& q : qs) {
                double d = 0.0;
                for (int i = 0; i < P; ++i) d += q[i] * v[i];
                for (int i = 0; i < P; ++i) v[i] -= d * q[i];
            }
        double r2 = 0.0;
        for (double x : v) r2 += x * x;
        if (n2 == 0.0 || r2 <= 1e-12 * n2) continue;
        kept.push_back(j);
        const double inv = 1.0 / sqrt(r2);
        for (double& x : v) x *= inv;
        qs.push_back(std::move(v));
    }
    return kept;
}

fst_status validate_params(const fst_fit_params* P, int64_t Q, fst_prec prec) {
    FST_REQUIRE(P != nullptr, "params is NULL");
    FST_REQUIRE(Q > 0, "Q must be positive");
    FST_REQUIRE(prec == FST_FP64 || prec == FST_FP32 || prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "unknown precision %d", (int)prec);
    for (int k = 0; k < 3; ++k) {
        FST_REQUIRE(P->grid[k] >= 2 && P->grid[k] <= kMaxGrid, "grid[%d] = %d outside 2..%d", k, P->grid[k],
                    kMaxGrid);
        FST_REQUIRE(P->max_rank[k] >= 1 && P->max_rank[k] <= FST_MAX_RANK, "max_rank[%d] = %d outside 1..%d", k,
                    P->max_rank[k], FST_MAX_RANK);
    }
    FST_REQUIRE(P->max_degree >= 0 && P->max_degree < kLarsMaxP, "max_degree = %d outside 0..%d", P->max_degree,
                kLarsMaxP - 1);
    FST_REQUIRE(P->grid_values != nullptr || (P->sample_frac > 0.0 && P->sample_frac <= 1.0),
                "sample_frac must be in (0, 1]");
    FST_REQUIRE(P->eps >= 0.0 && isfinite(P->eps), "eps must be finite and >= 0");
    FST_REQUIRE(P->oversample > 0.0 && isfinite(P->oversample), "oversample must be positive");
    if (P->wavelet) {
        FST_REQUIRE(P->wav_level >= 0 && P->wav_level <= FST_MAX_WAVELET_LEVEL && P->wav_degree >= 0 &&
                        P->wav_degree <= FST_MAX_WAVELET_DEGREE && ((P->wav_degree + 1) << P->wav_level) <= kLarsMaxP,
                    "wavelet space W_{%d,%d} outside the fit's limits ((q+1) 2^s <= %d)", P->wav_level,
                    P->wav_degree, kLarsMaxP);
    }
    return FST_OK;
}

}  // namespace

}  // namespace fst

using namespace fst;

extern "C" fst_status fst_fit(const float* xyz, const float* u, int64_t Q, const double lo_in[3],
                              const double hi_in[3], const fst_fit_params* params, fst_prec prec,
                              const fst_refit_opts* opts, fst_fit_trace* trace, fst_fit_report* report,
                              fst_model** out, fst_stream stream) {
    FST_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    FST_REQUIRE(xyz != nullptr && u != nullptr, "xyz or u is NULL");
    FST_TRY(validate_params(params, Q, prec));
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(pointer_device(xyz) == dev && pointer_device(u) == dev, "xyz and u must be device memory");
    const fst_fit_params& P = *params;
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = lo_in ? lo_in[k] : -1.0;
        hi[k] = hi_in ? hi_in[k] : 1.0;
        FST_REQUIRE(hi[k] > lo[k] && isfinite(lo[k]) && isfinite(hi[k]), "box: need lo < hi on axis %d", k);
    }
    cudaStream_t s = (cudaStream_t)stream;
    fst_fit_report rep{};
    Scratch sc;
    Timer tm(s);
    const int I[3] = {P.grid[0], P.grid[1], P.grid[2]};
    const int64_t NG = (int64_t)I[0] * I[1] * I[2];

    // ---------------------------------------------------------------- step 1
    tm.mark(0);
    double *bufA = nullptr, *bufB = nullptr;
    FST_TRY(sc.get(&bufA, NG));
    FST_TRY(sc.get(&bufB, NG));
    double* U = bufA;           // the grid tensor at the end of step 1
    double* other = bufB;
    if (P.grid_values) {
        FST_CUDA(cudaMemcpyAsync(bufA, P.grid_values, NG * sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
        const int64_t ns = std::min<int64_t>((int64_t)ceil(P.sample_frac * (double)Q), Q);
        rep.n_interp = ns;
        int64_t* idx = nullptr;
        uint8_t *fa = nullptr, *fb = nullptr;
        const int max_sweeps = I[0] + I[1] + I[2];
        unsigned long long* cnt = nullptr;   // [0]: empty after the splat, [1 + i]: after sweep i
        FST_TRY(sc.get(&idx, ns));
        FST_TRY(sc.get(&fa, NG));
        FST_TRY(sc.get(&fb, NG));
        FST_TRY(sc.get(&cnt, max_sweeps + 1));
        FST_TRY(sample_rows(P.seed, Q, ns, idx, s));
        FST_CUDA(cudaMemsetAsync(bufA, 0, NG * sizeof(double), s));
        FST_CUDA(cudaMemsetAsync(bufB, 0, NG * sizeof(double), s));
        FST_CUDA(cudaMemsetAsync(cnt, 0, (max_sweeps + 1) * sizeof(unsigned long long), s));
        splat_kernel<<<grid_blocks(ns, 256), 256, 0, s>>>(xyz, u, Q, idx, ns, lo[0], lo[1], lo[2], hi[0], hi[1],
                                                           hi[2], I[0], I[1], I[2], bufA, bufB);
        FST_CHECK_LAUNCH();
        node_values_kernel<<<grid_blocks(NG, 256), 256, 0, s>>>(bufA, bufB, NG, fa, cnt);
        FST_CHECK_LAUNCH();
        std::vector<unsigned long long> hc(max_sweeps + 1);
        FST_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        if (hc[0] == (unsigned long long)NG) {
            set_error("fst_fit: no grid node received a sample");
            return FST_EINVAL;
        }
        // sweeps in batches of 8; a sweep over a completely filled grid copies it unchanged
        double* cur = bufA;
        double* nxt = bufB;
        uint8_t* fcur = fa;
        uint8_t* fnxt = fb;
        int done_at = hc[0] == 0 ? 0 : -1, swept = 0;
        while (done_at < 0 && swept < max_sweeps) {
            const int batch = std::min(8, max_sweeps - swept);
            for (int b = 0; b < batch; ++b) {
                fill_sweep_kernel<<<grid_blocks(NG, 256), 256, 0, s>>>(cur, fcur, nxt, fnxt, I[0], I[1], I[2],
                                                                       cnt + 1 + swept + b);
                FST_CHECK_LAUNCH();
                std::swap(cur, nxt);
                std::swap(fcur, fnxt);
            }
            FST_CUDA(cudaMemcpyAsync(hc.data() + 1 + swept, cnt + 1 + swept, batch * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
            FST_CUDA(cudaStreamSynchronize(s));
            for (int b = 0; b < batch && done_at < 0; ++b)
                if (hc[1 + swept + b] == 0) done_at = swept + b + 1;
            swept += batch;
        }
        if (done_at < 0) {
            set_error("fst_fit: grid fill did not finish in %d sweeps", max_sweeps);
            return FST_ENOTCONV;
        }
        rep.fill_sweeps = done_at;
        U = cur;
        other = nxt;
    }
    if (trace && trace->grid_values)
        FST_CUDA(cudaMemcpyAsync(trace->grid_values, U, NG * sizeof(double), cudaMemcpyDeviceToHost, s));
    tm.mark(1);

    // ---------------------------------------------------------------- step 2
    double* norm2_d = nullptr;
    double *S = nullptr, *V = nullptr, *lam_d = nullptr;
    int *order_d = nullptr, *sweeps_d = nullptr;
    double* W[3] = {nullptr, nullptr, nullptr};
    const int nmax = std::max(I[0], std::max(I[1], I[2]));
    FST_TRY(sc.get(&norm2_d, 1));
    FST_TRY(sc.get(&S, (size_t)nmax * nmax));
    FST_TRY(sc.get(&V, (size_t)nmax * nmax));
    FST_TRY(sc.get(&lam_d, nmax));
    FST_TRY(sc.get(&order_d, nmax));
    FST_TRY(sc.get(&sweeps_d, 1));
    sumsq_kernel<<<1, 1024, 0, s>>>(U, NG, norm2_d);
    FST_CHECK_LAUNCH();
    double norm2 = 0.0;
    FST_CUDA(cudaMemcpyAsync(&norm2, norm2_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    const double thr = P.eps * P.eps * norm2 / 3.0;
    int dims[3] = {I[0], I[1], I[2]};
    int r[3] = {0, 0, 0};
    double* X = U;
    double* Y = other;
    for (int k = 0; k < 3; ++k) {
        const int n = dims[k];
        const dim3 gb((n + 15) / 16, (n + 15) / 16), tb(16, 16);
        mode_gram_kernel<<<gb, tb, 0, s>>>(X, k, dims[0], dims[1], dims[2], S);
        FST_CHECK_LAUNCH();
        const int mpl = n + (n & 1);
        const size_t jsm = (size_t)(mpl / 2) * (2 * sizeof(double) + 2 * sizeof(int));
        jacobi_eig_kernel<<<1, kEigThreads, jsm, s>>>(S, V, n, kEigMaxSweeps, sweeps_d);
        FST_CHECK_LAUNCH();
        diag_kernel<<<1, 256, 0, s>>>(S, n, lam_d);
        FST_CHECK_LAUNCH();
        std::vector<double> lam(n);
        int sweeps = 0;
        FST_CUDA(cudaMemcpyAsync(lam.data(), lam_d, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaMemcpyAsync(&sweeps, sweeps_d, sizeof(int), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        rep.eig_sweeps[k] = sweeps;
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
        std::vector<double> lam_sorted(n), tail(n + 1, 0.0);
        for (int i = 0; i < n; ++i) lam_sorted[i] = lam[order[i]];
        for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + lam_sorted[i];
        const int cap = std::min(P.max_rank[k], n);
        int rk = cap;
        if (!P.fixed_rank) {
            rk = n;
            for (int rr = 1; rr <= n; ++rr)
                if (tail[rr] <= thr) {
                    rk = rr;
                    break;
                }
            rk = std::min(rk, cap);
        }
        r[k] = rk;
        if (trace && trace->eigvals[k]) std::copy(lam_sorted.begin(), lam_sorted.end(), trace->eigvals[k]);
        FST_TRY(sc.get(&W[k], (size_t)n * rk));
        FST_CUDA(cudaMemcpyAsync(order_d, order.data(), rk * sizeof(int), cudaMemcpyHostToDevice, s));
        select_vectors_kernel<<<rk, 256, 0, s>>>(V, n, order_d, rk, W[k]);
        FST_CHECK_LAUNCH();
        if (trace && trace->W[k])
            FST_CUDA(cudaMemcpyAsync(trace->W[k], W[k], (size_t)n * rk * sizeof(double), cudaMemcpyDeviceToHost, s));
        int nd[3] = {dims[0], dims[1], dims[2]};
        nd[k] = rk;
        const int64_t ny = (int64_t)nd[0] * nd[1] * nd[2];
        ttm_kernel<<<grid_blocks(ny, 256), 256, 0, s>>>(X, k, dims[0], dims[1], dims[2], W[k], rk, Y);
        FST_CHECK_LAUNCH();
        std::swap(X, Y);
        dims[k] = rk;
        // `order` (host) is read by the copy above: finish it before the vector goes away
        FST_CUDA(cudaStreamSynchronize(s));
    }
    const int R = r[0] * r[1] * r[2];
    std::vector<double> core(R);
    FST_CUDA(cudaMemcpyAsync(core.data(), X, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    tm.mark(2);

    // ---------------------------------------------------------------- step 3
    const int Pn = P.max_degree + 1;
    const int ncols = r[0] + r[1] + r[2];
    const bool wav = P.wavelet != 0;
    const int Pw = wav ? (P.wav_degree + 1) << P.wav_level : 0;
    const int njobs = wav ? 2 * ncols : ncols;          // Legendre fits, then (with wavelets) W_{s,q} fits
    double* Phi[3] = {nullptr, nullptr, nullptr};
    double* Phw[3] = {nullptr, nullptr, nullptr};
    LarsJob* jobs_d = nullptr;
    int32_t *rows_d = nullptr, *nnz_d = nullptr;
    double *coef_d = nullptr, *loo_d = nullptr;
    std::vector<LarsJob> jobs;
    std::vector<double> phw_h[3];
    for (int k = 0; k < 3; ++k) {
        FST_TRY(sc.get(&Phi[k], (size_t)I[k] * Pn));
        legendre_design_kernel<<<1, 256, 0, s>>>(I[k], Pn, Phi[k]);
        FST_CHECK_LAUNCH();
        for (int j = 0; j < r[k]; ++j) jobs.push_back(LarsJob{Phi[k], W[k], r[k], j, I[k], Pn});
    }
    if (wav)
        for (int k = 0; k < 3; ++k) {
            wavelet_grid_design(I[k], P.wav_level, P.wav_degree, phw_h[k]);
            FST_TRY(sc.get(&Phw[k], phw_h[k].size()));
            FST_CUDA(cudaMemcpyAsync(Phw[k], phw_h[k].data(), phw_h[k].size() * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
            for (int j = 0; j < r[k]; ++j) jobs.push_back(LarsJob{Phw[k], W[k], r[k], j, I[k], Pw});
        }
    FST_TRY(sc.get(&jobs_d, njobs));
    FST_TRY(sc.get(&rows_d, (size_t)njobs * kLarsMaxP));
    FST_TRY(sc.get(&coef_d, (size_t)njobs * kLarsMaxP));
    FST_TRY(sc.get(&nnz_d, njobs));
    FST_TRY(sc.get(&loo_d, njobs));
    FST_CUDA(cudaMemcpyAsync(jobs_d, jobs.data(), njobs * sizeof(LarsJob), cudaMemcpyHostToDevice, s));
    const size_t lsm = 2 * (size_t)kLarsMaxP * kLarsMaxP * sizeof(double);
    FST_TRY(allow_smem(lars_loo_kernel, lsm));
    lars_loo_kernel<<<njobs, kLarsThreads, lsm, s>>>(jobs_d, rows_d, coef_d, nnz_d, loo_d);
    FST_CHECK_LAUNCH();
    std::vector<int32_t> rows_h((size_t)njobs * kLarsMaxP), nnz_h(njobs);
    std::vector<double> coef_h((size_t)njobs * kLarsMaxP), loo_h(njobs);
    FST_CUDA(cudaMemcpyAsync(rows_h.data(), rows_d, rows_h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(coef_h.data(), coef_d, coef_h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(nnz_h.data(), nnz_d, njobs * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(loo_h.data(), loo_d, njobs * sizeof(double), cudaMemcpyDeviceToHost, s));
    std::vector<double> Wh[3];
    if (wav)
        for (int k = 0; k < 3; ++k) {
            Wh[k].resize((size_t)I[k] * r[k]);
            FST_CUDA(cudaMemcpyAsync(Wh[k].data(), W[k], Wh[k].size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    tm.mark(3);
    FST_CUDA(cudaStreamSynchronize(s));
    // Algorithm 1's basis choice: a column keeps its W_{s,q} fit when that fit's leave-one-out
    // error is below the Legendre fit's by more than 1e-12 mean(y^2); `pick[c]` is the job whose
    // fit the column keeps
    std::vector<int> pick(ncols);
    std::vector<uint8_t> chose(ncols, 0);
    {
        int c0 = 0;
        for (int k = 0; k < 3; ++k) {
            for (int j = 0; j < r[k]; ++j) {
                const int c = c0 + j;
                pick[c] = c;
                if (!wav) continue;
                double ms = 0.0;
                for (int i = 0; i < I[k]; ++i) ms += Wh[k][(size_t)i * r[k] + j] * Wh[k][(size_t)i * r[k] + j];
                ms /= I[k];
                if (loo_h[ncols + c] < loo_h[c] - 1e-12 * ms) {
                    pick[c] = ncols + c;
                    chose[c] = 1;
                }
            }
            c0 += r[k];
        }
    }
    if (trace && trace->core_hosvd) std::copy(core.begin(), core.end(), trace->core_hosvd);
    // step 4: drop dependent factor functions; the core keeps the matching slices
    std::vector<int32_t> colptr[3], rowidx[3];
    std::vector<double> val[3];
    std::vector<int> keep[3];
    int col0 = 0;
    int64_t nnz_total = 0;
    std::vector<uint8_t> colwav[3];
    for (int k = 0; k < 3; ++k) {
        for (int j = 0; j < r[k]; ++j) {
            const int c = col0 + j, pc = pick[c];
            if (trace && trace->col_nnz) trace->col_nnz[c] = nnz_h[pc];
            if (trace && trace->col_loo) trace->col_loo[c] = loo_h[pc];
            if (trace && trace->col_wavelet) trace->col_wavelet[c] = chose[c];
            if (trace && trace->col_loo_alt && wav) trace->col_loo_alt[c] = loo_h[chose[c] ? c : ncols + c];
        }
        if (!wav) {
            std::vector<double> C((size_t)Pn * r[k], 0.0);
            for (int j = 0; j < r[k]; ++j) {
                const int c = col0 + j;
                for (int i = 0; i < nnz_h[c]; ++i)
                    C[(size_t)j * Pn + rows_h[(size_t)c * kLarsMaxP + i]] = coef_h[(size_t)c * kLarsMaxP + i];
            }
            keep[k] = independent_columns(C, Pn, r[k]);
        } else {
            // mixed spaces: the functions' inner products from exact quadrature samples
            std::vector<const int32_t*> rr;
            std::vector<const double*> vv;
            std::vector<int> ln;
            std::vector<uint8_t> iw;
            for (int j = 0; j < r[k]; ++j) {
                const int pc = pick[col0 + j];
                rr.push_back(&rows_h[(size_t)pc * kLarsMaxP]);
                vv.push_back(&coef_h[(size_t)pc * kLarsMaxP]);
                ln.push_back(nnz_h[pc]);
                iw.push_back(chose[col0 + j]);
            }
            std::vector<double> Smp;
            int L = 0;
            function_samples(P.max_degree, P.wav_level, P.wav_degree, rr, vv, ln, iw, Smp, L);
            keep[k] = independent_columns(Smp, L, r[k]);
        }
        colptr[k].push_back(0);
        for (int j : keep[k]) {
            const int pc = pick[col0 + j];
            for (int i = 0; i < nnz_h[pc]; ++i) {
                rowidx[k].push_back(rows_h[(size_t)pc * kLarsMaxP + i]);
                val[k].push_back(coef_h[(size_t)pc * kLarsMaxP + i]);
            }
            colptr[k].push_back(colptr[k].back() + nnz_h[pc]);
            colwav[k].push_back(chose[col0 + j]);
            rep.n_wavelet[k] += chose[col0 + j];
        }
        if (trace && trace->col_kept)
            for (int j = 0; j < r[k]; ++j)
                trace->col_kept[col0 + j] = std::find(keep[k].begin(), keep[k].end(), j) != keep[k].end();
        rep.r_hosvd[k] = r[k];
        rep.r[k] = (int32_t)keep[k].size();
        rep.nnz[k] = colptr[k].back();
        nnz_total += colptr[k].back();
        col0 += r[k];
    }
    {
        std::vector<double> c2((size_t)keep[0].size() * keep[1].size() * keep[2].size());
        size_t e = 0;
        for (int a : keep[0])
            for (int b : keep[1])
                for (int c : keep[2]) c2[e++] = core[((size_t)a * r[1] + b) * r[2] + c];
        core.swap(c2);
        for (int k = 0; k < 3; ++k) r[k] = (int)keep[k].size();
    }

    fst_model_desc d{};
    for (int k = 0; k < 3; ++k) {
        d.r[k] = r[k];
        d.p[k] = P.max_degree;
        d.lo[k] = lo[k];
        d.hi[k] = hi[k];
        d.colptr[k] = colptr[k].data();
        d.rowidx[k] = rowidx[k].data();
        d.val[k] = val[k].data();
    }
    d.alpha = core.data();
    fst_model* model = nullptr;
    if (rep.n_wavelet[0] + rep.n_wavelet[1] + rep.n_wavelet[2] > 0) {
        fst_wavelet_desc w{};
        w.level = P.wav_level;
        w.degree = P.wav_degree;
        for (int k = 0; k < 3; ++k) w.col_wavelet[k] = colwav[k].data();
        FST_TRY(fst_model_create_wavelet(&d, &w, &model));
    } else {
        FST_TRY(fst_model_create(&d, &model));
    }

    // ---------------------------------------------------------------- step 4
    const int Rf = r[0] * r[1] * r[2];
    const int64_t m = std::min<int64_t>((int64_t)ceil(P.oversample * (double)Rf), Q);
    const uint64_t refit_seed = P.seed + kRefitSeedOffset;
    fst_status st = FST_OK;
    if (prec == FST_FP64) {
        double *xyz64 = nullptr, *u64 = nullptr;
        st = sc.get(&xyz64, (size_t)3 * Q);
        if (st == FST_OK) st = sc.get(&u64, Q);
        if (st == FST_OK) {
            widen_kernel<<<grid_blocks(3 * Q, 256), 256, 0, s>>>(xyz, xyz64, 3 * Q);
            count_launch();
            widen_kernel<<<grid_blocks(Q, 256), 256, 0, s>>>(u, u64, Q);
            count_launch();
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "widen_kernel", __FILE__, __LINE__);
        }
        if (st == FST_OK) st = fst_refit_f64(model, xyz64, u64, Q, nullptr, m, refit_seed, opts, &rep.refit, stream);
    } else {
        st = fst_refit(model, xyz, u, Q, nullptr, m, refit_seed, prec, opts, &rep.refit, stream);
    }
    if (st != FST_OK) {
        fst_model_free(model);
        return st;
    }
    tm.mark(4);
    FST_CUDA(cudaStreamSynchronize(s));
    rep.m = m;
    rep.compression_ratio = (double)Q / (double)(Rf + nnz_total);
    rep.ms_interp = tm.ms(0, 1);
    rep.ms_hosvd = tm.ms(1, 2);
    rep.ms_sparse = tm.ms(2, 3);
    rep.ms_refit = tm.ms(3, 4);
    if (report) *report = rep;
    *out = model;
    return FST_OK;
}
