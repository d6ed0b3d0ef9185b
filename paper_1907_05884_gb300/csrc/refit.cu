// refit.cu -- randomized least-squares re-estimation of the core (Sec. 5,
// eq. rand_core; Algorithm 2 with uniform row sampling) and its entry points.
//
//   alpha^ = argmin_alpha || b - A alpha ||,  A_{s,(i,j,k)} = w1_i(y1_s) w2_j(y2_s) w3_k(y3_s)
//
// over m sampled rows s.  Steps:
//   1. rows: given, or drawn by the splitmix64 key sampler (sample.cu);
//   2. factor values U_k[s][j] = w^(k)_j(y_k of row s), b_s = u of row s;
//   3. normal matrix G = A^T A, lower triangle, in the working precision, the Khatri-Rao
//      rows generated on the fly from U_1..U_3 (never stored), h = A^T b in FP64;
//   4. Cholesky G = L L^T (chol.cu) and alpha_0 = L^-T L^-1 h;
//   5. refinement alpha += L^-T L^-1 A^T (b - A alpha), residual and A^T r accumulated
//      in FP64 through the factored (Khatri-Rao) form of A, so the fixed point is the
//      least-squares solution even when G carries only working-precision accuracy.
// If the working-precision factorisation fails or refinement diverges, the FP64 path
// (FP64 G, FP64 Cholesky) is used.
#include <math.h>

#include <algorithm>
#include <functional>
#include <vector>
#include <thread>
#include <string>
#include <atomic>

#include "basis.cuh"

namespace fst {

// ------------------------------------------------------------------ step 2
// Factor values of the sampled rows, computed in FP64 from the stored points and rounded
// once to the working precision T (so the Khatri-Rao rows carry no recurrence error).
template <typename T, int RM>
__global__ void __launch_bounds__(128) sampled_factors_kernel(const EvalArgs<double> a, const T* __restrict__ xyz,
                                                              int64_t Q, const int64_t* __restrict__ idx,
                                                              int64_t m, const T* __restrict__ u, T* U1, T* U2,
                                                              T* U3, T* bvec) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = blockDim.x, tid = threadIdx.x;
    double* ra = reinterpret_cast<double*>(smem);
    double* rb = ra + a.pm;
    double* Ws[3];
    Ws[0] = rb + a.pm;
    Ws[1] = Ws[0] + a.pe[0] * RM;
    Ws[2] = Ws[1] + a.pe[1] * RM;
    uint8_t* mk = reinterpret_cast<uint8_t*>(Ws[2] + a.pe[2] * RM);
    for (int i = tid; i < a.pm; i += B) {
        ra[i] = double(2 * i + 1) / double(i + 1);
        rb[i] = double(i) / double(i + 1);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int rk = a.r[k];
        for (int e = tid; e < a.pe[k] * RM; e += B) {
            const int nn = e / RM, j = e - nn * RM;
            Ws[k][e] = j < rk ? a.W[k][nn * rk + j] : 0.0;
        }
        for (int e = tid; e < a.pm; e += B) mk[k * a.pm + e] = e < a.pe[k] ? a.mask[k][e] : 0;
    }
    __syncthreads();
    T* outs[3] = {U1, U2, U3};
    for (int64_t s = (int64_t)blockIdx.x * B + tid; s < m; s += (int64_t)gridDim.x * B) {
        const int64_t q = idx[s];
        bvec[s] = u[q];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double y[1] = {(double)xyz[k * Q + q]};
            double t[1] = {fma(y[0], a.sc[k], a.of[k])};
            double acc[1][RM];
            factor_values<double, RM, 1>(t, Ws[k], mk + k * a.pm, a.pe[k], ra, rb, acc);
            piecewise_values<double, RM, 1>(y, t, a, k, acc);
            const int rk = a.r[k];
            for (int j = 0; j < rk; ++j) outs[k][s * rk + j] = (T)acc[0][j];
        }
    }
}

// ------------------------------------------------------------------ step 3 (CUDA cores)
// Lower 64x64 tiles of G = A^T A; K loop over sampled rows in chunks of 32.
template <typename T>
__global__ void __launch_bounds__(256) gram_simt_kernel(const T* __restrict__ U1, const T* __restrict__ U2,
                                                        const T* __restrict__ U3, int64_t m, int r1, int r2,
                                                        int r3, T* G) {
    constexpr int TS = 64, KC = 32;
    __shared__ __align__(16) T As[KC][TS];
    __shared__ __align__(16) T Bs[KC][TS];
    const int R = r1 * r2 * r3;
    const long long b = blockIdx.x;
    int ti = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while ((long long)ti * (ti + 1) / 2 > b) --ti;
    const int tc = (int)(b - (long long)ti * (ti + 1) / 2);
    const int tid = threadIdx.x;
    // the column of A this thread generates for the row tile and the column tile
    const int col = tid & 63, soff = tid >> 6;
    const int ar = ti * TS + col, ac = tc * TS + col;
    const bool vr = ar < R, vc = ac < R;
    const int ir = vr ? ar / (r2 * r3) : 0, jr = vr ? (ar / r3) % r2 : 0, kr = vr ? ar % r3 : 0;
    const int ic = vc ? ac / (r2 * r3) : 0, jc = vc ? (ac / r3) % r2 : 0, kc = vc ? ac % r3 : 0;
    const int ty = tid >> 4, tx = tid & 15;
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
    for (int64_t s0 = 0; s0 < m; s0 += KC) {
        __syncthreads();
#pragma unroll
        for (int l = 0; l < KC / 4; ++l) {
            const int ss = soff + 4 * l;
            const int64_t s = s0 + ss;
            T vr_v = T(0), vc_v = T(0);
            if (s < m) {
                if (vr) vr_v = U1[s * r1 + ir] * U2[s * r2 + jr] * U3[s * r3 + kr];
                if (vc) vc_v = U1[s * r1 + ic] * U2[s * r2 + jc] * U3[s * r3 + kc];
            }
            As[ss][col] = vr_v;
            Bs[ss][col] = vc_v;
        }
        __syncthreads();
#pragma unroll 8
        for (int t = 0; t < KC; ++t) {
            T av[4], bv[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) av[x] = As[t][ty * 4 + x];
#pragma unroll
            for (int y = 0; y < 4; ++y) bv[y] = Bs[t][tx * 4 + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int i = ti * TS + ty * 4 + x;
        if (i >= R) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int j = tc * TS + tx * 4 + y;
            if (j < R && j <= i) G[(size_t)i * R + j] = acc[x][y];
        }
    }
}

// ------------------------------------------------------------------ A^T r and b - A alpha
// Partial sums of g = A^T r over a chunk of rows per block: each thread owns three (i,j)
// pairs and their r3 accumulators (so every w3 row read feeds 3 r3 products); rows are
// staged through shared memory.  Block b writes its R partial sums to part[b * R ..];
// sum_partials_kernel adds them in FP64 (deterministic, no atomics).
template <typename T, int R3M, int PPT>
__device__ __forceinline__ void atr_body(const T* __restrict__ U1, const T* __restrict__ U2,
                                         const T* __restrict__ U3, const double* __restrict__ rv, int64_t m, int r1,
                                         int r2, int r3, int64_t rows_per_block, double* __restrict__ part, int blk) {
    constexpr int S = 64;
    __shared__ T u1s[S][FST_MAX_RANK + 1], u2s[S][FST_MAX_RANK + 1];
    __shared__ __align__(16) T u3s[S][R3M];
    __shared__ T rs[S];
    const int64_t lo = (int64_t)blk * rows_per_block;
    const int64_t hi = lo + rows_per_block < m ? lo + rows_per_block : m;
    const int npairs = r1 * r2;
    double* out = part + (size_t)blk * npairs * r3;
    for (int p0 = 0; p0 < npairs; p0 += PPT * blockDim.x) {
        int pi[PPT], pj[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int pair = p0 + threadIdx.x + p * blockDim.x;
            pi[p] = pair < npairs ? pair / r2 : 0;
            pj[p] = pair < npairs ? pair % r2 : 0;
        }
        T acc[PPT][R3M];
#pragma unroll
        for (int p = 0; p < PPT; ++p)
#pragma unroll
            for (int k = 0; k < R3M; ++k) acc[p][k] = T(0);
        for (int64_t s0 = lo; s0 < hi; s0 += S) {
            __syncthreads();
            // staging unrolled so that a thread's loads are in flight together
#pragma unroll 8
            for (int e = threadIdx.x; e < S * FST_MAX_RANK; e += blockDim.x) {
                const int ss = e / FST_MAX_RANK, c = e - ss * FST_MAX_RANK;
                const int64_t s = s0 + ss;
                const bool ok = s < hi;
                const T a = (ok && c < r1) ? U1[s * r1 + c] : T(0);
                const T b = (ok && c < r2) ? U2[s * r2 + c] : T(0);
                const T w = (ok && c < r3) ? U3[s * r3 + c] : T(0);
                const T rr = (ok && c == 0) ? (T)rv[s] : T(0);
                if (c < r1) u1s[ss][c] = a;
                if (c < r2) u2s[ss][c] = b;
                if (c < R3M) u3s[ss][c] = w;
                if (c == 0) rs[ss] = rr;
            }
            __syncthreads();
#pragma unroll 2
            for (int ss = 0; ss < S; ++ss) {
                T w3[R3M];
#pragma unroll
                for (int k = 0; k < R3M; k += 4) load4(&u3s[ss][k], w3[k], w3[k + 1], w3[k + 2], w3[k + 3]);
                const T r = rs[ss];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const T c = r * u1s[ss][pi[p]] * u2s[ss][pj[p]];
#pragma unroll
                    for (int k = 0; k < R3M; ++k) acc[p][k] = fma(c, w3[k], acc[p][k]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int pair = p0 + threadIdx.x + p * blockDim.x;
            if (pair < npairs) {
#pragma unroll
                for (int k = 0; k < R3M; ++k)
                    if (k < r3) out[(size_t)pair * r3 + k] = (double)acc[p][k];
            }
        }
    }
}

template <typename T, int R3M, int PPT>
__global__ void __launch_bounds__(256) atr_kernel(const T* __restrict__ U1, const T* __restrict__ U2,
                                                  const T* __restrict__ U3, const double* __restrict__ rv,
                                                  int64_t m, int r1, int r2, int r3, int64_t rows_per_block,
                                                  double* __restrict__ part, const int* stop) {
    if (stop && *stop) return;
    atr_body<T, R3M, PPT>(U1, U2, U3, rv, m, r1, r2, r3, rows_per_block, part, blockIdx.x);
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int nparts, int R, double* __restrict__ g,
                                    const int* stop) {
    if (stop && *stop) return;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < R; a += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * R + a];
        g[a] = s;
    }
}

// r_s = b_s - sum_i w1_i sum_j w2_j sum_k alpha_ijk w3_k (or, with scale +1 and no b, the
// product A alpha).  The sums over k and j run in T; for T = float alpha is split into
// alpha_hi + alpha_lo (both FP32) so the core keeps its FP64 digits; the sum over i and the
// subtraction from b run in FP64.
constexpr int kMaxRank = FST_MAX_RANK;
template <typename T, int R3M>
__device__ __forceinline__ void residual_body(const T* __restrict__ U1, const T* __restrict__ U2,
                                              const T* __restrict__ U3, const T* __restrict__ bvec,
                                              const double* __restrict__ alpha, int64_t m, int r1, int r2, int r3,
                                              double scale, double* rv, int blk, int nblk) {
    constexpr bool kSplit = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smem[];
    T* As = reinterpret_cast<T*>(smem);        // [r1*r2][R3M]
    T* Al = As + r1 * r2 * R3M;                // low parts (FP32 only)
    for (int e = threadIdx.x; e < r1 * r2 * R3M; e += blockDim.x) {
        const int ij = e / R3M, k = e - ij * R3M;
        const double a = k < r3 ? alpha[ij * r3 + k] : 0.0;
        const T hi = (T)a;
        As[e] = hi;
        if (kSplit) Al[e] = (T)(a - (double)hi);
    }
    __syncthreads();
    for (int64_t s = (int64_t)blk * blockDim.x + threadIdx.x; s < m; s += (int64_t)nblk * blockDim.x) {
        // the row's factor values in registers (w2 indexed by the unrolled j loop)
        T w3[R3M], w2[kMaxRank];
#pragma unroll
        for (int k = 0; k < R3M; ++k) w3[k] = k < r3 ? U3[s * r3 + k] : T(0);
#pragma unroll
        for (int j = 0; j < kMaxRank; ++j) w2[j] = j < r2 ? U2[s * r2 + j] : T(0);
        double f = 0.0;
        for (int i = 0; i < r1; ++i) {
            T si = T(0);
#pragma unroll
            for (int j = 0; j < kMaxRank; ++j) {
                if (j < r2) {
                    const T* arow = As + (i * r2 + j) * R3M;
                    T t0 = T(0), t1 = T(0);
#pragma unroll
                    for (int k = 0; k < R3M; k += 4) {
                        T a0, a1, a2, a3;
                        load4(arow + k, a0, a1, a2, a3);
                        t0 = fma(a0, w3[k], t0);
                        t1 = fma(a1, w3[k + 1], t1);
                        t0 = fma(a2, w3[k + 2], t0);
                        t1 = fma(a3, w3[k + 3], t1);
                    }
                    T t = t0 + t1;
                    if (kSplit) {
                        const T* lrow = Al + (i * r2 + j) * R3M;
                        T l0 = T(0), l1 = T(0);
#pragma unroll
                        for (int k = 0; k < R3M; k += 4) {
                            T a0, a1, a2, a3;
                            load4(lrow + k, a0, a1, a2, a3);
                            l0 = fma(a0, w3[k], l0);
                            l1 = fma(a1, w3[k + 1], l1);
                            l0 = fma(a2, w3[k + 2], l0);
                            l1 = fma(a3, w3[k + 3], l1);
                        }
                        t += l0 + l1;
                    }
                    si = fma(t, w2[j], si);
                }
            }
            f = fma((double)si, (double)U1[s * r1 + i], f);
        }
        rv[s] = (bvec ? (double)bvec[s] : 0.0) + scale * f;
    }
}

template <typename T, int R3M>
__global__ void __launch_bounds__(256) residual_kernel(const T* __restrict__ U1, const T* __restrict__ U2,
                                                       const T* __restrict__ U3, const T* __restrict__ bvec,
                                                       const double* __restrict__ alpha, int64_t m, int r1,
                                                       int r2, int r3, double scale, double* rv,
                                                       const int* stop) {
    if (stop && *stop) return;   // the conjugate gradients have stopped
    residual_body<T, R3M>(U1, U2, U3, bvec, alpha, m, r1, r2, r3, scale, rv, blockIdx.x, gridDim.x);
}

// Relative diagonal shift of the preconditioner's matrix, G_jj <- (1 + delta) G_jj: the
// factor of G + delta diag(G) still preconditions the conjugate gradients, which solve the
// unshifted normal equations.
constexpr float kPrecondShift = 2.44140625e-4f;   // 2^-12
__global__ void shift_diag_kernel(float* G, int R, float delta) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x)
        G[(size_t)i * R + i] *= 1.f + delta;
}

// out[k] = sum_i x_k[i] * y_k[i] for k < nd, by one block in a fixed order, so that a refit
// repeats bit for bit (the step lengths of the conjugate gradients depend on these sums)
constexpr int kDotThreads = 1024;
__device__ __forceinline__ void dots_body(const double* x0, const double* y0, const double* x1, const double* y1,
                                          int n, int nd, double* out) {
    __shared__ double red[2][kDotThreads / 32];
    double a0 = 0.0, a1 = 0.0;
    for (int i = threadIdx.x; i < n; i += kDotThreads) {
        a0 += x0[i] * y0[i];
        if (nd > 1) a1 += x1[i] * y1[i];
    }
    for (int o = 16; o; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = a0;
        red[1][warp] = a1;
    }
    __syncthreads();
    if (warp == 0) {
        a0 = red[0][lane];
        a1 = red[1][lane];
        for (int o = 16; o; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            out[0] = a0;
            if (nd > 1) out[1] = a1;
        }
    }
}
__global__ void __launch_bounds__(kDotThreads) dots_kernel(const double* x0, const double* y0, const double* x1,
                                                           const double* y1, int n, int nd, double* out) {
    dots_body(x0, y0, x1, y1, n, nd, out);
}

// Scalars of the conjugate gradients, kept on the device so that iterations are launched
// without a host round trip; stop: 1 converged, 2 broke down (not converged).
struct PcgState {
    double rz, ak, pp2, beta, last, prev;
    int stop, steps;
};

__device__ __forceinline__ void pcg_init_body(const double* __restrict__ norms, PcgState* st) {
    st->rz = norms[0];
    st->ak = st->pp2 = st->beta = st->last = st->prev = 0.0;
    st->stop = 0;
    st->steps = 0;
}
__global__ void pcg_init_kernel(const double* __restrict__ norms, PcgState* st) { pcg_init_body(norms, st); }

// after w = A^T A p: norms = (p.w, p.p); the step length
__device__ __forceinline__ void pcg_step_length_body(const double* __restrict__ norms, PcgState* st) {
    if (st->stop) return;
    const double pw = norms[0];
    if (!(pw > 0.0) || !isfinite(st->rz)) {
        st->stop = 2;
        return;
    }
    st->ak = st->rz / pw;
    st->pp2 = norms[1];
}
__global__ void pcg_step_length_kernel(const double* __restrict__ norms, PcgState* st) { pcg_step_length_body(norms, st); }

// after z = M^-1 r: norms = (r.z, alpha.alpha); the relative update and the stopping rule
// (below tol, or no longer shrinking at a level below floor_ok), else the next direction's beta
__device__ __forceinline__ void pcg_step_end_body(const double* __restrict__ norms, PcgState* st, double tol, double floor_ok) {
    if (st->stop) return;
    st->steps += 1;
    st->prev = st->last;
    const double nx0 = norms[0], nx1 = norms[1];
    const double last = nx1 > 0 ? fabs(st->ak) * sqrt(st->pp2 / nx1) : 0.0;
    st->last = last;
    if (!isfinite(last)) {
        st->stop = 2;
        return;
    }
    if (last <= tol || (st->steps >= 3 && last > 0.5 * st->prev && last <= floor_ok)) {
        st->stop = 1;
        return;
    }
    st->beta = nx0 / st->rz;
    st->rz = nx0;
}
__global__ void pcg_step_end_kernel(const double* __restrict__ norms, PcgState* st, double tol, double floor_ok) { pcg_step_end_body(norms, st, tol, floor_ok); }

// alpha += ak p (which 0), r -= ak w (1), p = z + beta p (2), with the scalars of st
__global__ void pcg_axpy_kernel(double* y, const double* x, const PcgState* st, int which, int n) {
    if (st->stop) return;
    const double a = which == 0 ? st->ak : which == 1 ? -st->ak : st->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = which == 2 ? x[i] + a * y[i] : y[i] + a * x[i];
}

template <typename T>
__global__ void to_double_kernel(const T* src, double* dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

template <typename T>
__global__ void from_double_kernel(const double* src, T* dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// ------------------------------------------------------------------ grouped refits
// The conjugate gradients of several refits advanced in shared launches: job j carries the
// vectors of one refit, and each kernel below does one step of the single-refit sequence for
// every job at once, with the single kernels' arithmetic (the same bodies and reduction
// orders), so a job's iterates equal those of its own refit bit for bit.
enum PcgVec { vRV = 0, vG, vAlpha, vAlpha0, vRR, vZZ, vPP, vWW, kPcgVecs };
struct PcgJob {
    const float* U1;
    const float* U2;
    const float* U3;
    const float* b;
    int64_t m;
    int r1, r2, r3, R;
    double* v[kPcgVecs];   // rv (m), then the R-vectors g, alpha, alpha0, r, z, p, w
    double* norms;
    double* part;          // A^T partial sums (nparts x R)
    PcgState* st;
    float* xw;             // the preconditioner solve's working copy
    int nparts, parts_per_block;   // A^T partition (the single refit's) and parts a block takes
    int64_t rows_per_block;
    long long rfirst, afirst;   // first block in its class's residual / A^T launch
};
template <long long PcgJob::*F>
__device__ __forceinline__ int pcg_job_of(const PcgJob* jobs, int n, long long x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].*F <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// rv = (b if use_b) + scale * A v[src], for the jobs of one rank class
template <int R3M>
__global__ void __launch_bounds__(256) residual_group_kernel(const PcgJob* __restrict__ jobs, int n, int src,
                                                             int use_b, double scale, int gated) {
    const int q = pcg_job_of<&PcgJob::rfirst>(jobs, n, blockIdx.x);
    const PcgJob& j = jobs[q];
    if (gated && j.st->stop) return;
    const long long nb = (q + 1 < n ? jobs[q + 1].rfirst : (long long)gridDim.x) - j.rfirst;
    residual_body<float, R3M>(j.U1, j.U2, j.U3, use_b ? j.b : nullptr, j.v[src], j.m, j.r1, j.r2, j.r3, scale,
                              j.v[vRV], (int)(blockIdx.x - j.rfirst), (int)nb);
}

// the partial sums of A^T rv (the single refit's row partition)
template <int R3M, int PPT>
__global__ void __launch_bounds__(256) atr_group_kernel(const PcgJob* __restrict__ jobs, int n, int gated) {
    const int q = pcg_job_of<&PcgJob::afirst>(jobs, n, blockIdx.x);
    const PcgJob& j = jobs[q];
    if (gated && j.st->stop) return;
    const int b0 = (int)(blockIdx.x - j.afirst) * j.parts_per_block;
    const int b1 = b0 + j.parts_per_block < j.nparts ? b0 + j.parts_per_block : j.nparts;
    for (int b = b0; b < b1; ++b)
        atr_body<float, R3M, PPT>(j.U1, j.U2, j.U3, j.v[vRV], j.m, j.r1, j.r2, j.r3, j.rows_per_block, j.part, b);
}

__global__ void sum_partials_group_kernel(const PcgJob* __restrict__ jobs, int dst, int gated) {
    const PcgJob& j = jobs[blockIdx.y];
    if (gated && j.st->stop) return;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < j.R; a += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int b = 0; b < j.nparts; ++b) sum += j.part[(size_t)b * j.R + a];
        j.v[dst][a] = sum;
    }
}

__global__ void __launch_bounds__(kDotThreads) dots_group_kernel(const PcgJob* __restrict__ jobs, int x0, int y0,
                                                                 int x1, int y1) {
    const PcgJob& j = jobs[blockIdx.x];
    dots_body(j.v[x0], j.v[y0], j.v[x1], j.v[y1], j.R, 2, j.norms);
}

// kind 0: init, 1: step length, 2: step end (one thread a job)
__global__ void pcg_scalar_group_kernel(const PcgJob* __restrict__ jobs, int n, int kind, double tol,
                                        double floor_ok) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const PcgJob& j = jobs[q];
    if (kind == 0) pcg_init_body(j.norms, j.st);
    else if (kind == 1) pcg_step_length_body(j.norms, j.st);
    else pcg_step_end_body(j.norms, j.st, tol, floor_ok);
}

// alpha += ak p (which 0), r -= ak w (1), p = z + beta p (2)
__global__ void pcg_axpy_group_kernel(const PcgJob* __restrict__ jobs, int which) {
    const PcgJob& j = jobs[blockIdx.y];
    const PcgState* st = j.st;
    if (st->stop) return;
    const double a = which == 0 ? st->ak : which == 1 ? -st->ak : st->beta;
    double* y = j.v[which == 0 ? vAlpha : which == 1 ? vRR : vPP];
    const double* x = j.v[which == 0 ? vPP : which == 1 ? vWW : vZZ];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < j.R; i += gridDim.x * blockDim.x)
        y[i] = which == 2 ? x[i] + a * y[i] : y[i] + a * x[i];
}

// v[dst] = v[src]; dir 0: xw = (float) v[vec]; dir 1: v[vec] = xw (all R-vectors)
__global__ void pcg_copy_group_kernel(const PcgJob* __restrict__ jobs, int dst, int src) {
    const PcgJob& j = jobs[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < j.R; i += gridDim.x * blockDim.x) j.v[dst][i] = j.v[src][i];
}
__global__ void pcg_convert_group_kernel(const PcgJob* __restrict__ jobs, int vec, int dir) {
    const PcgJob& j = jobs[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < j.R; i += gridDim.x * blockDim.x) {
        if (dir == 0) j.xw[i] = (float)j.v[vec][i];
        else j.v[vec][i] = (double)j.xw[i];
    }
}
__global__ void pcg_gather_states_kernel(const PcgJob* __restrict__ jobs, int n, PcgState* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = *jobs[q].st;
}

// ------------------------------------------------------------------ driver
struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit EventTimer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventRecord(a, s);
        return ms;
    }
    ~EventTimer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

static int grid_for(int64_t n, int block, int cap_per_sm = 8) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)sm_count() * cap_per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

template <typename T>
static fst_status launch_factors(const fst_model* M, const T* xyz, int64_t Q, const int64_t* idx, int64_t m,
                                 const T* u, T* U[3], T* bvec, cudaStream_t s) {
    EvalArgs<double> a = make_args<double>(M);
    bind(a, M);
    int rmax = M->r[0] > M->r[1] ? M->r[0] : M->r[1];
    rmax = M->r[2] > rmax ? M->r[2] : rmax;
    const int RMb = rmax <= 8 ? 8 : rmax <= 16 ? 16 : rmax <= 24 ? 24 : 32;
    const size_t smem = (2 * (size_t)a.pm + (size_t)(a.pe[0] + a.pe[1] + a.pe[2]) * RMb) * sizeof(double) + 3 * a.pm;
#define FST_FACT(RMV)                                                                                      \
    {                                                                                                      \
        auto kern = sampled_factors_kernel<T, RMV>;                                                        \
        FST_TRY(allow_smem(kern, smem));      \
        kern<<<grid_for(m, 128), 128, smem, s>>>(a, xyz, Q, idx, m, u, U[0], U[1], U[2], bvec);           \
    }
    if (RMb == 8) FST_FACT(8) else if (RMb == 16) FST_FACT(16) else if (RMb == 24) FST_FACT(24) else FST_FACT(32)
#undef FST_FACT
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <typename T>
static fst_status launch_atr(const fst_model* M, const T* const U[3], const double* rv, int64_t m, double* g,
                             cudaStream_t s, const int* stop = nullptr) {
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    const int R = M->R();
    if (m <= 0) {
        FST_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * (size_t)R, s));
        return FST_OK;
    }
    // pairs per thread: as many as the registers allow (3 x r3 <= 24 accumulators in FP32)
    const int ppt = sizeof(T) == 8 ? 1 : (r3 <= 24 ? 3 : 2);
    int threads = ((r1 * r2 + ppt - 1) / ppt + 31) / 32 * 32;
    if (threads > 256) threads = 256;
    int64_t nparts = 2LL * sm_count();
    int64_t rows_per_block = ((m + nparts - 1) / nparts + 31) / 32 * 32;
    nparts = (m + rows_per_block - 1) / rows_per_block;
    // per-model scratch (the caller holds the model's lock), so refits of different models on
    // different streams never share it
    DevBuf& pb = const_cast<fst_model*>(M)->rs.atr_part;
    FST_TRY(pb.ensure(sizeof(double) * (size_t)nparts * R));
    double* part = pb.as<double>();
    const unsigned grid = (unsigned)nparts;
#define FST_ATR(R3V, PPTV) \
    atr_kernel<T, R3V, PPTV><<<grid, threads, 0, s>>>(U[0], U[1], U[2], rv, m, r1, r2, r3, rows_per_block, part, stop)
    if (sizeof(T) == 8) {
        if (r3 <= 8) FST_ATR(8, 1);
        else if (r3 <= 16) FST_ATR(16, 1);
        else if (r3 <= 24) FST_ATR(24, 1);
        else FST_ATR(32, 1);
    } else {
        if (r3 <= 8) FST_ATR(8, 3);
        else if (r3 <= 16) FST_ATR(16, 3);
        else if (r3 <= 24) FST_ATR(24, 3);
        else FST_ATR(32, 2);
    }
#undef FST_ATR
    FST_CHECK_LAUNCH();
    sum_partials_kernel<<<(R + 255) / 256, 256, 0, s>>>(part, (int)nparts, R, g, stop);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <typename T>
static fst_status launch_residual(const fst_model* M, const T* const U[3], const T* bvec, const double* alpha,
                                  int64_t m, double* rv, cudaStream_t s, double scale = -1.0,
                                  const int* stop = nullptr) {
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    const int R3M = r3 <= 8 ? 8 : r3 <= 16 ? 16 : r3 <= 24 ? 24 : 32;
    const size_t smem = (size_t)r1 * r2 * R3M * sizeof(T) * (sizeof(T) == 4 ? 2 : 1);
    // 256 threads a block: two blocks (16 warps) fit beside the core's hi/lo copy at r = 24
    const int grid = grid_for(m, 256, 2);
#define FST_RES(V)                                                                                          \
    {                                                                                                       \
        auto kern = residual_kernel<T, V>;                                                                  \
        FST_TRY(allow_smem(kern, smem));                                                                    \
        kern<<<grid, 256, smem, s>>>(U[0], U[1], U[2], bvec, alpha, m, r1, r2, r3, scale, rv, stop);        \
    }
    if (R3M == 8) FST_RES(8) else if (R3M == 16) FST_RES(16) else if (R3M == 24) FST_RES(24) else FST_RES(32)
#undef FST_RES
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <typename T>
static fst_status launch_gram_simt(const fst_model* M, const T* const U[3], int64_t m, T* G, cudaStream_t s) {
    const int R = M->R();
    const long long nt = (R + 63) / 64;
    gram_simt_kernel<T><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(U[0], U[1], U[2], m, M->r[0], M->r[1],
                                                                      M->r[2], G);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

// Tensor-core Gram: from the packed Khatri-Rao operand; without memory for the packed copy,
// the kernel that generates the operand on the fly; for r3 < 4 there, the CUDA-core Gram.
static fst_status gram_tensor(const fst_model* M, const float* const U[3], int64_t m, float* G, fst_prec prec,
                              cudaStream_t s) {
    fst_status st = gram_pk_launch(M, U[0], U[1], U[2], m, G, prec, s);
    if (st != FST_ENOMEM) return st;
    st = gram_tc_launch(M, U[0], U[1], U[2], m, G, prec, s);
    if (st == FST_EUNSUPPORTED) st = launch_gram_simt<float>(M, U, m, G, s);
    return st;
}

// Working precision T for factors, Gram and Cholesky; FP64 vectors and refinement.
template <typename T>
static fst_status refit_impl(fst_model* M, const T* xyz, const T* u, int64_t Q, const int64_t* idx_in, int64_t m,
                             uint64_t seed, fst_prec prec, const fst_refit_opts* opts, fst_refit_report* rep,
                             cudaStream_t s) {
    const int R = M->R();
    RefitScratch& W = M->rs;
    const bool fp64 = sizeof(T) == 8;
    const int max_refine = opts ? opts->max_refine : 32;
    // FP32-valued factors bound the attainable accuracy near 1e-7: stop the CG at 1e-8
    const double tol = (opts && opts->refine_tol > 0) ? opts->refine_tol : (fp64 ? 1e-13 : 1e-8);
    const bool force64 = opts && opts->fp64_cholesky;
    fst_refit_report r;
    memset(&r, 0, sizeof r);
    r.m = m;

    EventTimer tm(s);
    // 1. rows
    const int64_t* idx = idx_in;
    if (!idx) {
        FST_TRY(W.idx.ensure(sizeof(int64_t) * (size_t)m));
        FST_TRY(sample_rows(seed, Q, m, W.idx.as<int64_t>(), s));
        idx = W.idx.as<int64_t>();
    }
    r.ms_sample = tm.stop();
    // 2. factor values of the sampled rows
    T* U[3];
    for (int k = 0; k < 3; ++k) {
        FST_TRY(W.U[k].ensure(sizeof(T) * (size_t)m * M->r[k]));
        U[k] = W.U[k].as<T>();
    }
    FST_TRY(W.b.ensure(sizeof(T) * (size_t)m));
    T* bvec = W.b.as<T>();
    FST_TRY(launch_factors<T>(M, xyz, Q, idx, m, u, U, bvec, s));
    r.ms_factors = tm.stop();

    FST_TRY(W.res.ensure(sizeof(double) * (size_t)m));
    FST_TRY(W.g.ensure(sizeof(double) * (size_t)R));
    FST_TRY(W.alpha.ensure(sizeof(double) * (size_t)R));
    FST_TRY(W.z.ensure(sizeof(double) * (size_t)R));
    FST_TRY(W.norms.ensure(sizeof(double) * 2));
    FST_TRY(W.flag.ensure(4 * sizeof(int)));   // flag + 8-byte aligned pivot floor
    double* rv = W.res.as<double>();
    double* g = W.g.as<double>();
    double* alpha = W.alpha.as<double>();
    double* alpha0 = W.z.as<double>();
    double* norms = W.norms.as<double>();
    int* flag = W.flag.as<int>();
    const T* const Uc[3] = {U[0], U[1], U[2]};

    // h = A^T b
    {
        const int grid = grid_for(m, 256);
        to_double_kernel<T><<<grid, 256, 0, s>>>(bvec, rv, m);
        FST_CHECK_LAUNCH();
    }
    FST_TRY(launch_atr<T>(M, Uc, rv, m, g, s));

    // 3-4. Gram and Cholesky in the working precision; if the FP32 factorisation of a
    // TF32 / BF16 Gram fails, the BF16x3 Gram (near-FP32 products) is tried next, then FP64
    bool use64 = fp64 || force64;
    fst_prec gram_prec = prec;
    bool shift = false;
    void* Lp = nullptr;
    for (int attempt = 0; attempt < 4; ++attempt) {
        FST_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), s));
        if (!use64) {
            FST_TRY(W.G.ensure(sizeof(float) * (size_t)R * R));
            float* G = W.G.as<float>();
            if (gram_prec == FST_FP32) {
                FST_TRY(launch_gram_simt<float>(M, reinterpret_cast<const float* const*>(Uc), m, G, s));
            } else {
                FST_TRY(gram_tensor(M, reinterpret_cast<const float* const*>(Uc), m, G, gram_prec, s));
            }
            r.ms_gram += tm.stop();
            if (shift) {
                shift_diag_kernel<<<grid_for(R, 256), 256, 0, s>>>(G, R, kPrecondShift);
                FST_CHECK_LAUNCH();
            }
            FST_TRY(cholesky_lower<float>(G, R, flag, W.chol_ws, s));
            Lp = G;
        } else {
            FST_TRY(W.G64.ensure(sizeof(double) * (size_t)R * R));
            double* G = W.G64.as<double>();
            const double* U64[3];
            if (fp64) {
                for (int k = 0; k < 3; ++k) U64[k] = reinterpret_cast<const double*>(Uc[k]);
            } else {
                // promote the working-precision factor values
                FST_TRY(W.delta.ensure(sizeof(double) * (size_t)m * (M->r[0] + M->r[1] + M->r[2])));
                double* base = W.delta.as<double>();
                for (int k = 0; k < 3; ++k) {
                    const int64_t n = m * M->r[k];
                    to_double_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(Uc[k], base, n);
                    FST_CHECK_LAUNCH();
                    U64[k] = base;
                    base += n;
                }
            }
            FST_TRY(launch_gram_simt<double>(M, U64, m, G, s));
            r.ms_gram += tm.stop();
            FST_TRY(cholesky_lower<double>(G, R, flag, W.chol_ws, s));
            Lp = G;
        }
        if (use64) {
            FST_TRY(W.Linv.ensure(3 * sizeof(double) * (size_t)((R + 63) / 64) * 64 * 64));   // + link matrices
            FST_TRY(chol_invert_diag<double>(static_cast<const double*>(Lp), R, W.Linv.as<double>(), s));
            FST_TRY(W.LT.ensure(sizeof(double) * (size_t)R * R));
            FST_TRY(chol_transpose<double>(static_cast<const double*>(Lp), R, W.LT.as<double>(), s));
        } else {
            FST_TRY(W.Linv.ensure(3 * sizeof(float) * (size_t)((R + 63) / 64) * 64 * 64));   // + link matrices
            FST_TRY(chol_invert_diag<float>(static_cast<const float*>(Lp), R, W.Linv.as<float>(), s));
            FST_TRY(W.LT.ensure(sizeof(float) * (size_t)R * R));
            FST_TRY(chol_transpose<float>(static_cast<const float*>(Lp), R, W.LT.as<float>(), s));
        }
        int hflag[2] = {0, 0};
        FST_CUDA(cudaMemcpyAsync(hflag, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        r.ms_cholesky += tm.stop();
        if (hflag[1]) {
            set_error("Cholesky: a bounded device wait expired (code %d)", hflag[1]);
            if (rep) *rep = r;
            return FST_ETIMEOUT;
        }
        if (!hflag[0]) break;
        if (use64) {
            set_error("normal matrix is not positive definite in FP64 (rank-deficient sample)");
            if (rep) *rep = r;
            return FST_ENOTSPD;
        }
        if (gram_prec == FST_TF32 || gram_prec == FST_BF16) {
            gram_prec = FST_BF16X3;
            r.fallback_bf16x3 = 1;
        } else if (!shift && gram_prec != FST_FP32) {
            shift = true;
            r.shifted_preconditioner = 1;
        } else {
            use64 = true;
            r.fallback_fp64 = 1;
        }
    }

    // the preconditioner solve runs in the factor's precision on a working copy
    FST_TRY(W.xw.ensure(sizeof(double) * (size_t)R));
    FST_TRY(W.yw.ensure(sizeof(double) * (size_t)R));
    // the CG state (its stop word also gates the solves, so the captured solve graph is the
    // same for every call); zeroed before the first solve
    FST_TRY(W.pcg_state.ensure(sizeof(PcgState)));
    PcgState* pst = W.pcg_state.as<PcgState>();
    const int* stop = &pst->stop;
    FST_CUDA(cudaMemsetAsync(pst, 0, sizeof(PcgState), s));
    const int* solve_stop = stop;
    auto solve = [&](double* x) -> fst_status {
        const int grid = grid_for(R, 256, 2);
        if (use64) {
            double* xw = W.xw.as<double>();
            FST_CUDA(cudaMemcpyAsync(xw, x, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
            FST_TRY(chol_solve_graph<double>(W.solve, static_cast<const double*>(Lp), W.LT.as<double>(),
                                             W.Linv.as<double>(), R, xw,
                                             W.yw.as<double>(), s, solve_stop));
            FST_CUDA(cudaMemcpyAsync(x, xw, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
            return FST_OK;
        }
        float* xw = W.xw.as<float>();
        from_double_kernel<float><<<grid, 256, 0, s>>>(x, xw, R);
        FST_CHECK_LAUNCH();
        FST_TRY(chol_solve_graph<float>(W.solve, static_cast<const float*>(Lp), W.LT.as<float>(), W.Linv.as<float>(),
                                        R, xw,
                                        W.yw.as<float>(), s, solve_stop));
        to_double_kernel<float><<<grid, 256, 0, s>>>(xw, x, R);
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    // the one-launch triangular solves report expired waits in their error word
    if (W.solve.sync.ptr) FST_CUDA(cudaMemsetAsync(W.solve.sync.ptr, 0, sizeof(int), s));
    // alpha_0 = G^-1 h
    FST_CUDA(cudaMemcpyAsync(alpha, g, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
    FST_TRY(solve(alpha));
    FST_CUDA(cudaMemcpyAsync(alpha0, alpha, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));

    // 5. refinement: conjugate gradients on the normal equations A^T A alpha = A^T b,
    // preconditioned by the factor L L^T of the working-precision G.  A p and A^T q are
    // applied through the factored Khatri-Rao form with FP64 accumulation, so the limit is
    // the least-squares solution whatever the accuracy of G (which only sets the speed).
    // Stop at tol, or when the step stops shrinking at a level below `floor_ok`.
    const double floor_ok = fp64 ? 1e-10 : 1e-5;
    FST_TRY(W.pcg.ensure(sizeof(double) * (size_t)R * 4));
    double* rr = W.pcg.as<double>();     // residual of the normal equations
    double* zz = rr + R;                 // preconditioned residual
    double* pp = zz + R;                 // search direction
    double* ww = pp + R;                 // A^T A p
    const int vgrid = grid_for(R, 256, 2);
    auto dots = [&](const double* x0, const double* y0, const double* x1, const double* y1, int nd) -> fst_status {
        dots_kernel<<<1, kDotThreads, 0, s>>>(x0, y0, x1, y1, R, nd, norms);
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    // iterations are launched kCheckEvery at a time; the host reads the state in between, and
    // the kernels of iterations launched after the stop return at once
    constexpr int kCheckEvery = 2;
    PcgState hs;
    memset(&hs, 0, sizeof hs);
    double last = 0.0;
    int steps = 0;
    bool converged = max_refine <= 0;
    if (max_refine > 0) {
        FST_TRY(launch_residual<T>(M, Uc, bvec, alpha, m, rv, s));         // b - A alpha
        FST_TRY(launch_atr<T>(M, Uc, rv, m, rr, s));                       // r = A^T (b - A alpha)
        FST_CUDA(cudaMemcpyAsync(zz, rr, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
        FST_TRY(solve(zz));
        FST_CUDA(cudaMemcpyAsync(pp, zz, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
        FST_TRY(dots(rr, zz, alpha, alpha, 2));
        pcg_init_kernel<<<1, 1, 0, s>>>(norms, pst);
        FST_CHECK_LAUNCH();
        for (int it = 0; it < max_refine; ++it) {
            FST_TRY(launch_residual<T>(M, Uc, nullptr, pp, m, rv, s, 1.0, stop));   // q = A p
            FST_TRY(launch_atr<T>(M, Uc, rv, m, ww, s, stop));                      // w = A^T q
            FST_TRY(dots(pp, ww, pp, pp, 2));
            pcg_step_length_kernel<<<1, 1, 0, s>>>(norms, pst);
            FST_CHECK_LAUNCH();
            pcg_axpy_kernel<<<vgrid, 256, 0, s>>>(alpha, pp, pst, 0, R);             // alpha += ak p
            FST_CHECK_LAUNCH();
            pcg_axpy_kernel<<<vgrid, 256, 0, s>>>(rr, ww, pst, 1, R);                // r -= ak w
            FST_CHECK_LAUNCH();
            FST_CUDA(cudaMemcpyAsync(zz, rr, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
            FST_TRY(solve(zz));
            FST_TRY(dots(rr, zz, alpha, alpha, 2));
            pcg_step_end_kernel<<<1, 1, 0, s>>>(norms, pst, tol, floor_ok);
            FST_CHECK_LAUNCH();
            pcg_axpy_kernel<<<vgrid, 256, 0, s>>>(pp, zz, pst, 2, R);                // p = z + beta p
            FST_CHECK_LAUNCH();
            if ((it + 1) % kCheckEvery == 0 || it + 1 == max_refine) {
                FST_CUDA(cudaMemcpyAsync(&hs, pst, sizeof hs, cudaMemcpyDeviceToHost, s));
                FST_CUDA(cudaStreamSynchronize(s));
                if (hs.stop) break;
            }
        }
        steps = hs.steps;
        last = hs.last;
        converged = hs.stop == 1;
        if (!converged && isfinite(last) && last <= floor_ok) converged = true;
    }
    r.ms_refine = tm.stop();
    {
        int serr = 0;
        FST_CUDA(cudaMemcpyAsync(&serr, W.solve.sync.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        if (serr) {
            set_error("triangular solve: a bounded device wait expired");
            if (rep) *rep = r;
            return FST_ETIMEOUT;
        }
    }
    r.refine_steps = steps;
    r.last_rel_update = last;
    if (!converged && max_refine > 0) {
        if (!use64 && !fp64 && !force64) {
            // the working-precision factor is too weak a preconditioner: redo in FP64
            fst_refit_opts o = opts ? *opts : fst_refit_opts{32, 0.0, 0};
            o.fp64_cholesky = 1;
            fst_refit_report r2;
            fst_status st = refit_impl<T>(M, xyz, u, Q, idx, m, seed, prec, &o, &r2, s);
            r2.fallback_fp64 = 1;
            r2.ms_sample += r.ms_sample;
            if (rep) *rep = r2;
            return st;
        }
        set_error("refinement did not converge (last relative update %.3e)", last);
        if (rep) *rep = r;
        return FST_ENOTCONV;
    }
    // first_rel_change and the new core
    std::vector<double> ha(R), h0(R);
    FST_CUDA(cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(h0.data(), alpha0, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    double dn = 0, an = 0;
    for (int i = 0; i < R; ++i) {
        dn += (ha[i] - h0[i]) * (ha[i] - h0[i]);
        an += ha[i] * ha[i];
    }
    r.first_rel_change = an > 0 ? sqrt(dn / an) : 0.0;
    for (int i = 0; i < R; ++i)
        if (!isfinite(ha[i])) {
            set_error("refit produced a non-finite core");
            if (rep) *rep = r;
            return FST_ENOTSPD;
        }
    M->alpha = ha;
    FST_TRY(model_upload_core(M));
    if (rep) *rep = r;
    return FST_OK;
}

template <typename T>
static fst_status refit_entry(fst_model* M, const T* xyz, const T* u, int64_t Q, const int64_t* idx, int64_t m,
                              uint64_t seed, fst_prec prec, const fst_refit_opts* opts, fst_refit_report* rep,
                              cudaStream_t s) {
    FST_REQUIRE(M != nullptr, "model is NULL");
    FST_REQUIRE(Q > 0 && m > 0, "Q and m must be positive");
    FST_REQUIRE(xyz && u, "xyz or u is NULL");
    if (m > Q) m = Q;
    FST_REQUIRE(m <= (int64_t)1 << 31, "m too large");
    if (m < (int64_t)M->R()) {
        set_error("m = %lld sampled rows < R = %d unknowns", (long long)m, M->R());
        return FST_ERANK;
    }
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == M->device, "model lives on device %d, current device is %d", M->device, dev);
    FST_REQUIRE(pointer_device(xyz) == dev && pointer_device(u) == dev, "xyz and u must be device memory");
    FST_REQUIRE(!idx || pointer_device(idx) == dev, "idx must be device memory");
    std::lock_guard<std::recursive_mutex> lk(M->mu);
    return refit_impl<T>(M, xyz, u, Q, idx, m, seed, prec, opts, rep, s);
}

// Scratch of grouped refits on one device: the factorisation schedule and the job tables.
constexpr int kGroupStreams = 8;
struct GroupScratch {
    std::mutex mu;
    DevBuf sched, tab, states;
    cudaStream_t side[kGroupStreams] = {};
    cudaEvent_t ev[kGroupStreams + 1] = {};
};
GroupScratch g_group[64];

static int rank_class(int r3) { return r3 <= 8 ? 0 : r3 <= 16 ? 1 : r3 <= 24 ? 2 : 3; }

using FailFn = std::function<void(int, fst_status)>;
static fst_status refit_group_shared(const std::vector<fst_refit_item>& items, const std::vector<int>& act,
                                     int max_refine, double tol, double floor_ok, GroupScratch& GS,
                                     std::vector<fst_refit_report>& reps, std::vector<char>& alone,
                                     const FailFn& fail, bool& expired, cudaStream_t s);

// Several refits with their factorisations and conjugate gradients in shared launches.
// Steps 1-3 (rows, factor values, A^T b, the Gram in `prec`) run per item; the FP32
// factorisations run as one schedule (cholesky_lower_group); the conjugate gradients of all
// items advance together, one launch per step for every item (per rank class where the kernel
// is specialised on r3).  An item whose factorisation fails, or whose iteration does not
// converge, is then redone alone by refit_impl (with its fallbacks), so every result equals
// that of fst_refit on the item.  The caller holds every model's lock.
static fst_status refit_group_impl(const std::vector<fst_refit_item>& items, fst_prec prec,
                                   const fst_refit_opts* opts, std::vector<fst_refit_report>& reps,
                                   std::vector<fst_status>& status, std::vector<std::string>& errors,
                                   cudaStream_t s) {
    const int n = (int)items.size();
    const int max_refine = opts ? opts->max_refine : 32;
    const double tol = (opts && opts->refine_tol > 0) ? opts->refine_tol : 1e-8;
    const double floor_ok = 1e-5;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    GroupScratch& GS = g_group[dev & 63];
    std::lock_guard<std::mutex> glk(GS.mu);
    std::vector<char> alone(n, 0);   // redo with refit_impl
    const FailFn fail = [&](int i, fst_status st) {
        status[i] = st;
        errors[i] = fst_last_error();
    };
    // 1-3 per item, spread over side streams that start after the caller's stream
    if (!GS.side[0]) {
        for (int k = 0; k < kGroupStreams; ++k) {
            FST_CUDA(cudaStreamCreateWithFlags(&GS.side[k], cudaStreamNonBlocking));
            FST_CUDA(cudaEventCreateWithFlags(&GS.ev[k], cudaEventDisableTiming));
        }
        FST_CUDA(cudaEventCreateWithFlags(&GS.ev[kGroupStreams], cudaEventDisableTiming));
    }
    EventTimer t1(s);
    FST_CUDA(cudaEventRecord(GS.ev[kGroupStreams], s));
    for (int k = 0; k < kGroupStreams; ++k) FST_CUDA(cudaStreamWaitEvent(GS.side[k], GS.ev[kGroupStreams], 0));
    std::vector<int> act;
    int nside = 0;
    for (int i = 0; i < n; ++i) {
        if (status[i] != FST_OK) continue;
        if (opts && opts->fp64_cholesky) {
            alone[i] = 1;
            continue;
        }
        fst_model* M = items[i].model;
        RefitScratch& W = M->rs;
        const int R = M->R();
        const int64_t m = items[i].m;
        fst_refit_report& r = reps[i];
        memset(&r, 0, sizeof r);
        r.m = m;
        cudaStream_t ss = GS.side[nside++ % kGroupStreams];
        auto step = [&]() -> fst_status {
            const cudaStream_t s = ss;
            FST_TRY(W.idx.ensure(sizeof(int64_t) * (size_t)m));
            FST_TRY(sample_rows(items[i].seed, items[i].Q, m, W.idx.as<int64_t>(), s));
            float* U[3];
            for (int k = 0; k < 3; ++k) {
                FST_TRY(W.U[k].ensure(sizeof(float) * (size_t)m * M->r[k]));
                U[k] = W.U[k].as<float>();
            }
            FST_TRY(W.b.ensure(sizeof(float) * (size_t)m));
            FST_TRY(launch_factors<float>(M, items[i].xyz, items[i].Q, W.idx.as<int64_t>(), m, items[i].u, U,
                                          W.b.as<float>(), s));
            FST_TRY(W.res.ensure(sizeof(double) * (size_t)m));
            FST_TRY(W.g.ensure(sizeof(double) * (size_t)R));
            FST_TRY(W.alpha.ensure(sizeof(double) * (size_t)R));
            FST_TRY(W.z.ensure(sizeof(double) * (size_t)R));
            FST_TRY(W.norms.ensure(sizeof(double) * 2));
            FST_TRY(W.flag.ensure(4 * sizeof(int)));
            const float* const Uc[3] = {U[0], U[1], U[2]};
            to_double_kernel<float><<<grid_for(m, 256), 256, 0, s>>>(W.b.as<float>(), W.res.as<double>(), m);
            FST_CHECK_LAUNCH();
            FST_TRY(launch_atr<float>(M, Uc, W.res.as<double>(), m, W.g.as<double>(), s));
            FST_CUDA(cudaMemsetAsync(W.flag.as<int>(), 0, 2 * sizeof(int), s));
            FST_TRY(W.G.ensure(sizeof(float) * (size_t)R * R));
            if (prec == FST_FP32)
                FST_TRY(launch_gram_simt<float>(M, Uc, m, W.G.as<float>(), s));
            else
                FST_TRY(gram_tensor(M, Uc, m, W.G.as<float>(), prec, s));
            return FST_OK;
        };
        const fst_status st = step();
        if (st != FST_OK) fail(i, st);
        else act.push_back(i);
    }
    for (int k = 0; k < kGroupStreams; ++k) {
        FST_CUDA(cudaEventRecord(GS.ev[k], GS.side[k]));
        FST_CUDA(cudaStreamWaitEvent(s, GS.ev[k], 0));
    }
    const double ms1 = t1.stop();
    for (int i : act) reps[i].ms_gram = ms1;   // rows, factor values and Grams of the whole group
    // 4-6 (a device wait that expired fails every item still to be done)
    bool expired = false;
    if (!act.empty())
        FST_TRY(refit_group_shared(items, act, max_refine, tol, floor_ok, GS, reps, alone, fail, expired, s));
    // 7. items redone alone (failed factorisation, no convergence, or FP64 asked for)
    for (int i = 0; i < n; ++i) {
        if (!alone[i] || status[i] != FST_OK) continue;
        if (expired) {
            status[i] = FST_ETIMEOUT;
            errors[i] = "a bounded device wait of the group expired";
            continue;
        }
        const fst_status st = refit_impl<float>(items[i].model, items[i].xyz, items[i].u, items[i].Q, nullptr,
                                                items[i].m, items[i].seed, prec, opts, &reps[i], s);
        if (st != FST_OK) fail(i, st);
    }
    return FST_OK;
}

// Steps 4-6 of a grouped refit for the items `act` (their Grams formed): the shared
// factorisation, then the shared conjugate gradients of the items whose factor exists, then
// their new cores.  Items to redo alone are marked in `alone`.
static fst_status refit_group_shared(const std::vector<fst_refit_item>& items, const std::vector<int>& act,
                                     int max_refine, double tol, double floor_ok, GroupScratch& GS,
                                     std::vector<fst_refit_report>& reps, std::vector<char>& alone,
                                     const FailFn& fail, bool& expired, cudaStream_t s) {
    const int n = (int)items.size();
    // 4. the factorisations, one schedule
    EventTimer tg(s);
    FST_TRY(GS.states.ensure(sizeof(int) * 4 + sizeof(PcgState) * (size_t)n));
    int* gsync = GS.states.as<int>();   // [0] factorisation waits, [2] solve error, [3] solve ticket
    PcgState* gst = reinterpret_cast<PcgState*>(gsync + 4);
    FST_CUDA(cudaMemsetAsync(gsync, 0, 4 * sizeof(int), s));
    {
        std::vector<CholItem> ci;
        for (int i : act) {
            RefitScratch& W = items[i].model->rs;
            ci.push_back(CholItem{W.G.as<float>(), items[i].model->R(), W.flag.as<int>(), &W.chol_ws});
        }
        FST_TRY(cholesky_lower_group(ci, GS.sched, gsync, s));
    }
    for (int i : act) {
        RefitScratch& W = items[i].model->rs;
        const int R = items[i].model->R();
        FST_TRY(W.Linv.ensure(3 * sizeof(float) * (size_t)((R + 63) / 64) * 64 * 64));
        FST_TRY(chol_invert_diag<float>(W.G.as<float>(), R, W.Linv.as<float>(), s));
        FST_TRY(W.LT.ensure(sizeof(float) * (size_t)R * R));
        FST_TRY(chol_transpose<float>(W.G.as<float>(), R, W.LT.as<float>(), s));
    }
    std::vector<int> hflag(act.size(), 0);
    for (size_t a = 0; a < act.size(); ++a)
        FST_CUDA(cudaMemcpyAsync(&hflag[a], items[act[a]].model->rs.flag.as<int>(), sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
    int hg = 0;
    FST_CUDA(cudaMemcpyAsync(&hg, gsync, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    const double ms_chol = tg.stop();
    if (hg) {
        set_error("Cholesky: a bounded device wait expired (code %d)", hg);
        for (int i : act) fail(i, FST_ETIMEOUT);
        expired = true;
        return FST_OK;
    }
    std::vector<int> pc;   // items going on to the conjugate gradients
    for (size_t a = 0; a < act.size(); ++a) {
        reps[act[a]].ms_cholesky = ms_chol;
        if (hflag[a]) alone[act[a]] = 1;
        else pc.push_back(act[a]);
    }

    // 5. the conjugate gradients of every remaining item, in shared launches
    if (!pc.empty()) {
        std::sort(pc.begin(), pc.end(), [&](int a, int b) {
            const int ca = rank_class(items[a].model->r[2]), cb = rank_class(items[b].model->r[2]);
            return ca != cb ? ca < cb : a < b;
        });
        const int np = (int)pc.size();
        std::vector<PcgJob> jobs(np);
        std::vector<SolveJob> sj(np);
        std::vector<int> Rs(np);
        int cls_off[5] = {0, 0, 0, 0, 0};
        long long rnext[4] = {0, 0, 0, 0}, anext[4] = {0, 0, 0, 0};
        int maxR = 0;
        for (int q = 0; q < np; ++q) {
            fst_model* M = items[pc[q]].model;
            RefitScratch& W = M->rs;
            const int R = M->R();
            const int64_t m = items[pc[q]].m;
            FST_TRY(W.xw.ensure(sizeof(double) * (size_t)R));
            FST_TRY(W.yw.ensure(sizeof(double) * (size_t)R));
            FST_TRY(W.pcg_state.ensure(sizeof(PcgState)));
            FST_TRY(W.pcg.ensure(sizeof(double) * (size_t)R * 4));
            FST_CUDA(cudaMemsetAsync(W.pcg_state.ptr, 0, sizeof(PcgState), s));
            // the single refit's A^T row partition
            int64_t nparts = 2LL * sm_count();
            const int64_t rpb = ((m + nparts - 1) / nparts + 31) / 32 * 32;
            nparts = (m + rpb - 1) / rpb;
            FST_TRY(W.atr_part.ensure(sizeof(double) * (size_t)nparts * R));
            PcgJob& j = jobs[q];
            j.U1 = W.U[0].as<float>();
            j.U2 = W.U[1].as<float>();
            j.U3 = W.U[2].as<float>();
            j.b = W.b.as<float>();
            j.m = m;
            j.r1 = M->r[0];
            j.r2 = M->r[1];
            j.r3 = M->r[2];
            j.R = R;
            double* pv = W.pcg.as<double>();
            j.v[vRV] = W.res.as<double>();
            j.v[vG] = W.g.as<double>();
            j.v[vAlpha] = W.alpha.as<double>();
            j.v[vAlpha0] = W.z.as<double>();
            j.v[vRR] = pv;
            j.v[vZZ] = pv + R;
            j.v[vPP] = pv + 2 * R;
            j.v[vWW] = pv + 3 * R;
            j.norms = W.norms.as<double>();
            j.part = W.atr_part.as<double>();
            j.st = W.pcg_state.as<PcgState>();
            j.xw = W.xw.as<float>();
            j.nparts = (int)nparts;
            j.rows_per_block = rpb;
            // one A^T part a block (fewer, longer blocks serialise the small items' parts)
            j.parts_per_block = 1;
            const int c = rank_class(j.r3);
            ++cls_off[c + 1];
            j.rfirst = rnext[c];
            rnext[c] += (m + 255) / 256;
            j.afirst = anext[c];
            anext[c] += (nparts + j.parts_per_block - 1) / j.parts_per_block;
            sj[q] = SolveJob{W.G.as<float>(), W.LT.as<float>(), W.Linv.as<float>(), W.xw.as<float>(),
                             W.yw.as<float>(), &j.st->stop, R, (R + 63) / 64};
            Rs[q] = R;
            maxR = std::max(maxR, R);
        }
        for (int c = 0; c < 4; ++c) cls_off[c + 1] += cls_off[c];
        const std::vector<int> tmap = solve_tickets(Rs);
        const size_t jb = (sizeof(PcgJob) * np + 255) / 256 * 256, sb = (sizeof(SolveJob) * np + 255) / 256 * 256;
        FST_TRY(GS.tab.ensure(jb + sb + sizeof(int) * tmap.size()));
        PcgJob* dj = GS.tab.as<PcgJob>();
        SolveJob* ds = reinterpret_cast<SolveJob*>(GS.tab.as<unsigned char>() + jb);
        int* dt = reinterpret_cast<int*>(GS.tab.as<unsigned char>() + jb + sb);
        FST_CUDA(cudaMemcpyAsync(dj, jobs.data(), sizeof(PcgJob) * np, cudaMemcpyHostToDevice, s));
        FST_CUDA(cudaMemcpyAsync(ds, sj.data(), sizeof(SolveJob) * np, cudaMemcpyHostToDevice, s));
        FST_CUDA(cudaMemcpyAsync(dt, tmap.data(), sizeof(int) * tmap.size(), cudaMemcpyHostToDevice, s));
        size_t res_smem[4] = {0, 0, 0, 0};
        for (int q = 0; q < np; ++q) {
            const int c = rank_class(jobs[q].r3);
            res_smem[c] = std::max(res_smem[c], (size_t)jobs[q].r1 * jobs[q].r2 * ((c + 1) * 8) * sizeof(float) * 2);
        }
        const dim3 vg((unsigned)std::min((maxR + 255) / 256, 64), (unsigned)np);
        auto residual = [&](int src, int use_b, double scale, int gated) -> fst_status {
            for (int c = 0; c < 4; ++c) {
                const int cn = cls_off[c + 1] - cls_off[c];
                if (!cn) continue;
                const PcgJob* jc = dj + cls_off[c];
#define FST_RESG(V)                                                                                     \
    {                                                                                                   \
        auto kern = residual_group_kernel<V>;                                                           \
        FST_TRY(allow_smem(kern, res_smem[c]));                                                         \
        kern<<<(unsigned)rnext[c], 256, res_smem[c], s>>>(jc, cn, src, use_b, scale, gated);            \
    }
                if (c == 0) FST_RESG(8) else if (c == 1) FST_RESG(16) else if (c == 2) FST_RESG(24) else FST_RESG(32)
#undef FST_RESG
                FST_CHECK_LAUNCH();
            }
            return FST_OK;
        };
        auto atr = [&](int dst, int gated) -> fst_status {
            for (int c = 0; c < 4; ++c) {
                const int cn = cls_off[c + 1] - cls_off[c];
                if (!cn) continue;
                const PcgJob* jc = dj + cls_off[c];
                const unsigned g = (unsigned)anext[c];
                if (c == 0) atr_group_kernel<8, 3><<<g, 256, 0, s>>>(jc, cn, gated);
                else if (c == 1) atr_group_kernel<16, 3><<<g, 256, 0, s>>>(jc, cn, gated);
                else if (c == 2) atr_group_kernel<24, 3><<<g, 256, 0, s>>>(jc, cn, gated);
                else atr_group_kernel<32, 2><<<g, 256, 0, s>>>(jc, cn, gated);
                FST_CHECK_LAUNCH();
            }
            sum_partials_group_kernel<<<vg, 256, 0, s>>>(dj, dst, gated);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        auto copy = [&](int dst, int src) -> fst_status {
            pcg_copy_group_kernel<<<vg, 256, 0, s>>>(dj, dst, src);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        auto solve = [&](int vec) -> fst_status {
            pcg_convert_group_kernel<<<vg, 256, 0, s>>>(dj, vec, 0);
            FST_CHECK_LAUNCH();
            FST_TRY(chol_solve_group<float>(ds, np, maxR, dt, (int)tmap.size(), gsync + 2, s));
            pcg_convert_group_kernel<<<vg, 256, 0, s>>>(dj, vec, 1);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        auto dots = [&](int x0, int y0, int x1, int y1) -> fst_status {
            dots_group_kernel<<<np, kDotThreads, 0, s>>>(dj, x0, y0, x1, y1);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        auto scalar = [&](int kind) -> fst_status {
            pcg_scalar_group_kernel<<<(np + 127) / 128, 128, 0, s>>>(dj, np, kind, tol, floor_ok);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        auto axpy = [&](int which) -> fst_status {
            pcg_axpy_group_kernel<<<vg, 256, 0, s>>>(dj, which);
            FST_CHECK_LAUNCH();
            return FST_OK;
        };
        EventTimer tr(s);
        // alpha_0 = G^-1 h
        FST_TRY(copy(vAlpha, vG));
        FST_TRY(solve(vAlpha));
        FST_TRY(copy(vAlpha0, vAlpha));
        std::vector<PcgState> hs(np);
        memset(hs.data(), 0, sizeof(PcgState) * np);
        if (max_refine > 0) {
            FST_TRY(residual(vAlpha, 1, -1.0, 0));        // b - A alpha
            FST_TRY(atr(vRR, 0));                         // r = A^T (b - A alpha)
            FST_TRY(copy(vZZ, vRR));
            FST_TRY(solve(vZZ));
            FST_TRY(copy(vPP, vZZ));
            FST_TRY(dots(vRR, vZZ, vAlpha, vAlpha));
            FST_TRY(scalar(0));
            constexpr int kCheckEvery = 2;
            for (int it = 0; it < max_refine; ++it) {
                FST_TRY(residual(vPP, 0, 1.0, 1));        // q = A p
                FST_TRY(atr(vWW, 1));                     // w = A^T q
                FST_TRY(dots(vPP, vWW, vPP, vPP));
                FST_TRY(scalar(1));
                FST_TRY(axpy(0));                         // alpha += ak p
                FST_TRY(axpy(1));                         // r -= ak w
                FST_TRY(copy(vZZ, vRR));
                FST_TRY(solve(vZZ));
                FST_TRY(dots(vRR, vZZ, vAlpha, vAlpha));
                FST_TRY(scalar(2));
                FST_TRY(axpy(2));                         // p = z + beta p
                if ((it + 1) % kCheckEvery == 0 || it + 1 == max_refine) {
                    pcg_gather_states_kernel<<<(np + 127) / 128, 128, 0, s>>>(dj, np, gst);
                    FST_CHECK_LAUNCH();
                    FST_CUDA(cudaMemcpyAsync(hs.data(), gst, sizeof(PcgState) * np, cudaMemcpyDeviceToHost, s));
                    FST_CUDA(cudaStreamSynchronize(s));
                    bool all = true;
                    for (const PcgState& x : hs) all = all && x.stop != 0;
                    if (all) break;
                }
            }
        }
        int serr = 0;
        FST_CUDA(cudaMemcpyAsync(&serr, gsync + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        const double ms_ref = tr.stop();
        if (serr) {
            set_error("triangular solve: a bounded device wait expired");
            for (int i : pc) fail(i, FST_ETIMEOUT);
            expired = true;
            return FST_OK;
        }
        // 6. the new cores
        for (int q = 0; q < np; ++q) {
            const int i = pc[q];
            fst_model* M = items[i].model;
            fst_refit_report& r = reps[i];
            r.ms_refine = ms_ref;
            const int R = M->R();
            bool converged = max_refine <= 0;
            if (max_refine > 0) {
                r.refine_steps = hs[q].steps;
                r.last_rel_update = hs[q].last;
                converged = hs[q].stop == 1 || (isfinite(hs[q].last) && hs[q].last <= floor_ok);
            }
            if (!converged) {
                alone[i] = 1;
                continue;
            }
            std::vector<double> ha(R), h0(R);
            FST_CUDA(cudaMemcpyAsync(ha.data(), jobs[q].v[vAlpha], sizeof(double) * R, cudaMemcpyDeviceToHost, s));
            FST_CUDA(cudaMemcpyAsync(h0.data(), jobs[q].v[vAlpha0], sizeof(double) * R, cudaMemcpyDeviceToHost, s));
            FST_CUDA(cudaStreamSynchronize(s));
            double dn = 0, an = 0;
            bool finite = true;
            for (int e = 0; e < R; ++e) {
                dn += (ha[e] - h0[e]) * (ha[e] - h0[e]);
                an += ha[e] * ha[e];
                finite = finite && isfinite(ha[e]);
            }
            r.first_rel_change = an > 0 ? sqrt(dn / an) : 0.0;
            if (!finite) {
                set_error("refit produced a non-finite core");
                fail(i, FST_ENOTSPD);
                continue;
            }
            M->alpha = ha;
            const fst_status st = model_upload_core(M);
            if (st != FST_OK) fail(i, st);
        }
    }
    return FST_OK;
}

}  // namespace fst

using namespace fst;

extern "C" fst_status fst_refit(fst_model* model, const float* xyz, const float* u, int64_t Q, const int64_t* idx,
                                int64_t m, uint64_t seed, fst_prec prec, const fst_refit_opts* opts,
                                fst_refit_report* report, fst_stream stream) {
    FST_REQUIRE(prec == FST_FP32 || prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_refit takes FP32/TF32/BF16/BF16X3; use fst_refit_f64 for FP64");
    return refit_entry<float>(model, xyz, u, Q, idx, m, seed, prec, opts, report, (cudaStream_t)stream);
}

// Many refits at once: `streams` worker threads, each with its own non-blocking stream, take
// the items in order and refit them, so the launches of different instances overlap on the
// device.  Every per-model scratch is private to its model; the per-device scratch the refit
// shares (the sampler's, the packed Gram operand) is ordered across streams on the device.
extern "C" fst_status fst_refit_batched(const fst_refit_item* items, int32_t count, fst_prec prec,
                                        const fst_refit_opts* opts, int32_t streams, fst_refit_report* reports) {
    FST_REQUIRE(count >= 0 && (count == 0 || items != nullptr), "items is NULL");
    FST_REQUIRE(prec == FST_FP32 || prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_refit_batched takes FP32/TF32/BF16/BF16X3");
    FST_REQUIRE(streams >= 1 && streams <= 64, "streams must be in 1..64");
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j)
            FST_REQUIRE(items[i].model != items[j].model, "items %d and %d refit the same model", j, i);
    if (count == 0) return FST_OK;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    const int nw = streams < count ? streams : count;
    std::atomic<int> next{0};
    std::vector<fst_status> status(count, FST_OK);
    std::vector<std::string> errors(count);
    std::vector<std::thread> workers;
    workers.reserve(nw);
    for (int w = 0; w < nw; ++w) {
        workers.emplace_back([&, w]() {
            (void)w;
            if (cudaSetDevice(dev) != cudaSuccess) {
                for (int i; (i = next.fetch_add(1)) < count;) status[i] = FST_ECUDA;
                return;
            }
            cudaStream_t s = nullptr;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                for (int i; (i = next.fetch_add(1)) < count;) status[i] = FST_ECUDA;
                return;
            }
            for (int i; (i = next.fetch_add(1)) < count;) {
                const fst_refit_item& it = items[i];
                status[i] = fst_refit(it.model, it.xyz, it.u, it.Q, nullptr, it.m, it.seed, prec, opts,
                                      reports ? &reports[i] : nullptr, (fst_stream)s);
                if (status[i] != FST_OK) errors[i] = fst_last_error();
            }
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        });
    }
    for (auto& t : workers) t.join();
    for (int i = 0; i < count; ++i)
        if (status[i] != FST_OK) {
            set_error("item %d: %s", i, errors[i].c_str());
            return status[i];
        }
    return FST_OK;
}

// Many refits with shared launches (see refit_group_impl): every item is checked as fst_refit
// checks it, the models are locked in address order, and the first failed item's status is
// returned after all items have run.
extern "C" fst_status fst_refit_grouped(const fst_refit_item* items, int32_t count, fst_prec prec,
                                        const fst_refit_opts* opts, fst_refit_report* reports, fst_stream stream) {
    FST_REQUIRE(count >= 0 && (count == 0 || items != nullptr), "items is NULL");
    FST_REQUIRE(prec == FST_FP32 || prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_refit_grouped takes FP32/TF32/BF16/BF16X3");
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j)
            FST_REQUIRE(items[i].model != items[j].model, "items %d and %d refit the same model", j, i);
    if (count == 0) return FST_OK;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    std::vector<fst_refit_item> it(items, items + count);
    std::vector<fst_status> status(count, FST_OK);
    std::vector<std::string> errors(count);
    std::vector<fst_refit_report> reps(count);
    for (int i = 0; i < count; ++i) {
        fst_refit_item& x = it[i];
        memset(&reps[i], 0, sizeof(fst_refit_report));
        auto bad = [&](fst_status st, const char* msg) {
            status[i] = st;
            errors[i] = msg;
        };
        if (!x.model) bad(FST_EINVAL, "model is NULL");
        else if (x.Q <= 0 || x.m <= 0) bad(FST_EINVAL, "Q and m must be positive");
        else if (!x.xyz || !x.u) bad(FST_EINVAL, "xyz or u is NULL");
        else if (x.model->device != dev) bad(FST_EINVAL, "model lives on another device");
        else if (pointer_device(x.xyz) != dev || pointer_device(x.u) != dev) bad(FST_EINVAL, "xyz and u must be device memory");
        else {
            if (x.m > x.Q) x.m = x.Q;
            if (x.m > ((int64_t)1 << 31)) bad(FST_EINVAL, "m too large");
            else if (x.m < (int64_t)x.model->R()) bad(FST_ERANK, "fewer sampled rows than unknowns (m < R)");
        }
    }
    std::vector<fst_model*> order;
    for (const fst_refit_item& x : it)
        if (x.model) order.push_back(x.model);
    std::sort(order.begin(), order.end());
    std::vector<std::unique_lock<std::recursive_mutex>> locks;
    for (fst_model* M : order) locks.emplace_back(M->mu);
    FST_TRY(refit_group_impl(it, prec, opts, reps, status, errors, (cudaStream_t)stream));
    if (reports)
        for (int i = 0; i < count; ++i) reports[i] = reps[i];
    for (int i = 0; i < count; ++i)
        if (status[i] != FST_OK) {
            set_error("item %d: %s", i, errors[i].c_str());
            return status[i];
        }
    return FST_OK;
}

extern "C" fst_status fst_refit_f64(fst_model* model, const double* xyz, const double* u, int64_t Q,
                                    const int64_t* idx, int64_t m, uint64_t seed, const fst_refit_opts* opts,
                                    fst_refit_report* report, fst_stream stream) {
    return refit_entry<double>(model, xyz, u, Q, idx, m, seed, FST_FP64, opts, report, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ Algorithm 2 with mixing
namespace fst {

// Rows of the mixed system before the transform: WB[q] = D_q [w1 (x) w2 (x) w3 (y_q), u_q] for
// q < Q (column (i r2 + j) r3 + k, then u), zero rows up to N; D_q = -1 when the top bit of
// the row's key under the sign seed is set.
__global__ void mix_rows_kernel(const double* __restrict__ U1, const double* __restrict__ U2,
                                const double* __restrict__ U3, const double* __restrict__ b, int64_t Q, int64_t N,
                                int r1, int r2, int r3, uint64_t seed, double* __restrict__ WB) {
    const int R = r1 * r2 * r3, C = R + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * C; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / C;
        const int c = (int)(e - q * C);
        double v = 0.0;
        if (q < Q) {
            if (c == R) {
                v = b[q];
            } else {
                const int i = c / (r2 * r3), j = (c / r3) % r2, k = c % r3;
                v = U1[q * r1 + i] * U2[q * r2 + j] * U3[q * r3 + k];
            }
            if (splitmix_key(seed, (uint64_t)q) >> 63) v = -v;
        }
        WB[e] = v;
    }
}

// One stage of the normalised Walsh-Hadamard transform along the rows (stride h):
// (a, b) -> (a + b, a - b) / sqrt(2) for rows i0 = (p / h) 2h + p % h and i0 + h.
__global__ void fwht_stage_kernel(double* __restrict__ WB, int64_t N, int C, int64_t h) {
    const double s = 0.70710678118654752440;
    const int64_t pairs = N / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pairs * C;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / C;
        const int c = (int)(e - p * C);
        const int64_t i0 = (p / h) * 2 * h + p % h, i1 = i0 + h;
        const double a = WB[i0 * C + c], bb = WB[i1 * C + c];
        WB[i0 * C + c] = (a + bb) * s;
        WB[i1 * C + c] = (a - bb) * s;
    }
}

// Lower triangle of E = A^T A over the sampled rows idx of WB (m x C, A = WB[idx]), in 32 x 32
// tiles: E[0:R, 0:R] is G, row R holds h = A_u^T b.
__global__ void __launch_bounds__(256) mixed_gram_kernel(const double* __restrict__ WB, int C,
                                                         const int64_t* __restrict__ idx, int64_t m,
                                                         double* __restrict__ E) {
    __shared__ double a[32][33], bt[32][33];
    int ti = 0;
    {
        const int t = blockIdx.x;
        ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
    }
    const int tj = blockIdx.x - ti * (ti + 1) / 2;
    const int r0 = ti * 32, c0 = tj * 32;
    const int tid = threadIdx.x, tr = tid >> 3, tc = (tid & 7) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t s0 = 0; s0 < m; s0 += 32) {
        for (int e = tid; e < 32 * 32; e += 256) {
            const int rr = e >> 5, cc = e & 31;
            const int64_t sidx = s0 + rr;
            const double* row = sidx < m ? WB + idx[sidx] * (int64_t)C : nullptr;
            a[rr][cc] = row && r0 + cc < C ? row[r0 + cc] : 0.0;
            bt[rr][cc] = row && c0 + cc < C ? row[c0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const double x = a[k][tr];
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[y] = fma(x, bt[k][tc + y], acc[y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int r = r0 + tr, c = c0 + tc + y;
        if (r < C && c < C && c <= r) E[(size_t)r * C + c] = acc[y];
    }
}

// E (C x C lower) -> G (R x R lower) and h
__global__ void split_gram_kernel(const double* __restrict__ E, int R, double* __restrict__ G, double* __restrict__ h) {
    const int C = R + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * R;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / R), c = (int)(e - (int64_t)r * R);
        G[e] = c <= r ? E[(size_t)r * C + c] : 0.0;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) h[c] = E[(size_t)R * C + c];
}

static fst_status refit_mixed_impl(fst_model* M, const double* xyz, const double* u, int64_t Q, int64_t m,
                                   uint64_t seed_signs, uint64_t seed_rows, fst_refit_report* rep, cudaStream_t s) {
    const int R = M->R();
    const int C = R + 1;
    int64_t N = 1;
    while (N < Q) N *= 2;
    RefitScratch& W = M->rs;
    fst_refit_report r;
    memset(&r, 0, sizeof r);
    r.m = m;
    EventTimer tm(s);
    // 1. factor values of every point, the signed Khatri-Rao rows, the transform
    FST_TRY(W.idx.ensure(sizeof(int64_t) * (size_t)Q));
    int64_t* all = W.idx.as<int64_t>();
    FST_TRY(sample_rows(0, Q, Q, all, s));       // m >= Q: every row, in order
    double* U[3];
    for (int k = 0; k < 3; ++k) {
        FST_TRY(W.U[k].ensure(sizeof(double) * (size_t)Q * M->r[k]));
        U[k] = W.U[k].as<double>();
    }
    FST_TRY(W.b.ensure(sizeof(double) * (size_t)Q));
    FST_TRY(launch_factors<double>(M, xyz, Q, all, Q, u, U, W.b.as<double>(), s));
    FST_TRY(W.mix.ensure(sizeof(double) * (size_t)N * C));
    double* WB = W.mix.as<double>();
    {
        int64_t total = N * C;
        int grid = (int)std::min<int64_t>((total + 255) / 256, 16LL * sm_count());
        mix_rows_kernel<<<grid, 256, 0, s>>>(U[0], U[1], U[2], W.b.as<double>(), Q, N, M->r[0], M->r[1], M->r[2],
                                             seed_signs, WB);
        FST_CHECK_LAUNCH();
        total = N / 2 * C;
        grid = (int)std::min<int64_t>((total + 255) / 256, 16LL * sm_count());
        for (int64_t h = 1; h < N; h *= 2) {
            fwht_stage_kernel<<<grid < 1 ? 1 : grid, 256, 0, s>>>(WB, N, C, h);
            FST_CHECK_LAUNCH();
        }
    }
    r.ms_sample = tm.stop();
    // 2. the sampled mixed rows and their normal equations
    FST_TRY(W.res.ensure(sizeof(int64_t) * (size_t)m));
    int64_t* idx = reinterpret_cast<int64_t*>(W.res.ptr);
    FST_TRY(sample_rows(seed_rows, N, m, idx, s));
    FST_TRY(W.G64.ensure(sizeof(double) * ((size_t)C * C + (size_t)R * R + R)));
    double* E = W.G64.as<double>();
    double* G = E + (size_t)C * C;
    double* h = G + (size_t)R * R;
    {
        const int nt = (C + 31) / 32;
        mixed_gram_kernel<<<nt * (nt + 1) / 2, 256, 0, s>>>(WB, C, idx, m, E);
        FST_CHECK_LAUNCH();
        split_gram_kernel<<<grid_for((int64_t)R * R, 256), 256, 0, s>>>(E, R, G, h);
        FST_CHECK_LAUNCH();
    }
    r.ms_gram = tm.stop();
    // 3. FP64 Cholesky and the two triangular solves: alpha = G^-1 h
    FST_TRY(W.flag.ensure(4 * sizeof(int)));
    int* flag = W.flag.as<int>();
    FST_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), s));
    FST_TRY(cholesky_lower<double>(G, R, flag, W.chol_ws, s));
    int hflag[2] = {0, 0};
    FST_CUDA(cudaMemcpyAsync(hflag, flag, sizeof hflag, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    r.ms_cholesky = tm.stop();
    if (hflag[1]) {
        set_error("Cholesky: a bounded device wait expired (code %d)", hflag[1]);
        if (rep) *rep = r;
        return FST_ETIMEOUT;
    }
    if (hflag[0]) {
        set_error("normal matrix of the mixed rows is not positive definite in FP64 (rank-deficient sample)");
        if (rep) *rep = r;
        return FST_ENOTSPD;
    }
    FST_TRY(W.Linv.ensure(3 * sizeof(double) * (size_t)((R + 63) / 64) * 64 * 64));
    FST_TRY(chol_invert_diag<double>(G, R, W.Linv.as<double>(), s));
    FST_TRY(W.LT.ensure(sizeof(double) * (size_t)R * R));
    FST_TRY(chol_transpose<double>(G, R, W.LT.as<double>(), s));
    FST_TRY(W.yw.ensure(sizeof(double) * (size_t)R));
    FST_TRY(W.solve.sync.ensure(4 * sizeof(int)));
    int* sync = W.solve.sync.as<int>();
    FST_CUDA(cudaMemsetAsync(sync, 0, sizeof(int), s));
    FST_TRY(chol_solve<double>(G, W.LT.as<double>(), W.Linv.as<double>(), R, h, W.yw.as<double>(), sync, s));
    std::vector<double> ha(R);
    int serr = 0;
    FST_CUDA(cudaMemcpyAsync(ha.data(), h, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(&serr, sync, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    r.ms_refine = tm.stop();
    if (serr) {
        set_error("triangular solve: a bounded device wait expired");
        if (rep) *rep = r;
        return FST_ETIMEOUT;
    }
    for (int i = 0; i < R; ++i)
        if (!isfinite(ha[i])) {
            set_error("mixed refit produced a non-finite core");
            if (rep) *rep = r;
            return FST_ENOTSPD;
        }
    M->alpha = ha;
    FST_TRY(model_upload_core(M));
    if (rep) *rep = r;
    return FST_OK;
}

}  // namespace fst

extern "C" fst_status fst_refit_mixed(fst_model* model, const double* xyz, const double* u, int64_t Q, int64_t m,
                                      uint64_t seed_signs, uint64_t seed_rows, fst_refit_report* report,
                                      fst_stream stream) {
    using namespace fst;
    FST_REQUIRE(model != nullptr && xyz && u, "model, xyz or u is NULL");
    FST_REQUIRE(Q > 0 && m > 0, "Q and m must be positive");
    int64_t N = 1;
    while (N < Q) N *= 2;
    FST_REQUIRE(m <= N, "m = %lld exceeds the %lld mixed rows", (long long)m, (long long)N);
    if (m < (int64_t)model->R()) {
        set_error("m = %lld sampled rows < R = %d unknowns", (long long)m, model->R());
        return FST_ERANK;
    }
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == model->device, "model lives on device %d, current device is %d", model->device, dev);
    FST_REQUIRE(pointer_device(xyz) == dev && pointer_device(u) == dev, "xyz and u must be device memory");
    std::lock_guard<std::recursive_mutex> lk(model->mu);
    return refit_mixed_impl(model, xyz, u, Q, m, seed_signs, seed_rows, report, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ normal matrix only
extern "C" fst_status fst_normal_matrix(const fst_model* M, const float* xyz, const float* u, int64_t Q,
                                        const int64_t* idx, int64_t m, fst_prec prec, float* G, double* h,
                                        fst_stream stream) {
    FST_REQUIRE(M != nullptr && xyz && u && idx && G, "model, xyz, u, idx or G is NULL");
    FST_REQUIRE(Q > 0 && m > 0 && m <= Q, "need 0 < m <= Q");
    FST_REQUIRE(prec == FST_FP32 || prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_normal_matrix takes FP32, TF32, BF16 or BF16X3");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == M->device, "model lives on device %d, current device is %d", M->device, dev);
    FST_REQUIRE(pointer_device(xyz) == dev && pointer_device(u) == dev && pointer_device(idx) == dev &&
                    pointer_device(G) == dev && (!h || pointer_device(h) == dev),
                "xyz, u, idx, G and h must be device memory");
    fst_model* MM = const_cast<fst_model*>(M);
    std::lock_guard<std::recursive_mutex> lk(MM->mu);
    cudaStream_t s = (cudaStream_t)stream;
    RefitScratch& W = MM->rs;
    float* U[3];
    for (int k = 0; k < 3; ++k) {
        FST_TRY(W.U[k].ensure(sizeof(float) * (size_t)m * M->r[k]));
        U[k] = W.U[k].as<float>();
    }
    FST_TRY(W.b.ensure(sizeof(float) * (size_t)m));
    FST_TRY(launch_factors<float>(M, xyz, Q, idx, m, u, U, W.b.as<float>(), s));
    const float* const Uc[3] = {U[0], U[1], U[2]};
    if (prec == FST_FP32) {
        FST_TRY(launch_gram_simt<float>(M, Uc, m, G, s));
    } else {
        FST_TRY(gram_tensor(M, Uc, m, G, prec, s));
    }
    if (h) {
        FST_TRY(W.res.ensure(sizeof(double) * (size_t)m));
        to_double_kernel<float><<<grid_for(m, 256), 256, 0, s>>>(W.b.as<float>(), W.res.as<double>(), m);
        FST_CHECK_LAUNCH();
        FST_TRY(launch_atr<float>(M, Uc, W.res.as<double>(), m, h, s));
    }
    return FST_OK;
}
