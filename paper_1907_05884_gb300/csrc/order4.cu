// order4.cu -- order-4 functional sparse Tucker models (eq. func_tuck with d = 4: three space
// axes and time, the SP4D case of Sec. 6 and Table 1): evaluation at unstructured points and
// the randomized least-squares core refit (Sec. 5, eq. rand_core; Algorithm 2 with uniform
// sampling).
//
// Ranks up to 64 a mode (the paper's SP4D ranks are 30 x 38 x 5 x 11, R = 62,700).  The
// evaluation runs on the CUDA cores: per point the four factor vectors, then the contraction
// with the core streamed through shared memory in slabs alpha_{i j . .} (r3 r4 values), the
// last factor vector in registers.  The refit is that of order-3 models with the third and
// fourth factors as one Kronecker factor: the normal matrix of the sampled rows from the
// packed Khatri-Rao operand on the tensor cores (BF16; 15.7 GB in FP32 at R = 62,700), its
// FP32 Cholesky factor with tensor-core trailing updates, and conjugate gradients on the
// normal equations preconditioned by that factor, with A p and A^T q applied in the factored
// four-way form (FP32 products, FP64 sums across row blocks and in the vectors).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fst_internal.cuh"

struct fst_model4 {
    int device = 0;
    int r[4] = {0, 0, 0, 0};
    int p[4] = {0, 0, 0, 0};
    int pe[4] = {0, 0, 0, 0};       // 1 + highest degree with a nonzero coefficient
    double lo[4], hi[4];
    std::vector<int32_t> colptr[4], rowidx[4];
    std::vector<double> val[4];
    std::vector<double> alpha;      // host copy of the core (C order)
    double* W64[4] = {nullptr, nullptr, nullptr, nullptr};   // (pe x r) with sqrt(2n+1) folded in
    float* W32[4] = {nullptr, nullptr, nullptr, nullptr};
    double* alpha64 = nullptr;
    float* alpha32 = nullptr;
    fst::DevBuf idx, U[4], b, rv, part, vec, ahl, scal, G, LT, Linv, chol_ws, xw, flag;
    std::recursive_mutex mu;
    long long R() const { return (long long)r[0] * r[1] * r[2] * r[3]; }
};

namespace fst {
namespace {

int bucket(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : 64; }

struct Args4 {
    int r[4], pe[4];
    double sc[4], of[4];    // t = sc y + of maps the box to [-1, 1]
};

Args4 args_of(const fst_model4* m) {
    Args4 a;
    for (int k = 0; k < 4; ++k) {
        a.r[k] = m->r[k];
        a.pe[k] = m->pe[k];
        a.sc[k] = 2.0 / (m->hi[k] - m->lo[k]);
        a.of[k] = -2.0 * m->lo[k] / (m->hi[k] - m->lo[k]) - 1.0;
    }
    return a;
}

// w_j = sum_n W[n r + j] L_n(t), n < pe, j < r (W with sqrt(2n+1) folded in): the Legendre
// recurrence L_{n+1} = ((2n+1) t L_n - n L_{n-1}) / (n+1), accumulated into a register array
template <typename T, int RM>
__device__ __forceinline__ void factor_regs(T t, const T* __restrict__ W, int pe, int r, T (&w)[RM]) {
#pragma unroll
    for (int j = 0; j < RM; ++j) w[j] = T(0);
    T Lm = T(0), L = T(1);
    for (int n = 0; n < pe; ++n) {
        const T* row = W + (size_t)n * r;
#pragma unroll
        for (int j = 0; j < RM; ++j)
            if (j < r) w[j] = fma(L, __ldg(row + j), w[j]);
        const T Ln = (T(2 * n + 1) * t * L - T(n) * Lm) / T(n + 1);
        Lm = L;
        L = Ln;
    }
}

// the same into shared memory, column j at s[j * stride] (any r)
template <typename T>
__device__ __forceinline__ void factor_smem(T t, const T* __restrict__ W, int pe, int r, T* s, int stride) {
    for (int j = 0; j < r; ++j) s[j * stride] = T(0);
    T Lm = T(0), L = T(1);
    for (int n = 0; n < pe; ++n) {
        const T* row = W + (size_t)n * r;
        for (int j = 0; j < r; ++j) s[j * stride] = fma(L, __ldg(row + j), s[j * stride]);
        const T Ln = (T(2 * n + 1) * t * L - T(n) * Lm) / T(n + 1);
        Lm = L;
        L = Ln;
    }
}

// f(x) for one point a thread: w1, w2, w3 in shared memory, w4 in registers; t_ij =
// sum_k w3_k sum_l alpha_ijkl w4_l over slabs staged in shared memory, sps slabs at a time,
// f = sum_ij w1_i w2_j t_ij with two accumulators.  Dynamic shared memory: (r1 + r2 + r3) x
// blockDim values, then sps r3 r4 core values.
template <typename T, int RM>
__global__ void __launch_bounds__(128) eval4_kernel(Args4 a, const T* __restrict__ W1, const T* __restrict__ W2,
                                                    const T* __restrict__ W3, const T* __restrict__ W4,
                                                    const T* __restrict__ alpha, const T* __restrict__ x, int64_t n,
                                                    T* __restrict__ out, int sps) {
    extern __shared__ __align__(16) unsigned char smem4[];
    T* sw = reinterpret_cast<T*>(smem4);
    const int B = blockDim.x, tid = threadIdx.x;
    const int r1 = a.r[0], r2 = a.r[1], r3 = a.r[2], r4 = a.r[3];
    T* slab = sw + (size_t)(r1 + r2 + r3) * B;
    const int slab_len = r3 * r4, npair = r1 * r2;
    const int64_t q = (int64_t)blockIdx.x * B + tid;
    const bool live = q < n;
    T w4[RM];
    const T* w3 = sw + (size_t)(r1 + r2) * B + tid;
    {
        const T y0 = live ? x[q] : T(0), y1 = live ? x[n + q] : T(0);
        const T y2 = live ? x[2 * n + q] : T(0), y3 = live ? x[3 * n + q] : T(0);
        factor_smem<T>(fma(y0, (T)a.sc[0], (T)a.of[0]), W1, a.pe[0], r1, sw + tid, B);
        factor_smem<T>(fma(y1, (T)a.sc[1], (T)a.of[1]), W2, a.pe[1], r2, sw + (size_t)r1 * B + tid, B);
        factor_smem<T>(fma(y2, (T)a.sc[2], (T)a.of[2]), W3, a.pe[2], r3, sw + (size_t)(r1 + r2) * B + tid, B);
        factor_regs<T, RM>(fma(y3, (T)a.sc[3], (T)a.of[3]), W4, a.pe[3], r4, w4);
    }
    T f0 = T(0), f1 = T(0);
    for (int p0 = 0; p0 < npair; p0 += sps) {
        const int ns = npair - p0 < sps ? npair - p0 : sps;
        __syncthreads();
        for (int e = tid; e < ns * slab_len; e += B) slab[e] = alpha[(size_t)p0 * slab_len + e];
        __syncthreads();
        for (int s = 0; s < ns; ++s) {
            const int pr = p0 + s, i = pr / r2, j = pr - i * r2;
            const T* sl = slab + s * slab_len;
            T t0 = T(0), t1 = T(0);
            for (int k = 0; k < r3; ++k) {
                T u = T(0);
#pragma unroll
                for (int l = 0; l < RM; ++l)
                    if (l < r4) u = fma(sl[k * r4 + l], w4[l], u);
                if (k & 1) t1 = fma(u, w3[(size_t)k * B], t1);
                else t0 = fma(u, w3[(size_t)k * B], t0);
            }
            const T c = sw[(size_t)i * B + tid] * sw[(size_t)(r1 + j) * B + tid];
            if (s & 1) f1 = fma(c, t0 + t1, f1);
            else f0 = fma(c, t0 + t1, f0);
        }
    }
    if (live) out[q] = f0 + f1;
}

// ------------------------------------------------------------------ refit
// Factor values of the sampled rows, in FP64 from the stored points, rounded once to FP32
// (16 columns at a time, the recurrence redone per group of columns); b = u at those rows.
__global__ void __launch_bounds__(128) sampled_factors4_kernel(Args4 a, const double* __restrict__ W0,
                                                               const double* __restrict__ W1,
                                                               const double* __restrict__ W2,
                                                               const double* __restrict__ W3, const float* __restrict__ x,
                                                               int64_t Q, const int64_t* __restrict__ idx, int64_t m,
                                                               const float* __restrict__ u, float* U0, float* U1,
                                                               float* U2, float* U3, float* __restrict__ b) {
    const double* Ws[4] = {W0, W1, W2, W3};
    float* Us[4] = {U0, U1, U2, U3};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = idx[s];
        b[s] = u[q];
        for (int k = 0; k < 4; ++k) {
            const int r = a.r[k], pe = a.pe[k];
            const double t = fma((double)x[k * Q + q], a.sc[k], a.of[k]);
            for (int j0 = 0; j0 < r; j0 += 16) {
                double acc[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.0;
                double Lm = 0.0, L = 1.0;
                for (int n = 0; n < pe; ++n) {
                    const double* row = Ws[k] + (size_t)n * r + j0;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                        if (j0 + jj < r) acc[jj] = fma(L, __ldg(row + jj), acc[jj]);
                    const double Ln = (double(2 * n + 1) * t * L - double(n) * Lm) / double(n + 1);
                    Lm = L;
                    L = Ln;
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if (j0 + jj < r) Us[k][s * r + j0 + jj] = (float)acc[jj];
            }
        }
    }
}

// ph + pl = p (FP64) as two FP32 arrays
__global__ void split_hilo_kernel(const double* __restrict__ p, float* __restrict__ ph, float* __restrict__ pl,
                                  int64_t R) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)p[i];
        ph[i] = h;
        pl[i] = (float)(p[i] - (double)h);
    }
}

// rv_s = (b_s if b) + scale * (A p)_s, A p = sum_ij w1_i w2_j sum_k w3_k sum_l p_ijkl w4_l, one
// row a thread: p as FP32 hi + lo slabs staged in shared memory (sps slabs of r3 r4 values
// each part), w3 in shared memory and w4 in registers; the slab sums in FP32, the sums over j
// in FP32 and over i in FP64.
template <int RM>
__global__ void __launch_bounds__(256) residual4_kernel(Args4 a, const float* __restrict__ U0,
                                                        const float* __restrict__ U1, const float* __restrict__ U2,
                                                        const float* __restrict__ U3, const float* __restrict__ b,
                                                        const float* __restrict__ ph, const float* __restrict__ pl,
                                                        int64_t m, double scale, double* __restrict__ rv, int sps) {
    extern __shared__ __align__(16) unsigned char smem4[];
    float* sh = reinterpret_cast<float*>(smem4);
    const int r1 = a.r[0], r2 = a.r[1], r3 = a.r[2], r4 = a.r[3];
    const int slab_len = r3 * r4;
    float* sl_ = sh + (size_t)sps * slab_len;
    float* w3 = sl_ + (size_t)sps * slab_len + threadIdx.x;   // w3_k at w3[k blockDim]
    const int npair = r1 * r2;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < m; s0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool live = s < m;
        float w4[RM];
#pragma unroll
        for (int l = 0; l < RM; ++l) w4[l] = live && l < r4 ? U3[s * r4 + l] : 0.f;
        for (int k = 0; k < r3; ++k) w3[(size_t)k * blockDim.x] = live ? U2[s * r3 + k] : 0.f;
        double f = 0.0;
        float si = 0.f;
        int icur = 0;
        for (int p0 = 0; p0 < npair; p0 += sps) {
            const int ns = npair - p0 < sps ? npair - p0 : sps;
            __syncthreads();
            for (int e = threadIdx.x; e < ns * slab_len; e += blockDim.x) {
                sh[e] = ph[(size_t)p0 * slab_len + e];
                sl_[e] = pl[(size_t)p0 * slab_len + e];
            }
            __syncthreads();
            for (int q = 0; q < ns; ++q) {
                const int pr = p0 + q, i = pr / r2, j = pr - i * r2;
                if (i != icur) {
                    if (live) f = fma((double)si, (double)U0[s * r1 + icur], f);
                    si = 0.f;
                    icur = i;
                }
                const float* hh = sh + q * slab_len;
                const float* ll = sl_ + q * slab_len;
                float th = 0.f, tl = 0.f;
                for (int k = 0; k < r3; ++k) {
                    float uh = 0.f, ul = 0.f;
#pragma unroll
                    for (int l = 0; l < RM; ++l)
                        if (l < r4) {
                            uh = fmaf(hh[k * r4 + l], w4[l], uh);
                            ul = fmaf(ll[k * r4 + l], w4[l], ul);
                        }
                    th = fmaf(uh, w3[(size_t)k * blockDim.x], th);
                    tl = fmaf(ul, w3[(size_t)k * blockDim.x], tl);
                }
                if (live) si = fmaf(th + tl, U1[s * r2 + j], si);
            }
        }
        if (live) {
            f = fma((double)si, (double)U0[s * r1 + icur], f);
            rv[s] = (b ? (double)b[s] : 0.0) + scale * f;
        }
    }
}

// Partial sums of A^T rv over the rows of part `blockIdx.x` (rows_per_part rows each): a
// thread owns triples (i, j, k) and the RM accumulators of their l; rows staged 32 at a time.
template <int RM>
__global__ void __launch_bounds__(256) atr4_kernel(Args4 a, const float* __restrict__ U0,
                                                   const float* __restrict__ U1, const float* __restrict__ U2,
                                                   const float* __restrict__ U3, const double* __restrict__ rv,
                                                   int64_t m, int64_t rows_per_part, double* __restrict__ part) {
    constexpr int S = 32;
    extern __shared__ __align__(16) unsigned char smem4[];
    const int r1 = a.r[0], r2 = a.r[1], r3 = a.r[2], r4 = a.r[3];
    float* u0s = reinterpret_cast<float*>(smem4);
    float* u1s = u0s + S * r1;
    float* u2s = u1s + S * r2;
    float* u3s = u2s + S * r3;
    float* qs = u3s + S * RM;
    const int64_t lo = (int64_t)blockIdx.x * rows_per_part;
    const int64_t hi = lo + rows_per_part < m ? lo + rows_per_part : m;
    const long long R = (long long)r1 * r2 * r3 * r4;
    double* out = part + (size_t)blockIdx.x * R;
    const int ntri = r1 * r2 * r3;
    for (int t0 = 0; t0 < ntri; t0 += blockDim.x) {
        const int tri = t0 + threadIdx.x;
        const bool own = tri < ntri;
        const int i = own ? tri / (r2 * r3) : 0, jk = own ? tri - i * r2 * r3 : 0, j = jk / r3, k = jk - j * r3;
        float acc[RM];
#pragma unroll
        for (int l = 0; l < RM; ++l) acc[l] = 0.f;
        for (int64_t s0 = lo; s0 < hi; s0 += S) {
            const int ns = hi - s0 < S ? (int)(hi - s0) : S;
            __syncthreads();
            auto stage = [&](const float* U, int r, float* dst, int ld) {
                for (int e = threadIdx.x; e < ns * r; e += blockDim.x) {
                    const int ss = e / r, c = e - ss * r;
                    dst[ss * ld + c] = U[(s0 + ss) * r + c];
                }
            };
            stage(U0, r1, u0s, r1);
            stage(U1, r2, u1s, r2);
            stage(U2, r3, u2s, r3);
            stage(U3, r4, u3s, RM);
            for (int e = threadIdx.x; e < ns; e += blockDim.x) qs[e] = (float)rv[s0 + e];
            __syncthreads();
            if (own) {
                for (int ss = 0; ss < ns; ++ss) {
                    const float c = qs[ss] * u0s[ss * r1 + i] * u1s[ss * r2 + j] * u2s[ss * r3 + k];
                    const float* w = u3s + ss * RM;
#pragma unroll
                    for (int l = 0; l < RM; ++l)
                        if (l < r4) acc[l] = fmaf(c, w[l], acc[l]);
                }
            }
        }
        if (own) {
#pragma unroll
            for (int l = 0; l < RM; ++l)
                if (l < r4) out[(size_t)tri * r4 + l] = (double)acc[l];
        }
    }
}

// U34[s][k r4 + l] = w3_k w4_l (the rows of the third and fourth factors as one Kronecker
// factor, so that the packed-operand Gram of order-3 rows serves)
__global__ void kron34_kernel(const float* __restrict__ U2, const float* __restrict__ U3, int64_t m, int r3, int r4,
                              float* __restrict__ U34) {
    const int64_t n = m * r3 * r4;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / (r3 * r4);
        const int kl = (int)(e - s * r3 * r4), k = kl / r4, l = kl - k * r4;
        U34[e] = U2[s * r3 + k] * U3[s * r4 + l];
    }
}

// lower triangle: acc (+)= g  (first: copy)
__global__ void add_lower4_kernel(float* __restrict__ acc, const float* __restrict__ g, int R, int first) {
    const int64_t n = (int64_t)R * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / R), j = (int)(e - (int64_t)i * R);
        if (j <= i) acc[e] = first ? g[e] : acc[e] + g[e];
    }
}

// G_jj <- (1 + delta) G_jj (the preconditioner of a Gram that does not factor in FP32)
__global__ void shift_diag4_kernel(float* G, int R, float delta) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x)
        G[(size_t)i * R + i] *= 1.f + delta;
}

// dir 0: f = (float) d; dir 1: d = f
__global__ void convert4_kernel(double* __restrict__ d, float* __restrict__ f, int dir, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dir == 0) f[i] = (float)d[i];
        else d[i] = (double)f[i];
    }
}

__global__ void sum_parts4_kernel(const double* __restrict__ part, int nparts, int64_t R, double* __restrict__ g) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < R; a += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int b = 0; b < nparts; ++b) sum += part[(size_t)b * R + a];
        g[a] = sum;
    }
}

// out[d] = x_d . y_d for d < nd, one block in a fixed order
constexpr int kDot4 = 1024;
__global__ void __launch_bounds__(kDot4) dots4_kernel(const double* x0, const double* y0, const double* x1,
                                                      const double* y1, const double* x2, const double* y2,
                                                      int64_t n, int nd, double* out) {
    __shared__ double red[3][kDot4 / 32];
    double a[3] = {0.0, 0.0, 0.0};
    const double* xs[3] = {x0, x1, x2};
    const double* ys[3] = {y0, y1, y2};
    for (int64_t i = threadIdx.x; i < n; i += kDot4)
        for (int d = 0; d < nd; ++d) a[d] += xs[d][i] * ys[d][i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o; o >>= 1) a[d] += __shfl_xor_sync(0xffffffffu, a[d], o);
        if (lane == 0) red[d][warp] = a[d];
    }
    __syncthreads();
    if (warp == 0) {
        for (int d = 0; d < 3; ++d) {
            double v = red[d][lane];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && d < nd) out[d] = v;
        }
    }
}

// op 0: y += a x; 2: y = x + a y
__global__ void vec4_kernel(double* __restrict__ y, const double* __restrict__ x, double a, int op, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (op == 0) y[i] += a * x[i];
        else y[i] = x[i] + a * y[i];
    }
}

}  // namespace
}  // namespace fst

// ------------------------------------------------------------------ host side
using namespace fst;

namespace {

fst_status free4(fst_model4* m) {
    for (int k = 0; k < 4; ++k) {
        if (m->W64[k]) cudaFree(m->W64[k]);
        if (m->W32[k]) cudaFree(m->W32[k]);
    }
    if (m->alpha64) cudaFree(m->alpha64);
    if (m->alpha32) cudaFree(m->alpha32);
    return FST_OK;
}

fst_status upload_core4(fst_model4* m) {
    const size_t R = (size_t)m->R();
    std::vector<float> a32(R);
    for (size_t i = 0; i < R; ++i) a32[i] = (float)m->alpha[i];
    FST_CUDA(cudaMemcpy(m->alpha64, m->alpha.data(), R * sizeof(double), cudaMemcpyHostToDevice));
    FST_CUDA(cudaMemcpy(m->alpha32, a32.data(), R * sizeof(float), cudaMemcpyHostToDevice));
    return FST_OK;
}

// the slabs of r3 r4 values a stage holds within `budget` bytes (at least one)
int slabs_per_stage(const fst_model4* m, size_t elem, size_t budget) {
    const size_t per = (size_t)m->r[2] * m->r[3] * elem;
    size_t n = budget / (per ? per : 1);
    if (n < 1) n = 1;
    if (n > 64) n = 64;
    return (int)n;
}

template <typename T>
fst_status launch_eval4(const fst_model4* m, const T* x, int64_t n, T* out, cudaStream_t s) {
    const int B = sizeof(T) == 8 ? 64 : 128;
    const int sps = slabs_per_stage(m, sizeof(T), 48 * 1024);
    const size_t smem = ((size_t)(m->r[0] + m->r[1] + m->r[2]) * B + (size_t)sps * m->r[2] * m->r[3]) * sizeof(T);
    const Args4 a = args_of(m);
    const T* Wp[4];
    for (int k = 0; k < 4; ++k) Wp[k] = sizeof(T) == 8 ? (const T*)m->W64[k] : (const T*)m->W32[k];
    const T* alpha = sizeof(T) == 8 ? (const T*)m->alpha64 : (const T*)m->alpha32;
    const unsigned grid = (unsigned)((n + B - 1) / B);
    const int RM = bucket(m->r[3]);
#define FST_EV4(V)                                                                                       \
    {                                                                                                    \
        auto kern = eval4_kernel<T, V>;                                                                  \
        FST_TRY(allow_smem(kern, smem));                                                                 \
        kern<<<grid, B, smem, s>>>(a, Wp[0], Wp[1], Wp[2], Wp[3], alpha, x, n, out, sps);                \
    }
    if (RM == 8) FST_EV4(8) else if (RM == 16) FST_EV4(16) else if (RM == 32) FST_EV4(32) else FST_EV4(64)
#undef FST_EV4
    FST_CHECK_LAUNCH();
    return FST_OK;
}

fst_status check_model4_call(const fst_model4* m) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == m->device, "model lives on device %d, current device is %d", m->device, dev);
    return FST_OK;
}

}  // namespace

extern "C" fst_status fst_model4_create(const fst_model4_desc* d, fst_model4** out) {
    FST_REQUIRE(d != nullptr && out != nullptr, "desc or out is NULL");
    *out = nullptr;
    long long R = 1;
    for (int k = 0; k < 4; ++k) {
        FST_REQUIRE(d->r[k] >= 1 && d->r[k] <= FST4_MAX_RANK, "rank r[%d] = %d outside 1..%d", k, d->r[k],
                    FST4_MAX_RANK);
        FST_REQUIRE(d->p[k] >= 0 && d->p[k] <= FST_MAX_DEGREE, "degree p[%d] = %d outside 0..%d", k, d->p[k],
                    FST_MAX_DEGREE);
        FST_REQUIRE(d->hi[k] > d->lo[k], "empty box in mode %d", k);
        FST_REQUIRE(d->colptr[k] && d->rowidx[k] && d->val[k], "coefficients of mode %d are NULL", k);
        R *= d->r[k];
    }
    FST_REQUIRE(d->alpha != nullptr, "alpha is NULL");
    FST_REQUIRE(R <= (1LL << 24), "core of %lld entries is too large", R);
    struct Guard {
        fst_model4* p;
        ~Guard() {
            if (p) {
                free4(p);
                delete p;
            }
        }
        fst_model4* operator->() const { return p; }
        fst_model4* get() const { return p; }
    } m{new fst_model4()};
    FST_CUDA(cudaGetDevice(&m->device));
    for (int k = 0; k < 4; ++k) {
        m->r[k] = d->r[k];
        m->p[k] = d->p[k];
        m->lo[k] = d->lo[k];
        m->hi[k] = d->hi[k];
        const int r = d->r[k];
        FST_REQUIRE(d->colptr[k][0] == 0, "colptr[%d][0] must be 0", k);
        for (int j = 0; j < r; ++j)
            FST_REQUIRE(d->colptr[k][j + 1] >= d->colptr[k][j], "colptr of mode %d decreases", k);
        const int nnz = d->colptr[k][r];
        m->colptr[k].assign(d->colptr[k], d->colptr[k] + r + 1);
        m->rowidx[k].assign(d->rowidx[k], d->rowidx[k] + nnz);
        m->val[k].assign(d->val[k], d->val[k] + nnz);
        int pe = 1;
        for (int e = 0; e < nnz; ++e) {
            const int n = d->rowidx[k][e];
            FST_REQUIRE(n >= 0 && n <= d->p[k], "degree %d of mode %d outside 0..%d", n, k, d->p[k]);
            if (d->val[k][e] != 0.0) pe = std::max(pe, n + 1);
        }
        m->pe[k] = pe;
        std::vector<double> W((size_t)pe * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int e = d->colptr[k][j]; e < d->colptr[k][j + 1]; ++e) {
                const int n = d->rowidx[k][e];
                if (n < pe) W[(size_t)n * r + j] += d->val[k][e] * sqrt(2.0 * n + 1.0);
            }
        std::vector<float> W32(W.begin(), W.end());
        FST_CUDA(cudaMalloc(&m->W64[k], W.size() * sizeof(double)));
        FST_CUDA(cudaMalloc(&m->W32[k], W.size() * sizeof(float)));
        FST_CUDA(cudaMemcpy(m->W64[k], W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice));
        FST_CUDA(cudaMemcpy(m->W32[k], W32.data(), W32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    m->alpha.assign(d->alpha, d->alpha + R);
    FST_CUDA(cudaMalloc(&m->alpha64, (size_t)R * sizeof(double)));
    FST_CUDA(cudaMalloc(&m->alpha32, (size_t)R * sizeof(float)));
    FST_TRY(upload_core4(m.get()));
    *out = m.p;
    m.p = nullptr;
    return FST_OK;
}

extern "C" void fst_model4_free(fst_model4* m) {
    if (!m) return;
    free4(m);
    delete m;
}

extern "C" fst_status fst_model4_read_core(const fst_model4* m, double* alpha) {
    FST_REQUIRE(m != nullptr && alpha != nullptr, "model or alpha is NULL");
    memcpy(alpha, m->alpha.data(), m->alpha.size() * sizeof(double));
    return FST_OK;
}

extern "C" fst_status fst_eval4(const fst_model4* m, const float* x, int64_t n, float* out, fst_stream stream) {
    FST_TRY(check_model4_call(m));
    FST_REQUIRE(n >= 0, "n must be non-negative");
    if (n == 0) return FST_OK;
    FST_REQUIRE(x && out, "x or out is NULL");
    return launch_eval4<float>(m, x, n, out, (cudaStream_t)stream);
}

extern "C" fst_status fst_eval4_f64(const fst_model4* m, const double* x, int64_t n, double* out,
                                    fst_stream stream) {
    FST_TRY(check_model4_call(m));
    FST_REQUIRE(n >= 0, "n must be non-negative");
    if (n == 0) return FST_OK;
    FST_REQUIRE(x && out, "x or out is NULL");
    return launch_eval4<double>(m, x, n, out, (cudaStream_t)stream);
}


// The core refit of an order-4 model (Sec. 5, eq. rand_core; Algorithm 2 with uniform
// sampling): rows by the sampler of the order-3 refit, factor values in FP64 rounded to FP32;
// G = A^T A in `prec` from the packed operand of rows (w1 (x) w2) (x) (w3 (x) w4) (the FP32
// sum of the Grams of blocks of 16,384 rows), its FP32
// Cholesky factor (if that fails, that of G + delta diag(G) for growing delta, which still
// preconditions the unshifted equations), alpha_0 = G^-1 A^T b, then conjugate
// gradients on A^T A alpha = A^T b preconditioned by the factor, A p and A^T q in the
// four-way factored form.  Stops when the relative update falls below tol, or stops
// shrinking at a level below 1e-6.
extern "C" fst_status fst_refit4(fst_model4* m, const float* x, const float* u, int64_t Q, int64_t mrows,
                                 uint64_t seed, fst_prec prec, const fst_refit_opts* opts, fst_refit_report* report,
                                 fst_stream stream) {
    FST_TRY(check_model4_call(m));
    FST_REQUIRE(x && u, "x or u is NULL");
    FST_REQUIRE(Q > 0 && mrows > 0, "Q and m must be positive");
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_refit4 assembles the normal matrix in TF32, BF16 or BF16X3");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(pointer_device(x) == dev && pointer_device(u) == dev, "x and u must be device memory");
    if (mrows > Q) mrows = Q;
    const long long RL = m->R();
    if (mrows < RL) {
        set_error("m = %lld sampled rows < R = %lld unknowns", (long long)mrows, RL);
        return FST_ERANK;
    }
    FST_REQUIRE(RL <= 131072, "R = %lld: the normal matrix of an order-4 refit is limited to R <= 131072", RL);
    const int R = (int)RL;
    std::lock_guard<std::recursive_mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const int max_refine = opts ? opts->max_refine : 200;
    const double tol = (opts && opts->refine_tol > 0) ? opts->refine_tol : 1e-8;
    // a preconditioner from a shifted Gram converges slowly, where an update of 1e-5 still
    // leaves an error several times larger: the stagnation floor is 1e-6
    const double floor_ok = 1e-6;
    fst_refit_report r;
    memset(&r, 0, sizeof r);
    r.m = mrows;
    cudaEvent_t ev[5];
    for (auto& e : ev) FST_CUDA(cudaEventCreate(&e));
    struct Ev {
        cudaEvent_t* e;
        ~Ev() {
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    FST_CUDA(cudaEventRecord(ev[0], s));
    const Args4 a = args_of(m);
    // 1-2. rows and factor values
    FST_TRY(m->idx.ensure(sizeof(int64_t) * (size_t)mrows));
    FST_TRY(sample_rows(seed, Q, mrows, m->idx.as<int64_t>(), s));
    float* U[4];
    size_t uoff[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) uoff[k + 1] = uoff[k] + (size_t)mrows * m->r[k];
    const size_t u34 = (size_t)mrows * m->r[2] * m->r[3];
    FST_TRY(m->U[0].ensure(sizeof(float) * (uoff[4] + u34)));
    for (int k = 0; k < 4; ++k) U[k] = m->U[0].as<float>() + uoff[k];
    float* U34 = m->U[0].as<float>() + uoff[4];
    FST_TRY(m->b.ensure(sizeof(float) * (size_t)mrows));
    float* b = m->b.as<float>();
    {
        const int grid = (int)std::min<int64_t>((mrows + 127) / 128, 8LL * sm_count());
        sampled_factors4_kernel<<<grid, 128, 0, s>>>(a, m->W64[0], m->W64[1], m->W64[2], m->W64[3], x, Q,
                                                      m->idx.as<int64_t>(), mrows, u, U[0], U[1], U[2], U[3], b);
        FST_CHECK_LAUNCH();
        kron34_kernel<<<8 * sm_count(), 256, 0, s>>>(U[2], U[3], mrows, m->r[2], m->r[3], U34);
        FST_CHECK_LAUNCH();
    }
    FST_CUDA(cudaEventRecord(ev[1], s));
    // vectors: alpha, alpha_0, g = A^T b, r, z, p, w (R doubles each); the residual rows; the
    // FP32 halves of p; the solve's FP32 working copies
    FST_TRY(m->vec.ensure(sizeof(double) * (size_t)R * 7));
    double* al = m->vec.as<double>();
    double* al0 = al + R;
    double* g = al0 + R;
    double* rr = g + R;
    double* zz = rr + R;
    double* pp = zz + R;
    double* ww = pp + R;
    FST_TRY(m->rv.ensure(sizeof(double) * (size_t)mrows));
    double* rv = m->rv.as<double>();
    FST_TRY(m->ahl.ensure(sizeof(float) * (size_t)R * 2));
    float* ph = m->ahl.as<float>();
    float* pl = ph + R;
    FST_TRY(m->xw.ensure(sizeof(float) * (size_t)R * 2));
    float* xw = m->xw.as<float>();
    float* yw = xw + R;
    FST_TRY(m->scal.ensure(sizeof(double) * 4));
    double* sc = m->scal.as<double>();
    FST_TRY(m->flag.ensure(sizeof(int) * 8));
    int* flag = m->flag.as<int>();            // [0] pivot, [1] factorisation waits, [2] Gram waits,
                                              // [4] solve error, [5] solve ticket
    // A^T partition: ~2 parts a SM, whole multiples of 32 rows
    int64_t nparts = 2LL * sm_count();
    const int64_t rpp = ((mrows + nparts - 1) / nparts + 31) / 32 * 32;
    nparts = (mrows + rpp - 1) / rpp;
    FST_TRY(m->part.ensure(sizeof(double) * (size_t)nparts * R));
    double* part = m->part.as<double>();
    const int RM4 = bucket(m->r[3]);
    const int sps = slabs_per_stage(m, 2 * sizeof(float), 64 * 1024);
    const size_t res_smem = ((size_t)sps * m->r[2] * m->r[3] * 2 + (size_t)m->r[2] * 256) * sizeof(float);
    const size_t atr_smem = ((size_t)32 * (m->r[0] + m->r[1] + m->r[2] + RM4) + 32) * sizeof(float);
    const int vgrid = (int)std::min<long long>((R + 255) / 256, 4LL * sm_count());
    auto residual = [&](const double* v, bool with_b, double scale) -> fst_status {
        split_hilo_kernel<<<vgrid, 256, 0, s>>>(v, ph, pl, R);
        FST_CHECK_LAUNCH();
        const int grid = (int)std::min<int64_t>((mrows + 255) / 256, 2LL * sm_count());
#define FST_RES4(V)                                                                                        \
    {                                                                                                      \
        auto kern = residual4_kernel<V>;                                                                   \
        FST_TRY(allow_smem(kern, res_smem));                                                               \
        kern<<<grid, 256, res_smem, s>>>(a, U[0], U[1], U[2], U[3], with_b ? b : nullptr, ph, pl, mrows,   \
                                         scale, rv, sps);                                                  \
    }
        if (RM4 == 8) FST_RES4(8) else if (RM4 == 16) FST_RES4(16) else if (RM4 == 32) FST_RES4(32) else FST_RES4(64)
#undef FST_RES4
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    auto atr = [&](double* out) -> fst_status {
#define FST_ATR4(V)                                                                                        \
    atr4_kernel<V><<<(unsigned)nparts, 256, atr_smem, s>>>(a, U[0], U[1], U[2], U[3], rv, mrows, rpp, part)
        if (RM4 == 8) FST_ATR4(8); else if (RM4 == 16) FST_ATR4(16); else if (RM4 == 32) FST_ATR4(32); else FST_ATR4(64);
#undef FST_ATR4
        FST_CHECK_LAUNCH();
        sum_parts4_kernel<<<vgrid, 256, 0, s>>>(part, (int)nparts, R, out);
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    auto dots = [&](const double* x0, const double* y0, const double* x1, const double* y1, double* h) -> fst_status {
        dots4_kernel<<<1, kDot4, 0, s>>>(x0, y0, x1, y1, nullptr, nullptr, R, 2, sc);
        FST_CHECK_LAUNCH();
        FST_CUDA(cudaMemcpyAsync(h, sc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        return FST_OK;
    };
    auto vec = [&](double* y, const double* xv, double c, int op) -> fst_status {
        vec4_kernel<<<vgrid, 256, 0, s>>>(y, xv, c, op, R);
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    // h = A^T b
    convert4_kernel<<<(int)std::min<int64_t>((mrows + 255) / 256, 8LL * sm_count()), 256, 0, s>>>(rv, b, 1, mrows);
    FST_CHECK_LAUNCH();
    FST_TRY(atr(g));
    // 3-4. the normal matrix and its factor.  The tensor cores accumulate the sums over the
    // rows in FP32 and their rounding grows with the number of rows (1e-3 of the largest
    // diagonal entry at R = 62,700, m = 4R in one pass), so G is the FP32 sum of the Grams of
    // blocks of kGramRows rows.  A Gram that still does not factor is factored again from the
    // saved sum with growing relative diagonal shifts: the factor of G + delta diag(G) still
    // preconditions the unshifted equations, which the conjugate gradients solve.
    constexpr int64_t kGramRows = 16384;
    FST_TRY(m->G.ensure(sizeof(float) * (size_t)R * R));
    FST_TRY(m->LT.ensure(sizeof(float) * (size_t)R * R));
    float* G = m->G.as<float>();
    float* Gsave = m->LT.as<float>();
    FST_CUDA(cudaMemsetAsync(flag, 0, 8 * sizeof(int), s));
    const int r34 = m->r[2] * m->r[3];
    const int agrid = 16 * sm_count();
    for (int64_t s0 = 0; s0 < mrows; s0 += kGramRows) {
        const int64_t nr = std::min<int64_t>(kGramRows, mrows - s0);
        FST_TRY(gram_pk_rows(U[0] + s0 * m->r[0], U[1] + s0 * m->r[1], U34 + s0 * r34, nr, m->r[0], m->r[1], r34, G,
                             prec, flag + 2, s));
        add_lower4_kernel<<<agrid, 256, 0, s>>>(Gsave, G, R, s0 == 0 ? 1 : 0);
        FST_CHECK_LAUNCH();
    }
    FST_CUDA(cudaEventRecord(ev[2], s));
    FST_CUDA(cudaMemcpyAsync(G, Gsave, sizeof(float) * (size_t)R * R, cudaMemcpyDeviceToDevice, s));
    const float shifts[5] = {0.f, 2.44140625e-4f, 3.90625e-3f, 3.125e-2f, 0.25f};   // 0, 2^-12, 2^-8, 2^-5, 2^-2
    for (int attempt = 0;; ++attempt) {
        if (attempt > 0) {
            FST_CUDA(cudaMemcpyAsync(G, Gsave, sizeof(float) * (size_t)R * R, cudaMemcpyDeviceToDevice, s));
            shift_diag4_kernel<<<vgrid, 256, 0, s>>>(G, R, shifts[attempt]);
            FST_CHECK_LAUNCH();
            r.shifted_preconditioner = attempt;
        }
        FST_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), s));
        FST_TRY(cholesky_lower<float>(G, R, flag, m->chol_ws, s));
        int hf[2] = {0, 0};
        FST_CUDA(cudaMemcpyAsync(hf, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        FST_CUDA(cudaStreamSynchronize(s));
        if (hf[1]) {
            set_error("order-4 refit: a bounded device wait of the factorisation expired");
            return FST_ETIMEOUT;
        }
        if (!hf[0]) break;
        if (attempt == 4) {
            set_error("order-4 refit: the normal matrix is not positive definite in FP32 (rank-deficient sample)");
            return FST_ENOTSPD;
        }
    }
    FST_TRY(m->Linv.ensure(3 * sizeof(float) * (size_t)((R + 63) / 64) * 64 * 64));
    FST_TRY(chol_invert_diag<float>(G, R, m->Linv.as<float>(), s));
    FST_TRY(chol_transpose<float>(G, R, m->LT.as<float>(), s));
    FST_CUDA(cudaEventRecord(ev[3], s));
    auto solve = [&](double* v) -> fst_status {   // v <- (L L^T)^-1 v in the factor's precision
        convert4_kernel<<<vgrid, 256, 0, s>>>(v, xw, 0, R);
        FST_CHECK_LAUNCH();
        FST_TRY(chol_solve<float>(G, m->LT.as<float>(), m->Linv.as<float>(), R, xw, yw, flag + 4, s));
        convert4_kernel<<<vgrid, 256, 0, s>>>(v, xw, 1, R);
        FST_CHECK_LAUNCH();
        return FST_OK;
    };
    // 5. alpha_0 = G^-1 h, then the preconditioned conjugate gradients
    FST_CUDA(cudaMemcpyAsync(al, g, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
    FST_TRY(solve(al));
    FST_CUDA(cudaMemcpyAsync(al0, al, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
    int steps = 0, stop = max_refine <= 0 ? 1 : 0;
    double last = 0.0, prev = 0.0;
    if (max_refine > 0) {
        FST_TRY(residual(al, true, -1.0));
        FST_TRY(atr(rr));
        FST_CUDA(cudaMemcpyAsync(zz, rr, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
        FST_TRY(solve(zz));
        FST_CUDA(cudaMemcpyAsync(pp, zz, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
        double h[2];
        FST_TRY(dots(rr, zz, al, al, h));
        double rz = h[0];
        for (int it = 0; it < max_refine && rz > 0.0; ++it) {
            FST_TRY(residual(pp, false, 1.0));   // q = A p
            FST_TRY(atr(ww));                     // w = A^T q
            FST_TRY(dots(pp, ww, pp, pp, h));
            const double pw = h[0], pp2 = h[1];
            if (!(pw > 0.0) || !isfinite(pw)) {
                stop = 2;
                break;
            }
            const double ak = rz / pw;
            FST_TRY(vec(al, pp, ak, 0));          // alpha += ak p
            FST_TRY(vec(rr, ww, -ak, 0));         // r -= ak w
            FST_CUDA(cudaMemcpyAsync(zz, rr, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
            FST_TRY(solve(zz));                   // z = M^-1 r
            FST_TRY(dots(rr, zz, al, al, h));
            ++steps;
            prev = last;
            last = h[1] > 0.0 ? fabs(ak) * sqrt(pp2 / h[1]) : 0.0;
            if (!isfinite(last)) {
                stop = 2;
                break;
            }
            if (last <= tol || (steps >= 3 && last > 0.5 * prev && last <= floor_ok)) {
                stop = 1;
                break;
            }
            const double beta = h[0] / rz;
            rz = h[0];
            FST_TRY(vec(pp, zz, beta, 2));        // p = z + beta p
        }
        if (rz <= 0.0 && steps == 0) stop = 1;    // r = 0: alpha_0 solves the problem
    }
    FST_CUDA(cudaEventRecord(ev[4], s));
    std::vector<double> ha((size_t)R), h0((size_t)R);
    FST_CUDA(cudaMemcpyAsync(ha.data(), al, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaMemcpyAsync(h0.data(), al0, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    int serr = 0;
    FST_CUDA(cudaMemcpyAsync(&serr, flag + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    float t[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
    r.ms_factors = t[0];
    r.ms_gram = t[1];
    r.ms_cholesky = t[2];
    r.ms_refine = t[3];
    r.refine_steps = steps;
    r.last_rel_update = last;
    double dn = 0, an = 0;
    for (int i = 0; i < R; ++i) {
        dn += (ha[i] - h0[i]) * (ha[i] - h0[i]);
        an += ha[i] * ha[i];
    }
    r.first_rel_change = an > 0 ? sqrt(dn / an) : 0.0;
    if (report) *report = r;
    if (serr) {
        set_error("order-4 refit: a bounded device wait of the triangular solves expired");
        return FST_ETIMEOUT;
    }
    if (stop != 1 && !(isfinite(last) && last <= floor_ok)) {
        set_error("order-4 refit: conjugate gradients did not converge (last relative update %.3e after %d steps)",
                  last, steps);
        return FST_ENOTCONV;
    }
    for (double v : ha)
        if (!isfinite(v)) {
            set_error("order-4 refit produced a non-finite core");
            return FST_ENOTSPD;
        }
    m->alpha = ha;
    return upload_core4(m);
}
