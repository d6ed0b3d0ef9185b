// chol.cu -- blocked right-looking Cholesky G = L L^T of the normal matrix of the
// sampled least-squares problem (Algorithm 2, last step: solve the sampled LS), and
// the two triangular solves x <- L^-T L^-1 x.
//
// G is R x R row-major; only its lower triangle is read and L overwrites it.  Panel
// width NB = 64.  Per panel: (1) one block factors the diagonal block in shared
// memory; (2) a block per 64 rows solves the panel below, L21 = A21 L11^-T;
// (3) the trailing lower triangle is updated, A22 -= L21 L21^T, in 64 x 64 tiles.
// A non-positive (or NaN) pivot sets *d_flag; the caller reads it after the stream
// synchronises, so no step waits on the device.
#include <math.h>

#include "fst_internal.cuh"

namespace fst {

constexpr int NB = 64;

// Pivot floor: 16 * unit roundoff * the largest diagonal entry of G.  A pivot at or
// below it means G is numerically singular in T.
template <typename T>
__global__ void pivot_floor_kernel(const T* G, int R, T* floor_out) {
    __shared__ T red[256];
    T mx = T(0);
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const T d = G[(size_t)i * R + i];
        mx = d > mx ? d : mx;
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o && red[threadIdx.x + o] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const T eps = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
        *floor_out = T(16) * eps * red[0];
    }
}

template <typename T>
__global__ void potrf_diag_kernel(T* G, int R, int k0, int kb, int* flag, const T* floor_p) {
    __shared__ T A[NB][NB + 1];
    const int tid = threadIdx.x, B = blockDim.x;
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        A[i][j] = j <= i ? G[(size_t)(k0 + i) * R + k0 + j] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
            const T d = A[j][j];
            if (!(d > *floor_p)) atomicOr(flag, 1);
            A[j][j] = sqrt(d);
        }
        __syncthreads();
        const T piv = A[j][j];
        for (int i = j + 1 + tid; i < kb; i += B) A[i][j] /= piv;
        __syncthreads();
        const int w = kb - j - 1;
        for (int e = tid; e < w * w; e += B) {
            const int i = j + 1 + e / w, c = j + 1 + e % w;
            if (c <= i) A[i][c] -= A[i][j] * A[c][j];
        }
        __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        if (j <= i) G[(size_t)(k0 + i) * R + k0 + j] = A[i][j];
    }
}

// L21 = A21 L11^-T for rows row0 .. row0+63 (row0 = k0 + kb + 64*blockIdx.x).
template <typename T>
__global__ void trsm_panel_kernel(T* G, int R, int k0, int kb) {
    extern __shared__ __align__(16) unsigned char trsm_smem[];
    T (*L)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(trsm_smem);
    T (*X)[NB + 1] = L + NB;
    const int tid = threadIdx.x, B = blockDim.x;
    const int row0 = k0 + kb + NB * blockIdx.x;
    const int rows = R - row0 < NB ? R - row0 : NB;
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        L[i][j] = j <= i ? G[(size_t)(k0 + i) * R + k0 + j] : T(0);
    }
    for (int e = tid; e < rows * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        X[i][j] = G[(size_t)(row0 + i) * R + k0 + j];
    }
    __syncthreads();
    if (tid < rows) {
        for (int c = 0; c < kb; ++c) {
            T s = X[tid][c];
            for (int cc = 0; cc < c; ++cc) s -= X[tid][cc] * L[c][cc];
            X[tid][c] = s / L[c][c];
        }
    }
    __syncthreads();
    for (int e = tid; e < rows * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        G[(size_t)(row0 + i) * R + k0 + j] = X[i][j];
    }
}

// A22 -= L21 L21^T on lower 64x64 tiles of the trailing matrix starting at t0 = k0 + kb.
template <typename T>
__global__ void __launch_bounds__(256) syrk_update_kernel(T* G, int R, int k0, int kb, int t0) {
    constexpr int KC = 32;                    // panel columns staged per step
    __shared__ __align__(16) T As[KC][NB];   // [t][row within tile]
    __shared__ __align__(16) T Bs[KC][NB];
    // lower tile index (ti >= tc) from the linear block id
    const long long b = blockIdx.x;
    int ti = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while ((long long)ti * (ti + 1) / 2 > b) --ti;
    const int tc = (int)(b - (long long)ti * (ti + 1) / 2);
    const int r0 = t0 + ti * NB, c0 = t0 + tc * NB;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
    for (int tb = 0; tb < kb; tb += KC) {
        __syncthreads();
        for (int e = tid; e < NB * KC; e += 256) {
            const int i = e / KC, t = e - i * KC;
            const bool inb = tb + t < kb;
            As[t][i] = (r0 + i < R && inb) ? G[(size_t)(r0 + i) * R + k0 + tb + t] : T(0);
            Bs[t][i] = (c0 + i < R && inb) ? G[(size_t)(c0 + i) * R + k0 + tb + t] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < KC; ++t) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[t][ty * 4 + a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[t][tx * 4 + c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = r0 + ty * 4 + a;
        if (i >= R) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = c0 + tx * 4 + c;
            if (j < R && j <= i) G[(size_t)i * R + j] -= acc[a][c];
        }
    }
}

// ---------------------------------------------------------------- FP32 path, 128-wide panels
// Diagonal block of width kb <= PB in shared memory (dynamic).
template <int PB>
__global__ void potrf_diag_wide_kernel(float* G, int R, int k0, int kb, int* flag, const float* floor_p) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float (*A)[PB + 1] = reinterpret_cast<float (*)[PB + 1]>(dsm);
    const int tid = threadIdx.x, B = blockDim.x;
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        A[i][j] = j <= i ? G[(size_t)(k0 + i) * R + k0 + j] : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
            const float d = A[j][j];
            if (!(d > *floor_p)) atomicOr(flag, 1);
            A[j][j] = sqrtf(d);
        }
        __syncthreads();
        const float inv = 1.f / A[j][j];
        for (int i = j + 1 + tid; i < kb; i += B) A[i][j] *= inv;
        __syncthreads();
        // trailing update of the block: a 16 x (B/16) thread grid over (row, column)
        const int tc = tid & 15, tr = tid >> 4, nr = B >> 4;
        for (int i = j + 1 + tr; i < kb; i += nr) {
            const float lij = A[i][j];
            for (int c = j + 1 + tc; c <= i; c += 16) A[i][c] -= lij * A[c][j];
        }
        __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        if (j <= i) G[(size_t)(k0 + i) * R + k0 + j] = A[i][j];
    }
}

// L21 = A21 L11^-T, 32 rows per block, thread per row.
template <int PB>
__global__ void trsm_panel_wide_kernel(float* G, int R, int k0, int kb) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float (*L)[PB + 1] = reinterpret_cast<float (*)[PB + 1]>(dsm);
    float (*X)[PB + 1] = L + PB;
    const int tid = threadIdx.x, B = blockDim.x;
    const int row0 = k0 + kb + 32 * blockIdx.x;
    const int rows = R - row0 < 32 ? R - row0 : 32;
    for (int e = tid; e < kb * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        L[i][j] = j <= i ? G[(size_t)(k0 + i) * R + k0 + j] : 0.f;
    }
    for (int e = tid; e < rows * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        X[i][j] = G[(size_t)(row0 + i) * R + k0 + j];
    }
    __shared__ float Linvd[PB];
    for (int c = tid; c < kb; c += B) Linvd[c] = 1.f / G[(size_t)(k0 + c) * R + k0 + c];
    __syncthreads();
    if (tid < rows) {
        // forward substitution along the row, four independent partial sums per column
        for (int c = 0; c < kb; ++c) {
            float s0 = X[tid][c], s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int cc = 0;
            for (; cc + 3 < c; cc += 4) {
                s0 -= X[tid][cc] * L[c][cc];
                s1 -= X[tid][cc + 1] * L[c][cc + 1];
                s2 -= X[tid][cc + 2] * L[c][cc + 2];
                s3 -= X[tid][cc + 3] * L[c][cc + 3];
            }
            for (; cc < c; ++cc) s0 -= X[tid][cc] * L[c][cc];
            X[tid][c] = ((s0 + s1) + (s2 + s3)) * Linvd[c];
        }
    }
    __syncthreads();
    for (int e = tid; e < rows * kb; e += B) {
        const int i = e / kb, j = e - i * kb;
        G[(size_t)(row0 + i) * R + k0 + j] = X[i][j];
    }
}

// A22 -= L21 L21^T on lower 128 x 128 tiles, 8 x 8 outputs per thread, K in chunks of 32.
__global__ void __launch_bounds__(256) syrk128_kernel(float* G, int R, int k0, int kb, int t0) {
    constexpr int TS = 128, KC = 32;
    __shared__ __align__(16) float As[KC][TS + 4];
    __shared__ __align__(16) float Bs[KC][TS + 4];
    const long long b = blockIdx.x;
    int ti = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while ((long long)ti * (ti + 1) / 2 > b) --ti;
    const int tj = (int)(b - (long long)ti * (ti + 1) / 2);
    const int r0 = t0 + ti * TS, c0 = t0 + tj * TS;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const bool vec = (R & 3) == 0 && (k0 & 3) == 0;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int tb = 0; tb < kb; tb += KC) {
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * 256;
            const int row = e >> 3, c4 = (e & 7) * 4;
            float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
            const int ga = r0 + row, gb = c0 + row, kk = tb + c4;
            if (vec && kk + 3 < kb) {
                if (ga < R) {
                    const float4 x = *reinterpret_cast<const float4*>(G + (size_t)ga * R + k0 + kk);
                    va[0] = x.x; va[1] = x.y; va[2] = x.z; va[3] = x.w;
                }
                if (gb < R) {
                    const float4 x = *reinterpret_cast<const float4*>(G + (size_t)gb * R + k0 + kk);
                    vb[0] = x.x; vb[1] = x.y; vb[2] = x.z; vb[3] = x.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (kk + q < kb) {
                        if (ga < R) va[q] = G[(size_t)ga * R + k0 + kk + q];
                        if (gb < R) vb[q] = G[(size_t)gb * R + k0 + kk + q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[c4 + q][row] = va[q];
                Bs[c4 + q][row] = vb[q];
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gi = r0 + ty * 8 + i;
        if (gi >= R) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gj = c0 + tx * 8 + j;
            if (gj < R && gj <= gi) G[(size_t)gi * R + gj] -= acc[i][j];
        }
    }
}

template <typename T>
fst_status cholesky_lower(T* G, int R, int* d_flag, cudaStream_t s) {
    // d_flag points at two ints of scratch: the flag, then room for the pivot floor
    T* floor_p = reinterpret_cast<T*>(d_flag + 2);
    pivot_floor_kernel<T><<<1, 256, 0, s>>>(G, R, floor_p);
    FST_CHECK_LAUNCH();
    if (sizeof(T) == 4) {
        constexpr int PB = 128;
        float* Gf = reinterpret_cast<float*>(G);
        const float* fl = reinterpret_cast<const float*>(floor_p);
        const size_t diag_smem = (size_t)PB * (PB + 1) * sizeof(float);
        const size_t trsm_smem = (size_t)(PB + 32) * (PB + 1) * sizeof(float);
        FST_CUDA(cudaFuncSetAttribute(potrf_diag_wide_kernel<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem));
        FST_CUDA(cudaFuncSetAttribute(trsm_panel_wide_kernel<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)trsm_smem));
        for (int k0 = 0; k0 < R; k0 += PB) {
            const int kb = R - k0 < PB ? R - k0 : PB;
            potrf_diag_wide_kernel<PB><<<1, 512, diag_smem, s>>>(Gf, R, k0, kb, d_flag, fl);
            FST_CHECK_LAUNCH();
            const int t0 = k0 + kb;
            const int rest = R - t0;
            if (rest <= 0) break;
            trsm_panel_wide_kernel<PB><<<(rest + 31) / 32, 128, trsm_smem, s>>>(Gf, R, k0, kb);
            FST_CHECK_LAUNCH();
            const long long nt = (rest + 127) / 128;
            syrk128_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(Gf, R, k0, kb, t0);
            FST_CHECK_LAUNCH();
        }
        return FST_OK;
    }
    const size_t trsm_smem = 2 * NB * (NB + 1) * sizeof(T);
    FST_CUDA(cudaFuncSetAttribute(trsm_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)trsm_smem));
    for (int k0 = 0; k0 < R; k0 += NB) {
        const int kb = R - k0 < NB ? R - k0 : NB;
        potrf_diag_kernel<T><<<1, 256, 0, s>>>(G, R, k0, kb, d_flag, floor_p);
        FST_CHECK_LAUNCH();
        const int t0 = k0 + kb;
        const int rest = R - t0;
        if (rest <= 0) break;
        trsm_panel_kernel<T><<<(rest + NB - 1) / NB, NB, trsm_smem, s>>>(G, R, k0, kb);
        FST_CHECK_LAUNCH();
        const long long nt = (rest + NB - 1) / NB;
        syrk_update_kernel<T><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(G, R, k0, kb, t0);
        FST_CHECK_LAUNCH();
    }
    return FST_OK;
}

// ------------------------------------------------------------------ triangular solves
// Linv[b] = L_bb^-1 for every 64 x 64 diagonal block (computed once per factorisation):
// thread c solves L_bb X = e_c by forward substitution for column c of the inverse.
template <typename T>
__global__ void invert_diag_kernel(const T* L, int R, T* Linv) {
    __shared__ T Ls[NB][NB + 1];
    const int b = blockIdx.x, k0 = b * NB;
    const int kb = R - k0 < NB ? R - k0 : NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e - i * NB;
        Ls[i][j] = (i < kb && j <= i) ? L[(size_t)(k0 + i) * R + k0 + j] : T(i == j ? 1 : 0);
    }
    __syncthreads();
    T* out = Linv + (size_t)b * NB * NB;    // row-major [i][c]
    const int c = threadIdx.x;
    if (c < NB) {
        T col[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            T s = i == c ? T(1) : T(0);
#pragma unroll
            for (int k = 0; k < i; ++k) s -= Ls[i][k] * col[k];
            col[i] = i < c ? T(0) : s / Ls[i][i];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) out[i * NB + c] = col[i];
    }
}

// Forward step for diagonal block b: every block forms x_b = Linv_bb xin_b, block 0 stores it
// in y; rows below block b (64 per block, a warp per row) subtract L_{i,b} x_b from xin.
template <typename T>
__global__ void __launch_bounds__(256) fwd_step_kernel(const T* L, const T* Linv, int R, int b, T* xin, T* y) {
    __shared__ T xs[NB], xb[NB];
    const int k0 = b * NB, kb = R - k0 < NB ? R - k0 : NB;
    for (int i = threadIdx.x; i < NB; i += blockDim.x) xs[i] = i < kb ? xin[k0 + i] : T(0);
    __syncthreads();
    const T* Li = Linv + (size_t)b * NB * NB;
    {
        // x_b = Linv_bb xs: four threads per row, 16 contiguous entries each (coalesced)
        const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < NB / 4; ++c) s += Li[i * NB + part * (NB / 4) + c] * xs[part * (NB / 4) + c];
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (part == 0) xb[i] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < kb; i += blockDim.x) y[k0 + i] = xb[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = k0 + kb + blockIdx.x * NB;
    for (int rr = warp; rr < NB; rr += blockDim.x >> 5) {
        const int i = r0 + rr;
        if (i >= R) break;
        T s = T(0);
        for (int c = lane; c < kb; c += 32) s += L[(size_t)i * R + k0 + c] * xb[c];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) xin[i] -= s;
    }
}

// Backward step for block b: x_b = Linv_bb^T yin_b stored in out; rows above subtract
// L_{b,i}^T x_b from yin (thread per row, coalesced along i).
template <typename T>
__global__ void __launch_bounds__(256) bwd_step_kernel(const T* L, const T* Linv, int R, int b, T* yin, T* out) {
    __shared__ T ys[NB], xb[NB];
    const int k0 = b * NB, kb = R - k0 < NB ? R - k0 : NB;
    for (int i = threadIdx.x; i < NB; i += blockDim.x) ys[i] = i < kb ? yin[k0 + i] : T(0);
    __syncthreads();
    const T* Li = Linv + (size_t)b * NB * NB;
    for (int i = threadIdx.x; i < NB; i += blockDim.x) {
        T s = T(0);
        for (int c = 0; c < NB; ++c) s += Li[c * NB + i] * ys[c];
        xb[i] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < kb; i += blockDim.x) out[k0 + i] = xb[i];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k0) {
        T s = T(0);
        for (int c = 0; c < kb; ++c) s += L[(size_t)(k0 + c) * R + i] * xb[c];
        yin[i] -= s;
    }
}

template <typename T>
fst_status chol_invert_diag(const T* L, int R, T* Linv, cudaStream_t s) {
    const int nblk = (R + NB - 1) / NB;
    invert_diag_kernel<T><<<nblk, NB, 0, s>>>(L, R, Linv);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

// x <- L^-T L^-1 x (x and y: R values of T; y is scratch).
template <typename T>
fst_status chol_solve(const T* L, const T* Linv, int R, T* x, T* y, cudaStream_t s) {
    const int nblk = (R + NB - 1) / NB;
    for (int b = 0; b < nblk; ++b) {
        const int rest = R - (b + 1) * NB;
        const int grid = rest > 0 ? (rest + NB - 1) / NB : 1;
        fwd_step_kernel<T><<<grid, 256, 0, s>>>(L, Linv, R, b, x, y);
        FST_CHECK_LAUNCH();
    }
    for (int b = nblk - 1; b >= 0; --b) {
        const int k0 = b * NB;
        const int grid = k0 > 0 ? (k0 + 255) / 256 : 1;
        bwd_step_kernel<T><<<grid, 256, 0, s>>>(L, Linv, R, b, y, x);
        FST_CHECK_LAUNCH();
    }
    return FST_OK;
}

template fst_status cholesky_lower<float>(float*, int, int*, cudaStream_t);
template fst_status cholesky_lower<double>(double*, int, int*, cudaStream_t);
template <typename T>
fst_status chol_solve_graph(SolveGraph& g, const T* L, const T* Linv, int R, T* x, T* y, cudaStream_t s) {
    if (!g.exec || g.L != L || g.Linv != Linv || g.x != x || g.R != R || g.elem != (int)sizeof(T)) {
        if (g.exec) {
            FST_CUDA(cudaStreamSynchronize(s));
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        if (!g.cap) FST_CUDA(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
        FST_CUDA(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = fst_kernel_launches();
        fst_status st = chol_solve<T>(L, Linv, R, x, y, g.cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g.cap, &graph);
        if (st != FST_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        g.nodes = fst_kernel_launches() - before;
        g.L = L;
        g.Linv = Linv;
        g.x = x;
        g.R = R;
        g.elem = (int)sizeof(T);
    }
    FST_CUDA(cudaGraphLaunch(g.exec, s));
    count_launches(g.nodes);
    return FST_OK;
}

template fst_status chol_solve_graph<float>(SolveGraph&, const float*, const float*, int, float*, float*, cudaStream_t);
template fst_status chol_solve_graph<double>(SolveGraph&, const double*, const double*, int, double*, double*,
                                             cudaStream_t);

template fst_status chol_invert_diag<float>(const float*, int, float*, cudaStream_t);
template fst_status chol_invert_diag<double>(const double*, int, double*, cudaStream_t);
template fst_status chol_solve<float>(const float*, const float*, int, float*, float*, cudaStream_t);
template fst_status chol_solve<double>(const double*, const double*, int, double*, double*, cudaStream_t);

}  // namespace fst
