// chol.cu -- blocked right-looking Cholesky G = L L^T of the normal matrix of the
// sampled least-squares problem (Algorithm 2, last step: solve the sampled LS), and
// the two triangular solves x <- L^-T L^-1 x.
//
// G is R x R row-major; only its lower triangle is read and L overwrites it.  FP64: panel
// width NB = 64; per panel (1) one block factors the diagonal block in shared memory;
// (2) a block per 64 rows solves the panel below, L21 = A21 L11^-T; (3) the trailing
// lower triangle is updated, A22 -= L21 L21^T, in 64 x 64 tiles on the CUDA cores.
// FP32: 128-wide panels with the trailing update on the tensor cores (see below).
// A non-positive (or NaN) pivot sets d_flag[0]; the caller reads it after the stream
// synchronises, so no step waits on the host.
#include <math.h>

#include <cuda_bf16.h>

#include "fst_internal.cuh"
#include "tc_ptx.cuh"

namespace fst {

constexpr int NB = 64;

// Pivot floors, one per column: 16 * unit roundoff * G_jj.  A pivot (the Schur complement
// of column j) at or below its floor means G is numerically singular in T at the scale of
// that column; the test is invariant under diagonal scaling of G.
template <typename T>
__global__ void pivot_floor_kernel(const T* G, int R, T* floors) {
    const T eps = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x)
        floors[i] = T(16) * eps * G[(size_t)i * R + i];
}

template <typename T>
__global__ void potrf_diag_kernel(T* G, int R, int k0, int kb, int* flag, const T* floors) {
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
            if (!(d > floors[k0 + j])) atomicOr(flag, 1);
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

// ---------------------------------------------------------------- FP32 path, tensor cores
// 128-wide panels.  Per panel: (1) one block factors the diagonal block in shared memory in
// 32-wide sub-panels (a warp factors each 32 x 32 block in registers, the rows below solve
// against it, the rest of the block takes a register-tiled rank-32 update) and inverts the
// four 32 x 32 diagonal blocks of L11; (2) the panel below, L21 = A21 L11^-T, is solved by
// 32-column block substitution with those inverses and written to G in FP32 and, split into
// BF16 high and low parts, as tensor-core operand tiles; (3) each lower 128 x 128 tile of
// the trailing matrix takes A22 -= L21_i L21_j^T from tcgen05 MMAs (BF16x3: hi*hi + hi*lo +
// lo*hi, FP32 accumulation in tensor memory), operands moved by bulk copies and the G tile
// read ahead into registers.
constexpr int PB = 128;
constexpr int SUB = 32;
constexpr int AS = PB + 4;                          // row stride (floats) of shared panels
constexpr uint32_t kPartBytes = 16384;              // 128 rows x 64 K BF16, one of hi / lo
constexpr uint32_t kHalfBytes = 2 * kPartBytes;     // K-half: hi then lo
constexpr uint32_t kTileBytes = 2 * kHalfBytes;     // two K-halves of a 128-row operand tile
constexpr long long kCholWaitLimit = 2000000000LL;  // ~1 s of clock cycles

// byte offset of (row, k) of a packed operand tile (hi part; the lo part is kPartBytes on)
__device__ __forceinline__ uint32_t packed_off(int row, int k) {
    return (uint32_t)(k >> 6) * kHalfBytes + tc::kmajor_offset((uint32_t)row, (uint32_t)(k & 63) * 2u, 128u);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
}

// Diagonal block [k0, k0+kb) factored in place (L11 written to G) in FS-wide sub-panels:
// (a) a warp factors the FS x FS block in registers (shuffles), (b) the rows below solve
// against it (thread per row), (c) the rest of the block takes a register-tiled rank-FS
// update.  With want_inv, the inverses of the four 32 x 32 diagonal blocks of L11 go to
// Dinv (4 x 32 x 32, row-major).  512 threads; dynamic shared memory: A (PB x AS) and the
// transposed sub-panel P (FS x PB), reused for the inverses (4 x 32 x 32 floats).
constexpr int FS = 16;
static_assert(FS * PB <= 4 * SUB * SUB, "the sub-panel buffer is reused for the diagonal inverses");
__device__ __forceinline__ void potrf_inv_body(float* G, int R, int k0, int kb, int* flag, const float* floors,
                                               float* Dinv, int want_inv) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float (*A)[AS] = reinterpret_cast<float (*)[AS]>(dsm);
    float (*P)[PB] = reinterpret_cast<float (*)[PB]>(dsm + sizeof(float) * PB * AS);   // P[k][row]
    __shared__ float invd[PB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // all 32 loads of a thread in flight at once
        float v[PB * PB / 512];
#pragma unroll
        for (int u = 0; u < PB * PB / 512; ++u) {
            const int e = tid + u * 512, i = e >> 7, j = e & (PB - 1);
            v[u] = (i < kb && j <= i) ? G[(size_t)(k0 + i) * R + k0 + j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < PB * PB / 512; ++u) {
            const int e = tid + u * 512;
            A[e >> 7][e & (PB - 1)] = v[u];
        }
    }
    __syncthreads();
    for (int sb = 0; sb < kb; sb += FS) {
        const int w = kb - sb < FS ? kb - sb : FS;
        if (warp == 0) {
            // (a) FS x FS diagonal block in registers: lane i < FS holds row sb + i (padded
            // rows beyond kb are identity rows; lanes >= FS idle along)
            const int li = lane < FS ? lane : FS - 1;
            float a[FS];
            float dinv = 1.f, piv = 1.f;
            const float fl = lane < w ? floors[k0 + sb + lane] : 0.f;
#pragma unroll
            for (int c = 0; c < FS; ++c)
                a[c] = li < w ? (c <= li ? A[sb + li][sb + c] : 0.f) : (c == li ? 1.f : 0.f);
#pragma unroll 16
            for (int j = 0; j < FS; ++j) {
                const float d = __shfl_sync(0xffffffffu, a[j], j);
                // the pivot's reciprocal square root from the hardware approximation (a few
                // ulp; the factor preconditions the conjugate gradients), its root as d / sqrt(d)
                const float inv = rsqrtf(d);
                const float sq = d * inv;
                if (lane == j) {
                    dinv = inv;
                    piv = d;
                }
                a[j] = lane == j ? sq : (lane > j ? a[j] * inv : a[j]);
#pragma unroll 15
                for (int c = j + 1; c < FS; ++c) {
                    const float lcj = __shfl_sync(0xffffffffu, a[j], c);
                    if (lane >= c) a[c] = fmaf(-a[j], lcj, a[c]);
                }
            }
            // the pivot test after the chain: no global load inside it
            if (lane < w && !(piv > fl)) atomicOr(flag, 1);
            if (lane < w) {
#pragma unroll
                for (int c = 0; c < FS; ++c) {
                    const float v = c <= lane ? a[c] : 0.f;
                    A[sb + lane][sb + c] = v;
                    P[c][sb + lane] = v;
                }
                invd[sb + lane] = dinv;
            }
        }
        __syncthreads();
        const int below = sb + w, nb = kb - below;
        // (b) rows below the sub-block: x = a L_sub^-T, thread per row
        if (tid < nb) {
            const int i = below + tid;
            float x[FS];
#pragma unroll
            for (int c = 0; c < FS; ++c) x[c] = A[i][sb + c];
#pragma unroll
            for (int c = 0; c < FS; ++c) {
                float s0 = x[c], s1 = 0.f;
#pragma unroll
                for (int k = 0; k < c; k += 2) {
                    s0 = fmaf(-x[k], A[sb + c][sb + k], s0);
                    if (k + 1 < c) s1 = fmaf(-x[k + 1], A[sb + c][sb + k + 1], s1);
                }
                x[c] = (s0 + s1) * invd[sb + c];
            }
#pragma unroll
            for (int c = 0; c < FS; ++c) {
                A[i][sb + c] = x[c];
                P[c][i] = x[c];
            }
        }
        __syncthreads();
        // (c) rank-FS update of the rest of the block, 4 x 4 lower tiles per thread
        const int nt4 = (nb + 3) >> 2;
        for (int t = tid; t < nt4 * (nt4 + 1) / 2; t += 512) {
            int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
            while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while (ti * (ti + 1) / 2 > t) --ti;
            const int tcol = t - ti * (ti + 1) / 2;
            const int i0 = below + 4 * ti, c0 = below + 4 * tcol;
            float acc[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll
            for (int k = 0; k < FS; ++k) {
                const float4 pi = *reinterpret_cast<const float4*>(&P[k][i0]);
                const float4 pc = *reinterpret_cast<const float4*>(&P[k][c0]);
                const float vi[4] = {pi.x, pi.y, pi.z, pi.w}, vc[4] = {pc.x, pc.y, pc.z, pc.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(vi[x], vc[y], acc[x][y]);
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y)
                    if (i0 + x < kb && c0 + y <= i0 + x) A[i0 + x][c0 + y] -= acc[x][y];
        }
        __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += 512) {
        const int i = e / kb, j = e - i * kb;
        if (j <= i) G[(size_t)(k0 + i) * R + k0 + j] = A[i][j];
    }
    if (!want_inv) return;
    // inverses of the four diagonal 32 x 32 blocks (needs kb = PB): warp d, lane c solves
    // L_dd x = e_c with x in shared memory (P reused, column c per lane: rolled loops);
    // entries above the diagonal come out zero
    if (warp < 4) {
        const int d = warp, c = lane, o = d * SUB;
        float* X = &P[0][0] + d * SUB * SUB;        // [i][c] for this block
        for (int i = 0; i < SUB; ++i) {
            float s0 = i == c ? 1.f : 0.f, s1 = 0.f;
            int k = 0;
            for (; k + 1 < i; k += 2) {
                s0 = fmaf(-A[o + i][o + k], X[k * SUB + c], s0);
                s1 = fmaf(-A[o + i][o + k + 1], X[(k + 1) * SUB + c], s1);
            }
            if (k < i) s0 = fmaf(-A[o + i][o + k], X[k * SUB + c], s0);
            const float xi = (s0 + s1) * invd[o + i];
            X[i * SUB + c] = xi;
            Dinv[(o + i) * SUB + c] = xi;
        }
    }
}

__global__ void __launch_bounds__(512) potrf_inv_kernel(float* G, int R, int k0, int kb, int* flag,
                                                        const float* floors, float* Dinv, int want_inv) {
    potrf_inv_body(G, R, k0, kb, flag, floors, Dinv, want_inv);
}

// One step of a factorisation of several normal matrices at once (a grouped refit): the
// same panel of every matrix that still has it.  Each kernel below takes the step's jobs,
// one per matrix; a job's blocks (or tiles) are [first, first of the next job).
struct CholJob {
    float* G;
    const float* floors;
    float* Dinv;
    unsigned char* Lp;      // the packed panel this step writes (trsm) or the first panel (update)
    size_t pstride;
    int* flag;
    int R, k0, kb, want_inv;
    int t0, nt, ncol, npan; // trailing update: first row/column, tile rows, tile columns, panels
    long long first;
};
__device__ __forceinline__ int job_of(const CholJob* jobs, int njobs, long long x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__global__ void __launch_bounds__(512) potrf_inv_group_kernel(const CholJob* __restrict__ jobs) {
    const CholJob& j = jobs[blockIdx.x];
    potrf_inv_body(j.G, j.R, j.k0, j.kb, j.flag, j.floors, j.Dinv, j.want_inv);
}

// L21 = A21 L11^-T for kTrsmRows panel rows per block (256 threads): 32-column block
// substitution, X_d = (A_d - sum_{e<d} X_e L_de^T) Dinv_d^T.  Writes L21 (FP32) into G and the
// BF16 hi/lo operand tiles of the trailing update (rows at or beyond R as zeros).  Few rows a
// block keep each block's chain short (the panel solve sits on the factorisation's critical
// path) and spread the panel over more SMs.
constexpr int kTrsmRows = 32;
constexpr int kTrsmCQ = 256 / kTrsmRows;          // threads per row
constexpr int kTrsmNJ = SUB / kTrsmCQ;            // columns of a 32-column block per thread
__device__ __forceinline__ void trsm_pack_body(float* G, int R, int k0, const float* Dinv, unsigned char* Lp,
                                               int blk) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float (*X)[AS] = reinterpret_cast<float (*)[AS]>(dsm);                                        // panel rows
    float (*L)[AS] = reinterpret_cast<float (*)[AS]>(dsm + sizeof(float) * kTrsmRows * AS);      // L11
    float (*D)[SUB + 4] = reinterpret_cast<float (*)[SUB + 4]>(dsm + sizeof(float) * (kTrsmRows + PB) * AS);
    const int tid = threadIdx.x;
    const int t0 = k0 + PB;
    const int r0 = blk * kTrsmRows;
    const bool vec = (R & 3) == 0;
    {
        // the panel rows and L11: every load of a thread in flight at once
        constexpr int NX = kTrsmRows * (PB / 4) / 256, NL = PB * (PB / 4) / 256;
        float4 xv[NX], lv4[NL];
#pragma unroll
        for (int u = 0; u < NX; ++u) {
            const int e = tid + u * 256, r = e / (PB / 4), c4 = (e % (PB / 4)) * 4;
            const int g = t0 + r0 + r;
            const float* src = G + (size_t)g * R + k0 + c4;
            xv[u] = g >= R ? make_float4(0.f, 0.f, 0.f, 0.f)
                           : vec ? *reinterpret_cast<const float4*>(src) : make_float4(src[0], src[1], src[2], src[3]);
        }
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int e = tid + u * 256, r = e / (PB / 4), c4 = (e % (PB / 4)) * 4;
            const float* src = G + (size_t)(k0 + r) * R + k0 + c4;
            lv4[u] = vec ? *reinterpret_cast<const float4*>(src) : make_float4(src[0], src[1], src[2], src[3]);
        }
#pragma unroll
        for (int u = 0; u < NX; ++u) {
            const int e = tid + u * 256;
            *reinterpret_cast<float4*>(&X[e / (PB / 4)][(e % (PB / 4)) * 4]) = xv[u];
        }
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int e = tid + u * 256;
            *reinterpret_cast<float4*>(&L[e / (PB / 4)][(e % (PB / 4)) * 4]) = lv4[u];
        }
    }
    for (int e = tid; e < 4 * SUB * SUB; e += 256) D[e / SUB][e % SUB] = Dinv[e];
    __syncthreads();
    // thread: row r and the kTrsmNJ columns cq + kTrsmCQ j of the current 32-column block
    // (interleaved, so the threads of a row read consecutive L rows: no bank conflicts)
    const int r = tid / kTrsmCQ, cq = tid % kTrsmCQ;
    for (int d = 0; d < 4; ++d) {
        const int cb = d * SUB + cq;
        float y[kTrsmNJ];
#pragma unroll
        for (int j = 0; j < kTrsmNJ; ++j) y[j] = X[r][cb + kTrsmCQ * j];
        for (int k = 0; k < d * SUB; k += 4) {
            const float4 xk = *reinterpret_cast<const float4*>(&X[r][k]);
#pragma unroll
            for (int j = 0; j < kTrsmNJ; ++j) {
                const float4 lk = *reinterpret_cast<const float4*>(&L[cb + kTrsmCQ * j][k]);
                y[j] = fmaf(-xk.x, lk.x, y[j]);
                y[j] = fmaf(-xk.y, lk.y, y[j]);
                y[j] = fmaf(-xk.z, lk.z, y[j]);
                y[j] = fmaf(-xk.w, lk.w, y[j]);
            }
        }
        __syncthreads();   // every thread has read X's block d before it is overwritten
#pragma unroll
        for (int j = 0; j < kTrsmNJ; ++j) X[r][cb + kTrsmCQ * j] = y[j];
        __syncthreads();
        float xo[kTrsmNJ];
#pragma unroll
        for (int j = 0; j < kTrsmNJ; ++j) xo[j] = 0.f;
        for (int t = 0; t < SUB; t += 4) {
            const float4 yv = *reinterpret_cast<const float4*>(&X[r][d * SUB + t]);
#pragma unroll
            for (int j = 0; j < kTrsmNJ; ++j) {
                const float4 dv = *reinterpret_cast<const float4*>(&D[cb + kTrsmCQ * j][t]);
                xo[j] = fmaf(yv.x, dv.x, xo[j]);
                xo[j] = fmaf(yv.y, dv.y, xo[j]);
                xo[j] = fmaf(yv.z, dv.z, xo[j]);
                xo[j] = fmaf(yv.w, dv.w, xo[j]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kTrsmNJ; ++j) X[r][cb + kTrsmCQ * j] = xo[j];
        __syncthreads();
    }
    // write L21 to G and the packed operand rows: chunks of 8 columns, (PB / 8) / kTrsmCQ a thread
    const int g = t0 + r0 + r;
#pragma unroll
    for (int h = 0; h < PB / 8 / kTrsmCQ; ++h) {
        const int c0 = (h * kTrsmCQ + cq) * 8;
        float v[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = g < R ? X[r][c0 + j] : 0.f;
        if (g < R) {
            float* dst = G + (size_t)g * R + k0 + c0;
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j] = v[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) lo[j] = v[j] - __bfloat162float(__float2bfloat16_rn(v[j]));
        const int pr = r0 + r;
        unsigned char* tile = Lp + (size_t)(pr >> 7) * kTileBytes;
        const uint32_t off = packed_off(pr & 127, c0);
        *reinterpret_cast<uint4*>(tile + off) =
            make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
        *reinterpret_cast<uint4*>(tile + kPartBytes + off) = make_uint4(
            pack_bf16x2(lo[0], lo[1]), pack_bf16x2(lo[2], lo[3]), pack_bf16x2(lo[4], lo[5]), pack_bf16x2(lo[6], lo[7]));
    }
}

__global__ void __launch_bounds__(256) trsm_pack_kernel(float* G, int R, int k0, const float* Dinv,
                                                        unsigned char* Lp, int blk0) {
    trsm_pack_body(G, R, k0, Dinv, Lp, blk0 + blockIdx.x);
}
__global__ void __launch_bounds__(256) trsm_pack_group_kernel(const CholJob* __restrict__ jobs, int njobs) {
    const CholJob& j = jobs[job_of(jobs, njobs, blockIdx.x)];
    trsm_pack_body(j.G, j.R, j.k0, j.Dinv, j.Lp, (int)(blockIdx.x - j.first));
}

// A22 -= L21_i L21_j^T over the lower 128 x 128 tiles (ti >= tj) of the trailing matrix
// that starts at row/column t0.  Persistent: one CTA per SM walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 8 (one thread) moves the operands through a ring of
// kSyrkStages stages, one K-half of A and B (hi and lo) per stage, with bulk copies; warp 9
// (one thread) issues the MMAs into one of two 128-column TMEM accumulators; warps 0-7 read
// their 64 G entries of the tile into registers first, then take the accumulator
// (warp w: lanes 32(w%4).., columns 64(w/4)..), subtract and store -- so the G traffic of a
// tile overlaps the copies and MMAs of the next.
constexpr int kSyrkStages = 3;
constexpr int kSyrkThreads = 10 * 32;
__device__ __forceinline__ void lower_tile(long long t, int& ti, int& tj) {
    int x = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(x + 1) * (x + 2) / 2 <= t) ++x;
    while ((long long)x * (x + 1) / 2 > t) --x;
    ti = x;
    tj = (int)(t - (long long)x * (x + 1) / 2);
}

// Tile t of the lower trapezoid of an nt x nt tile grid cut to its first ncol tile columns:
// the ncol (ncol + 1) / 2 tiles of the leading triangle, then ncol tiles per further row.
__device__ __forceinline__ void trapezoid_tile(long long t, int ncol, int& ti, int& tj) {
    const long long tri = (long long)ncol * (ncol + 1) / 2;
    if (t < tri) {
        lower_tile(t, ti, tj);
    } else {
        const long long u = t - tri;
        ti = ncol + (int)(u / ncol);
        tj = (int)(u % ncol);
    }
}

// npan panels of 128 columns each make the K = 128 npan of the update; panel p's packed
// rows start 128 (npan - 1 - p) rows above t0 (each panel was packed from the row after its
// own diagonal block), at Lp + p * pstride.
struct SyrkTile {
    float* G;
    const unsigned char* Lp;
    size_t pstride;
    int R, t0, npan, ti, tj;
};
// the tiles of one trailing update
struct SyrkOne {
    float* G;
    const unsigned char* Lp;
    size_t pstride;
    int R, t0, nt, ncol, npan;
    long long first;    // tiles [first, count) of the trapezoid
    __device__ long long count() const {
        return (long long)ncol * (ncol + 1) / 2 + (long long)(nt - ncol) * ncol - first;
    }
    __device__ SyrkTile tile(long long t) const {
        SyrkTile x{G, Lp, pstride, R, t0, npan, 0, 0};
        trapezoid_tile(t + first, ncol, x.ti, x.tj);
        return x;
    }
};
// the tiles of the updates of several matrices (CholJob: first = the job's first tile)
struct SyrkGroup {
    const CholJob* jobs;
    int njobs;
    long long total;
    __device__ long long count() const { return total; }
    __device__ SyrkTile tile(long long t) const {
        const CholJob& j = jobs[job_of(jobs, njobs, t)];
        SyrkTile x{j.G, j.Lp, j.pstride, j.R, j.t0, j.npan, 0, 0};
        trapezoid_tile(t - j.first, j.ncol, x.ti, x.tj);
        return x;
    }
};

template <class Src>
__device__ __forceinline__ void syrk_tc_body(const Src& src, int* err) {
    extern __shared__ unsigned char syrk_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)syrk_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kSyrkStages * 2 * kHalfBytes);
    uint64_t* empty = full + kSyrkStages;
    uint64_t* tfull = empty + kSyrkStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = src.count();

    if (warp == 0) tc::tmem_alloc(tmem_slot, 256);
    if (tid == 0) {
        for (int s = 0; s < kSyrkStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 8);
        }
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    auto fail = [&](int code) {
        *abort_flag = 1;
        atomicOr(err, code);
    };

    if (warp == 8) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const SyrkTile x = src.tile(t);
                const int ti = x.ti, tj = x.tj, npan = x.npan, nh = 2 * npan;   // K-halves of 64
                const unsigned char* Lp = x.Lp;
                const size_t pstride = x.pstride;
                const bool diag = ti == tj;
                for (int h = 0; h < nh; ++h, ++it) {
                    const int s = it % kSyrkStages;
                    const uint32_t ph = (uint32_t)((it / kSyrkStages) & 1);
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, kCholWaitLimit)) {
                        fail(1);
                        break;
                    }
                    const int pan = h >> 1, up = npan - 1 - pan;
                    const unsigned char* src = Lp + (size_t)pan * pstride + (size_t)(h & 1) * kHalfBytes;
                    unsigned char* st = sm + s * 2 * kHalfBytes;
                    tc::mbar_arrive_expect_tx(&full[s], diag ? kHalfBytes : 2 * kHalfBytes);
                    tc::bulk_g2s(st, src + (size_t)(ti + up) * kTileBytes, kHalfBytes, &full[s]);
                    if (!diag)
                        tc::bulk_g2s(st + kHalfBytes, src + (size_t)(tj + up) * kTileBytes, kHalfBytes, &full[s]);
                }
            }
        }
    } else if (warp == 9) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t SBO = (128 / 16) * 128;
            constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
            int it = 0, n = 0;
            bool issued = false;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++n) {
                const SyrkTile x = src.tile(t);
                const bool diag = x.ti == x.tj;
                const int nh = 2 * x.npan;
                const int b = n & 1;
                if (!tc::mbar_wait(&tempty[b], (uint32_t)((n >> 1) & 1) ^ 1u, kCholWaitLimit)) {
                    fail(2);
                    break;
                }
                tc::fence_after_sync();
                bool ok = true;
                for (int h = 0; h < nh; ++h, ++it) {
                    const int s = it % kSyrkStages;
                    const uint32_t ph = (uint32_t)((it / kSyrkStages) & 1);
                    if (!tc::mbar_wait(&full[s], ph, kCholWaitLimit)) {
                        fail(4);
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_base = tc::smem_u32(sm + s * 2 * kHalfBytes);
                    const uint32_t b_base = diag ? a_base : a_base + kHalfBytes;
                    const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t ko = ks * 256;
                        const uint64_t ah = tc::make_desc(a_base + ko, 128, SBO);
                        const uint64_t al = tc::make_desc(a_base + kPartBytes + ko, 128, SBO);
                        const uint64_t bh = tc::make_desc(b_base + ko, 128, SBO);
                        const uint64_t bl = tc::make_desc(b_base + kPartBytes + ko, 128, SBO);
                        tc::mma_bf16(d, ah, bh, idesc, (h > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_bf16(d, ah, bl, idesc, 1u);
                        tc::mma_bf16(d, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                    issued = true;
                }
                if (!ok) break;
                tc::mma_commit(&tfull[b]);
            }
            if (issued) {
                // every MMA of this CTA completes before tensor memory is released
                tc::mma_commit(drain);
                if (!tc::mbar_wait(drain, 0u, kCholWaitLimit)) atomicOr(err, 16);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        int n = 0;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++n) {
            const SyrkTile x = src.tile(t);
            const int ti = x.ti, tj = x.tj, R = x.R, t0 = x.t0;
            float* G = x.G;
            const bool vec = (R & 3) == 0;
            const bool diag = ti == tj;
            const int grow = t0 + ti * 128 + (warp & 3) * 32 + lane;
            const int gcol0 = t0 + tj * 128 + (warp >> 2) * 64;
            float gv[64];
            if (grow < R) {
                const float* src = G + (size_t)grow * R + gcol0;
                if (vec && gcol0 + 64 <= R) {
#pragma unroll
                    for (int e = 0; e < 64; e += 4) {
                        const float4 x = *reinterpret_cast<const float4*>(src + e);
                        gv[e] = x.x;
                        gv[e + 1] = x.y;
                        gv[e + 2] = x.z;
                        gv[e + 3] = x.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 64; ++e) gv[e] = gcol0 + e < R ? src[e] : 0.f;
                }
            }
            const int b = n & 1;
            if (!tc::mbar_wait(&tfull[b], (uint32_t)((n >> 1) & 1), kCholWaitLimit)) {
                fail(8);
                break;
            }
            tc::fence_after_sync();
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * 128 + (warp >> 2) * 64);
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float v[16];
                tc::tmem_ld16(taddr + (uint32_t)c0, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; ++e) gv[c0 + e] -= v[e];
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[b]);
            if (grow < R) {
                float* dst = G + (size_t)grow * R + gcol0;
                if (vec && !diag && gcol0 + 64 <= R) {
#pragma unroll
                    for (int e = 0; e < 64; e += 4)
                        *reinterpret_cast<float4*>(dst + e) = make_float4(gv[e], gv[e + 1], gv[e + 2], gv[e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 64; ++e)
                        if (gcol0 + e < R && gcol0 + e <= grow) dst[e] = gv[e];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

__global__ void __launch_bounds__(kSyrkThreads, 1)
syrk_tc_kernel(float* G, int R, int t0, int nt, int ncol, const unsigned char* Lp, size_t pstride, int npan,
               int* err, long long first) {
    syrk_tc_body(SyrkOne{G, Lp, pstride, R, t0, nt, ncol, npan, first}, err);
}
__global__ void __launch_bounds__(kSyrkThreads, 1)
syrk_tc_group_kernel(const CholJob* __restrict__ jobs, int njobs, long long total, int* err) {
    syrk_tc_body(SyrkGroup{jobs, njobs, total}, err);
}

// FP32 factorisation in super-panels of kSuperPanels 128-column panels.  Per panel: factor
// the diagonal block, solve and pack the panel below it, and update only the columns of the
// rest of the super-panel (K = 128); after the super-panel, one update of the whole trailing
// matrix with K = 128 kSuperPanels from the panels' packed operands.  The trailing matrix is
// read and written once per super-panel instead of once per panel.
// ws: pivot floors (R floats), the diagonal-block inverses, kSuperPanels packed operands of
// ceil(R / 128) tiles each.  The pivot flag goes to d_flag[0], an expired device wait to d_flag[1].
constexpr int kSuperPanels = 4;
static size_t packed_panel_bytes(int R) { return (size_t)((R + PB - 1) / PB) * kTileBytes; }

static fst_status syrk_tc(float* G, int R, int t0, int nt, int ncol, const unsigned char* Lp, size_t pstride,
                          int npan, int* err, size_t smem, cudaStream_t s, int max_grid = 0, long long first = 0) {
    // tiles [first, end) of the trapezoid of nt tile rows and ncol tile columns
    const long long ntiles = (long long)ncol * (ncol + 1) / 2 + (long long)(nt - ncol) * ncol - first;
    if (ntiles <= 0) return FST_OK;
    const int cap = max_grid > 0 ? max_grid : sm_count();
    const int grid = ntiles < cap ? (int)ntiles : cap;
    syrk_tc_kernel<<<grid, kSyrkThreads, smem, s>>>(G, R, t0, nt, ncol, Lp, pstride, npan, err, first);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

// The side stream of the look-ahead trailing updates, with its events: one set per host
// thread (the factorisations a thread issues run one after another; concurrent refits run on
// different threads), created on first use and destroyed with the thread.
struct LookAhead {
    int device = -1;
    cudaStream_t side = nullptr, panel = nullptr;
    cudaEvent_t chain = nullptr, rest = nullptr, head = nullptr, tail = nullptr;
    void release() {
        if (!side) return;
        cudaStreamSynchronize(side);
        cudaStreamSynchronize(panel);
        cudaStreamDestroy(side);
        cudaStreamDestroy(panel);
        cudaEventDestroy(chain);
        cudaEventDestroy(rest);
        cudaEventDestroy(head);
        cudaEventDestroy(tail);
        side = nullptr;
    }
    ~LookAhead() { release(); }
};
static fst_status look_ahead(LookAhead*& out) {
    thread_local LookAhead la;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    if (la.side && la.device != dev) la.release();
    if (!la.side) {
        FST_CUDA(cudaStreamCreateWithFlags(&la.side, cudaStreamNonBlocking));
        FST_CUDA(cudaStreamCreateWithFlags(&la.panel, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&la.chain, &la.rest, &la.head, &la.tail})
            FST_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        la.device = dev;
    }
    out = &la;
    return FST_OK;
}

// Two levels of look-ahead.  Across super-panels: after a super-panel's panels, the update of
// the next super-panel's columns (all rows below) runs on the caller's stream and the update
// of the rest of the trailing matrix on a side stream, on all but kChainSMs of the SMs, so it
// overlaps the next super-panel's latency-bound panel chain (80 of 152 SMs left to the chain
// measured best: 9.87 ms at R = 13,824 against 10.32 with 24 and 11.05 without); the packed
// panels of consecutive super-panels alternate between two sets, so that update never reads
// panels the next chain rewrites.  Within a super-panel: of panel p's solve and update, only
// the rows and the tile the next panel's diagonal block needs run on the caller's stream; the
// rest runs on a panel stream while the next diagonal block is factored (the diagonal-block
// inverses alternate between two buffers for that), and the next panel's solve waits for it.
// Every tile still receives the same updates in the same order: the factor is bit-identical.
constexpr int kChainSMs = 80;
static fst_status cholesky_lower_tc(float* G, int R, int* d_flag, const float* floors, unsigned char* ws_tail,
                                    cudaStream_t s) {
    float* Dinv2[2] = {reinterpret_cast<float*>(ws_tail), reinterpret_cast<float*>(ws_tail) + 4 * SUB * SUB};
    unsigned char* Lbase = ws_tail + 2 * 4 * SUB * SUB * sizeof(float);
    const size_t pstride = packed_panel_bytes(R);
    const size_t potrf_smem = sizeof(float) * (PB * AS + 4 * SUB * SUB);   // P: FS x PB, then the inverses
    const size_t trsm_smem = sizeof(float) * ((kTrsmRows + PB) * AS + 4 * SUB * (SUB + 4));
    const size_t syrk_smem = kSyrkStages * 2 * kHalfBytes + 1024 + 1024;
    FST_TRY(allow_smem(potrf_inv_kernel, potrf_smem));
    FST_TRY(allow_smem(trsm_pack_kernel, trsm_smem));
    FST_TRY(allow_smem(syrk_tc_kernel, syrk_smem));
    LookAhead* la = nullptr;
    FST_TRY(look_ahead(la));
    bool rest_pending = false;    // a side update was issued (la->rest marks its end)
    bool panel_pending = false;   // panel-stream work was issued (la->tail marks its end)
    auto join_panel = [&]() -> fst_status {
        if (panel_pending) FST_CUDA(cudaStreamWaitEvent(s, la->tail, 0));
        panel_pending = false;
        return FST_OK;
    };
    auto finish = [&]() -> fst_status {
        FST_TRY(join_panel());
        if (rest_pending) FST_CUDA(cudaStreamWaitEvent(s, la->rest, 0));
        return FST_OK;
    };
    constexpr int SBW = kSuperPanels * PB;
    constexpr int kHeadBlocks = PB / kTrsmRows;   // solve blocks of the rows of the next diagonal block
    int pan_index = 0;
    for (int K0 = 0; K0 < R; K0 += SBW) {
        unsigned char* Lp = Lbase + (size_t)((K0 / SBW) & 1) * kSuperPanels * pstride;
        int npan = 0;
        for (int p = 0; p < kSuperPanels; ++p, ++pan_index) {
            const int k0 = K0 + p * PB;
            if (k0 >= R) break;
            const int kb = R - k0 < PB ? R - k0 : PB;
            const int rest = R - k0 - kb;
            float* Dinv = Dinv2[pan_index & 1];
            potrf_inv_kernel<<<1, 512, potrf_smem, s>>>(G, R, k0, kb, d_flag, floors, Dinv, rest > 0 ? 1 : 0);
            FST_CHECK_LAUNCH();
            if (rest <= 0) return finish();
            ++npan;
            const int nt = (rest + PB - 1) / PB;
            unsigned char* Lpp = Lp + (size_t)p * pstride;
            int ncol = (K0 + SBW - (k0 + PB)) / PB;   // columns of the super-panel right of this panel
            if (ncol > nt) ncol = nt;
            // this panel's solve reads rows the previous panel's remaining update writes
            FST_TRY(join_panel());
            const int nblk = (PB / kTrsmRows) * nt;
            if (ncol > 0 && nblk > kHeadBlocks) {
                // the next diagonal block first: its rows of the solve, then its tile of the update
                trsm_pack_kernel<<<kHeadBlocks, 256, trsm_smem, s>>>(G, R, k0, Dinv, Lpp, 0);
                FST_CHECK_LAUNCH();
                FST_TRY(syrk_tc(G, R, k0 + PB, 1, 1, Lpp, pstride, 1, d_flag + 1, syrk_smem, s));
                FST_CUDA(cudaEventRecord(la->head, s));
                FST_CUDA(cudaStreamWaitEvent(la->panel, la->head, 0));
                trsm_pack_kernel<<<nblk - kHeadBlocks, 256, trsm_smem, la->panel>>>(G, R, k0, Dinv, Lpp, kHeadBlocks);
                FST_CHECK_LAUNCH();
                FST_TRY(syrk_tc(G, R, k0 + PB, nt, ncol, Lpp, pstride, 1, d_flag + 1, syrk_smem, la->panel, 0, 1));
                FST_CUDA(cudaEventRecord(la->tail, la->panel));
                panel_pending = true;
            } else {
                trsm_pack_kernel<<<nblk, 256, trsm_smem, s>>>(G, R, k0, Dinv, Lpp, 0);
                FST_CHECK_LAUNCH();
                if (ncol > 0) FST_TRY(syrk_tc(G, R, k0 + PB, nt, ncol, Lpp, pstride, 1, d_flag + 1, syrk_smem, s));
            }
        }
        const int T0 = K0 + npan * PB;
        if (T0 >= R) break;
        const int nt = (R - T0 + PB - 1) / PB;
        const int nnext = nt < kSuperPanels ? nt : kSuperPanels;
        // the previous side update wrote into the next strip's tiles, and read the panel set
        // the chain after this one rewrites: both wait for it here (and the panel stream's last work)
        FST_TRY(finish());
        if (nt > nnext) {
            FST_CUDA(cudaEventRecord(la->chain, s));               // this super-panel's panels are packed
            FST_CUDA(cudaStreamWaitEvent(la->side, la->chain, 0));
            FST_TRY(syrk_tc(G, R, T0 + nnext * PB, nt - nnext, nt - nnext, Lp + (size_t)nnext * kTileBytes, pstride,
                            npan, d_flag + 1, syrk_smem, la->side, std::max(sm_count() - kChainSMs, sm_count() / 4)));
            FST_CUDA(cudaEventRecord(la->rest, la->side));
            rest_pending = true;
        } else {
            rest_pending = false;
        }
        FST_TRY(syrk_tc(G, R, T0, nt, nnext, Lp, pstride, npan, d_flag + 1, syrk_smem, s));
    }
    return finish();
}

// FP32 factorisations of several normal matrices in shared launches (a grouped refit): the
// schedule of cholesky_lower_tc run for all matrices at once, panel by panel, each launch
// doing one step for every matrix that still has it, so a matrix's arithmetic is exactly
// that of its own factorisation.  The whole schedule is built on the host and uploaded
// once (sched); gerr collects expired device waits of every matrix.
fst_status cholesky_lower_group(const std::vector<CholItem>& items, DevBuf& sched, int* gerr, cudaStream_t s) {
    const size_t potrf_smem = sizeof(float) * (PB * AS + 4 * SUB * SUB);
    const size_t trsm_smem = sizeof(float) * ((kTrsmRows + PB) * AS + 4 * SUB * (SUB + 4));
    const size_t syrk_smem = kSyrkStages * 2 * kHalfBytes + 1024 + 1024;
    FST_TRY(allow_smem(potrf_inv_group_kernel, potrf_smem));
    FST_TRY(allow_smem(trsm_pack_group_kernel, trsm_smem));
    FST_TRY(allow_smem(syrk_tc_group_kernel, syrk_smem));
    const int n = (int)items.size();
    std::vector<const float*> floors(n);
    std::vector<float*> dinv(n);
    std::vector<unsigned char*> lp(n);
    std::vector<size_t> pstride(n);
    int maxR = 0;
    for (int i = 0; i < n; ++i) {
        const int R = items[i].R;
        const size_t floor_bytes = ((size_t)R * sizeof(float) + 255) / 256 * 256;
        const size_t tail = 4 * SUB * SUB * sizeof(float) + kSuperPanels * packed_panel_bytes(R);
        FST_TRY(items[i].ws->ensure(floor_bytes + tail));
        float* fl = items[i].ws->as<float>();
        pivot_floor_kernel<float><<<(R + 255) / 256 < 1024 ? (R + 255) / 256 : 1024, 256, 0, s>>>(items[i].G, R, fl);
        FST_CHECK_LAUNCH();
        floors[i] = fl;
        dinv[i] = reinterpret_cast<float*>(items[i].ws->as<unsigned char>() + floor_bytes);
        lp[i] = items[i].ws->as<unsigned char>() + floor_bytes + 4 * SUB * SUB * sizeof(float);
        pstride[i] = packed_panel_bytes(R);
        maxR = std::max(maxR, R);
    }
    // the schedule: launches of kind 0 (diagonal blocks), 1 (panel solves), 2 (updates)
    struct Launch {
        int kind, off, njobs;
        long long total;
    };
    std::vector<CholJob> jobs;
    std::vector<Launch> launches;
    std::vector<char> done(n, 0);
    std::vector<int> npan(n, 0);
    auto job = [&](int i) {
        CholJob j{};
        j.G = items[i].G;
        j.floors = floors[i];
        j.Dinv = dinv[i];
        j.pstride = pstride[i];
        j.flag = items[i].flag;
        j.R = items[i].R;
        return j;
    };
    constexpr int SBW = kSuperPanels * PB;
    for (int K0 = 0; K0 < maxR; K0 += SBW) {
        std::fill(npan.begin(), npan.end(), 0);
        for (int p = 0; p < kSuperPanels; ++p) {
            const int k0 = K0 + p * PB;
            Launch lf{0, (int)jobs.size(), 0, 0}, ls{1, 0, 0, 0}, lu{2, 0, 0, 0};
            std::vector<CholJob> tj, uj;
            for (int i = 0; i < n; ++i) {
                const int R = items[i].R;
                if (done[i] || k0 >= R) continue;
                const int kb = R - k0 < PB ? R - k0 : PB;
                const int rest = R - k0 - kb;
                CholJob f = job(i);
                f.k0 = k0;
                f.kb = kb;
                f.want_inv = rest > 0 ? 1 : 0;
                f.first = lf.njobs;
                jobs.push_back(f);
                ++lf.njobs;
                if (rest <= 0) {
                    done[i] = 1;
                    continue;
                }
                ++npan[i];
                const int nt = (rest + PB - 1) / PB;
                CholJob t = job(i);
                t.k0 = k0;
                t.Lp = lp[i] + (size_t)p * pstride[i];
                t.first = ls.total;
                ls.total += (long long)(PB / kTrsmRows) * nt;
                tj.push_back(t);
                int ncol = (K0 + SBW - (k0 + PB)) / PB;
                if (ncol > nt) ncol = nt;
                if (ncol > 0) {
                    CholJob u = t;
                    u.t0 = k0 + PB;
                    u.nt = nt;
                    u.ncol = ncol;
                    u.npan = 1;
                    u.first = lu.total;
                    lu.total += (long long)ncol * (ncol + 1) / 2 + (long long)(nt - ncol) * ncol;
                    uj.push_back(u);
                }
            }
            lf.total = lf.njobs;
            if (lf.njobs) launches.push_back(lf);
            if (!tj.empty()) {
                ls.off = (int)jobs.size();
                ls.njobs = (int)tj.size();
                jobs.insert(jobs.end(), tj.begin(), tj.end());
                launches.push_back(ls);
            }
            if (!uj.empty()) {
                lu.off = (int)jobs.size();
                lu.njobs = (int)uj.size();
                jobs.insert(jobs.end(), uj.begin(), uj.end());
                launches.push_back(lu);
            }
        }
        Launch lu{2, (int)jobs.size(), 0, 0};
        for (int i = 0; i < n; ++i) {
            const int R = items[i].R;
            if (done[i] || npan[i] == 0) continue;
            const int T0 = K0 + npan[i] * PB;
            if (T0 >= R) continue;
            CholJob u = job(i);
            u.Lp = lp[i];
            u.t0 = T0;
            u.nt = (R - T0 + PB - 1) / PB;
            u.ncol = u.nt;
            u.npan = npan[i];
            u.first = lu.total;
            lu.total += (long long)u.nt * (u.nt + 1) / 2;
            jobs.push_back(u);
            ++lu.njobs;
        }
        if (lu.njobs) launches.push_back(lu);
    }
    if (jobs.empty()) return FST_OK;
    FST_TRY(sched.ensure(sizeof(CholJob) * jobs.size()));
    CholJob* dj = sched.as<CholJob>();
    FST_CUDA(cudaMemcpyAsync(dj, jobs.data(), sizeof(CholJob) * jobs.size(), cudaMemcpyHostToDevice, s));
    for (const Launch& L : launches) {
        const CholJob* j = dj + L.off;
        if (L.kind == 0) {
            potrf_inv_group_kernel<<<L.njobs, 512, potrf_smem, s>>>(j);
        } else if (L.kind == 1) {
            trsm_pack_group_kernel<<<(unsigned)L.total, 256, trsm_smem, s>>>(j, L.njobs);
        } else {
            const int grid = L.total < sm_count() ? (int)L.total : sm_count();
            syrk_tc_group_kernel<<<grid, kSyrkThreads, syrk_smem, s>>>(j, L.njobs, L.total, gerr);
        }
        FST_CHECK_LAUNCH();
    }
    // the upload's host buffer must outlive the copy: wait for it before `jobs` is freed
    FST_CUDA(cudaStreamSynchronize(s));
    return FST_OK;
}

template <typename T>
fst_status cholesky_lower(T* G, int R, int* d_flag, DevBuf& ws, cudaStream_t s) {
    // ws: per-column pivot floors, then (FP32) the panel scratch of the tensor-core path
    const size_t floor_bytes = ((size_t)R * sizeof(T) + 255) / 256 * 256;
    const size_t tail = sizeof(T) == 4 ? 2 * 4 * SUB * SUB * sizeof(float) + 2 * kSuperPanels * packed_panel_bytes(R) : 0;
    FST_TRY(ws.ensure(floor_bytes + tail));
    T* floors = ws.as<T>();
    pivot_floor_kernel<T><<<(R + 255) / 256 < 1024 ? (R + 255) / 256 : 1024, 256, 0, s>>>(G, R, floors);
    FST_CHECK_LAUNCH();
    if (sizeof(T) == 4)
        return cholesky_lower_tc(reinterpret_cast<float*>(G), R, d_flag, reinterpret_cast<const float*>(floors),
                                 ws.as<unsigned char>() + floor_bytes, s);
    const size_t trsm_smem = 2 * NB * (NB + 1) * sizeof(T);
    FST_TRY(allow_smem(trsm_panel_kernel<T>, trsm_smem));
    for (int k0 = 0; k0 < R; k0 += NB) {
        const int kb = R - k0 < NB ? R - k0 : NB;
        potrf_diag_kernel<T><<<1, 256, 0, s>>>(G, R, k0, kb, d_flag, floors);
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

// The link matrices of the triangular solves: the last dependency of block row i folded
// into its diagonal solve, Kf_i = L_ii^-1 L_{i,i-1} (forward) and
// Kb_i = L_ii^-T L_{i+1,i}^T (backward), so y_i = L_ii^-1 (b_i - sum_{j<i-1} L_ij y_j) - Kf_i y_{i-1}
// and the chain from one block row to the next is one 64 x 64 product.
template <typename T>
__global__ void __launch_bounds__(256) link_blocks_kernel(const T* __restrict__ L, int R, const T* __restrict__ Linv,
                                                          T* __restrict__ Kf, T* __restrict__ Kb) {
    __shared__ T li[NB][NB + 1];
    __shared__ T tl[NB][NB + 1];
    const int i = blockIdx.x, nblk = gridDim.x, k0 = i * NB, tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += 256) li[e / NB][e % NB] = Linv[(size_t)i * NB * NB + e];
    if (i >= 1) {
        // tl[k][c] = L[k0 + k][(i - 1) NB + c]
        for (int e = tid; e < NB * NB; e += 256) {
            const int k = e / NB, c = e % NB;
            tl[k][c] = k0 + k < R ? L[(size_t)(k0 + k) * R + (i - 1) * NB + c] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < NB * NB; e += 256) {
            const int r = e / NB, c = e % NB;
            T acc = T(0);
            for (int k = 0; k < NB; ++k) acc += li[r][k] * tl[k][c];
            Kf[(size_t)i * NB * NB + e] = acc;
        }
        __syncthreads();
    }
    if (i + 1 < nblk) {
        // tl[c][k] = L[(i + 1) NB + c][k0 + k]
        for (int e = tid; e < NB * NB; e += 256) {
            const int c = e / NB, k = e % NB;
            const int row = (i + 1) * NB + c;
            tl[c][k] = row < R ? L[(size_t)row * R + k0 + k] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < NB * NB; e += 256) {
            const int r = e / NB, c = e % NB;
            T acc = T(0);
            for (int k = 0; k < NB; ++k) acc += li[k][r] * tl[c][k];
            Kb[(size_t)i * NB * NB + e] = acc;
        }
    }
}

// One direction of x <- L^-T L^-1 x in a single launch.  Block row i (64 rows) is solved
// by one block: forward, y_i = Linv_ii (b_i - sum_{j<i} L_ij y_j); backward (TRANS),
// x_i = Linv_ii^T (y_i - sum_{j>i} L_ji^T x_j).  Blocks take block rows in solve order
// from a ticket counter, so a block only waits for rows already taken by running blocks
// (no deadlock whatever the residency).  The output vector is filled with an all-ones bit
// pattern (a NaN that arithmetic never produces) before the launch; a value is published
// by one relaxed store and a consumer spins on exactly the values it needs until they
// differ from that pattern, so there are no flags, fences or block-wide barriers on the
// chain.  Every spin is bounded; on expiry the block records an error in sync[0] and goes
// on with what it read (the rows after it then finish without waiting out their own
// limits).  sync: [0] error word, [1] ticket (zeroed before the launch).
constexpr long long kSolveWaitLimit = 2000000000LL;
// A shorter budget set by fst_set_wait_limit (0: kSolveWaitLimit), read once per block.
__device__ long long g_solve_wait_limit = 0;

__device__ __forceinline__ bool unpublished(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ bool unpublished(double v) {
    return (unsigned long long)__double_as_longlong(v) == 0xffffffffffffffffull;
}
__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
// a computed value never takes the unpublished pattern
template <typename T>
__device__ __forceinline__ T publishable(T v) {
    return unpublished(v) ? (T)NAN : v;
}

// wait for p to be published (bounded by `limit` clock cycles); returns the value
template <typename T>
__device__ __forceinline__ T wait_value(const T* p, int* err, long long limit) {
    T v = ld_relaxed(p);
    if (!unpublished(v)) return v;
    const long long t0 = clock64();
    while (unpublished(v = ld_relaxed(p))) {
        if (clock64() - t0 > limit) {
            atomicOr(err, 1);
            return T(0);
        }
    }
    return v;
}

// M is L (forward) or L^T (backward, TRANS), both row-major: block row i reads the tiles
// M[i-block][j-block] for j < i (forward) or j > i (backward) along its own rows.
template <typename T, bool TRANS>
__device__ __forceinline__ void trsv_body(const T* __restrict__ M, const T* __restrict__ Linv,
                                          const T* __restrict__ K, int R, int nblk, const T* bin, T* out,
                                          int* sync, int i, long long limit) {
    __shared__ T lis[NB][NB + 1];   // Linv of the diagonal block
    __shared__ T red[8][NB];
    __shared__ T vs[NB];
    __shared__ T xl[NB];            // the values of the last dependency
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = i * NB, kb = R - k0 < NB ? R - k0 : NB;
    {
        const T* Li = Linv + (size_t)i * NB * NB;
        for (int e = tid; e < NB * NB; e += 256) lis[e / NB][e % NB] = Li[e];
    }
    const int ntiles = TRANS ? nblk - 1 - i : i;   // block rows this one depends on
    // the link matrix (thread (r, q): row r, columns 16q .. 16q + 15), loaded off the chain
    const int lr = tid >> 2, lq = tid & 3;
    T kr[16];
    if (ntiles > 0) {
        const T* Ki = K + (size_t)i * NB * NB + lr * NB + 16 * lq;
#pragma unroll
        for (int u = 0; u < 16; ++u) kr[u] = Ki[u];
    }
    // tile mapping (coalesced along the rows of M): warp w owns rows 8w .. 8w+7 of the
    // block row, lane l the columns l and l + 32 of the tile; every dependency but the
    // last is summed here
    T acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = T(0);
    const int nsum = ntiles - 1;
    auto load_tile = [&](int n, T (&lv)[16]) {
        const int j0 = (TRANS ? nblk - 1 - n : n) * NB;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int row = k0 + warp * 8 + u;
            const bool rok = row < R;
            lv[2 * u] = (rok && j0 + lane < R) ? M[(size_t)row * R + j0 + lane] : T(0);
            lv[2 * u + 1] = (rok && j0 + lane + 32 < R) ? M[(size_t)row * R + j0 + lane + 32] : T(0);
        }
    };
    // a ring of kTrsvDepth tiles in registers: the loads of the next kTrsvDepth - 1 tiles fly
    // while one is summed (late block rows stream many tiles)
    constexpr int kTrsvDepth = sizeof(T) == 4 ? 8 : 4;
    T ring[kTrsvDepth][16];
#pragma unroll
    for (int d = 0; d + 1 < kTrsvDepth; ++d)
        if (d < nsum) load_tile(d, ring[d]);
    for (int n0 = 0; n0 < nsum; n0 += kTrsvDepth) {
#pragma unroll
        for (int d = 0; d < kTrsvDepth; ++d) {
            const int n = n0 + d;
            if (n < nsum) {
                if (n + kTrsvDepth - 1 < nsum) load_tile(n + kTrsvDepth - 1, ring[(d + kTrsvDepth - 1) % kTrsvDepth]);
                const int j0 = (TRANS ? nblk - 1 - n : n) * NB;
                const T* xj = out + j0;
                // both values in one batch of L2 loads; spin only on one not yet published
                T x0 = j0 + lane < R ? __ldcg(xj + lane) : T(0);
                T x1 = j0 + lane + 32 < R ? __ldcg(xj + lane + 32) : T(0);
                if (unpublished(x0)) x0 = wait_value(xj + lane, sync, limit);
                if (unpublished(x1)) x1 = wait_value(xj + lane + 32, sync, limit);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += ring[d][2 * u] * x0 + ring[d][2 * u + 1] * x1;
            }
        }
    }
    // row sums across the warp
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        T v = acc[u];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[0][warp * 8 + u] = v;
    }
    __syncthreads();
    if (tid < NB) vs[tid] = tid < kb ? bin[k0 + tid] - red[0][tid] : T(0);
    __syncthreads();
    // c_i = Linv_ii v (forward) or Linv_ii^T v (backward): thread (q, c) sums 16 terms
    {
        const int q = tid >> 6, c = tid & 63;
        T s2 = T(0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int a = q * 16 + u;
            s2 += (TRANS ? lis[a][c] : lis[c][a]) * vs[a];
        }
        red[4 + q][c] = s2;
    }
    __syncthreads();
    if (ntiles == 0) {
        if (tid < kb) {
            const T v = (red[4][tid] + red[5][tid]) + (red[6][tid] + red[7][tid]);
            st_relaxed(out + k0 + tid, publishable(v));
        }
        return;
    }
    // the last dependency: out_i = c_i - K_i x_last
    if (warp == 0) {
        const int j0 = (TRANS ? i + 1 : i - 1) * NB;
        const T* xj = out + j0;
        T x0 = j0 + lane < R ? __ldcg(xj + lane) : T(0);
        T x1 = j0 + lane + 32 < R ? __ldcg(xj + lane + 32) : T(0);
        if (unpublished(x0)) x0 = wait_value(xj + lane, sync, limit);
        if (unpublished(x1)) x1 = wait_value(xj + lane + 32, sync, limit);
        xl[lane] = x0;
        xl[lane + 32] = x1;
    }
    __syncthreads();
    T s3 = T(0);
#pragma unroll
    for (int u = 0; u < 16; ++u) s3 += kr[u] * xl[16 * lq + u];
    s3 += __shfl_xor_sync(0xffffffffu, s3, 1);
    s3 += __shfl_xor_sync(0xffffffffu, s3, 2);
    if (lq == 0 && lr < kb) {
        const T c = (red[4][lr] + red[5][lr]) + (red[6][lr] + red[7][lr]);
        st_relaxed(out + k0 + lr, publishable(c - s3));
    }
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) trsv_kernel(const T* __restrict__ M, const T* __restrict__ Linv,
                                                   const T* __restrict__ K, int R, int nblk, const T* bin, T* out,
                                                   int* sync, const int* stop) {
    if (stop && *stop) return;   // the caller's iteration has already stopped (no block waits then)
    const long long limit = g_solve_wait_limit > 0 ? g_solve_wait_limit : kSolveWaitLimit;
    __shared__ int s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(&sync[1], 1);
    __syncthreads();
    const int t = s_ticket;
    trsv_body<T, TRANS>(M, Linv, K, R, nblk, bin, out, sync, TRANS ? nblk - 1 - t : t, limit);
}

// The solves of several factored matrices in one launch per direction (a grouped refit).
// Tickets are handed out step by step across the matrices: ticket t is block row step
// tmap[t] & 0xffff (in solve order) of matrix tmap[t] >> 16, and every ticket of an earlier
// step precedes it, so a block again waits only for rows already taken.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) trsv_group_kernel(const SolveJob* __restrict__ jobs,
                                                         const int* __restrict__ tmap, int* sync) {
    const long long limit = g_solve_wait_limit > 0 ? g_solve_wait_limit : kSolveWaitLimit;
    __shared__ int s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(&sync[1], 1);
    __syncthreads();
    const int code = tmap[s_ticket];
    const SolveJob& J = jobs[code >> 16];
    if (J.stop && *J.stop) return;   // this matrix's iteration has stopped: nothing waits on it
    const int step = code & 0xffff;
    const T* Li = static_cast<const T*>(J.Linv);
    const size_t nb2 = (size_t)J.nblk * NB * NB;
    if (TRANS)
        trsv_body<T, true>(static_cast<const T*>(J.LT), Li, Li + 2 * nb2, J.R, J.nblk, static_cast<const T*>(J.y),
                           static_cast<T*>(J.x), sync, J.nblk - 1 - step, limit);
    else
        trsv_body<T, false>(static_cast<const T*>(J.L), Li, Li + nb2, J.R, J.nblk, static_cast<const T*>(J.x),
                            static_cast<T*>(J.y), sync, step, limit);
}

// fills the solve's output vector of every matrix with the unpublished pattern (which 0: y,
// 1: x) and, from the first block, zeroes the ticket
template <typename T>
__global__ void solve_fill_group_kernel(const SolveJob* __restrict__ jobs, int which, int* sync) {
    const SolveJob& J = jobs[blockIdx.y];
    T* v = static_cast<T*>(which ? J.x : J.y);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.R; i += gridDim.x * blockDim.x) {
        if (sizeof(T) == 4)
            reinterpret_cast<unsigned int*>(v)[i] = 0xffffffffu;
        else
            reinterpret_cast<unsigned long long*>(v)[i] = ~0ull;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) sync[1] = 0;
}

// LT = L^T on the lower triangle's 32 x 32 tiles (the strict upper blocks of LT that the
// backward solve reads are all written).
template <typename T>
__global__ void transpose_lower_kernel(const T* __restrict__ L, int R, T* __restrict__ LT) {
    __shared__ T tl[32][33];
    const long long b = blockIdx.x;
    int ti = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while ((long long)ti * (ti + 1) / 2 > b) --ti;
    const int tj = (int)(b - (long long)ti * (ti + 1) / 2);
    const int r0 = ti * 32, c0 = tj * 32, x = threadIdx.x;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int row = r0 + y, col = c0 + x;
        tl[y][x] = (row < R && col < R) ? L[(size_t)row * R + col] : T(0);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int row = c0 + y, col = r0 + x;
        if (row < R && col < R) LT[(size_t)row * R + col] = tl[x][y];
    }
}

template <typename T>
fst_status chol_transpose(const T* L, int R, T* LT, cudaStream_t s) {
    const long long nt = (R + 31) / 32;
    transpose_lower_kernel<T><<<(unsigned)(nt * (nt + 1) / 2), dim3(32, 8), 0, s>>>(L, R, LT);
    FST_CHECK_LAUNCH();
    return FST_OK;
}
template fst_status chol_transpose<float>(const float*, int, float*, cudaStream_t);
template fst_status chol_transpose<double>(const double*, int, double*, cudaStream_t);

template <typename T>
fst_status chol_invert_diag(const T* L, int R, T* Linv, cudaStream_t s) {
    const int nblk = (R + NB - 1) / NB;
    invert_diag_kernel<T><<<nblk, NB, 0, s>>>(L, R, Linv);
    FST_CHECK_LAUNCH();
    link_blocks_kernel<T><<<nblk, 256, 0, s>>>(L, R, Linv, Linv + (size_t)nblk * NB * NB,
                                                 Linv + 2 * (size_t)nblk * NB * NB);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

// x <- L^-T L^-1 x (x and y: R values of T; y is scratch; LT = L^T; sync: 2 ints, the first
// the error word, left as it is).  The output of each direction is filled with the all-ones
// pattern first (both memsets and both kernels are captured by chol_solve_graph).
template <typename T>
fst_status chol_solve(const T* L, const T* LT, const T* Linv, int R, T* x, T* y, int* sync, cudaStream_t s,
                      const int* stop) {
    const int nblk = (R + NB - 1) / NB;
    FST_CUDA(cudaMemsetAsync(sync + 1, 0, sizeof(int), s));
    FST_CUDA(cudaMemsetAsync(y, 0xff, sizeof(T) * (size_t)R, s));
    const T* Kf = Linv + (size_t)nblk * NB * NB;
    const T* Kb = Linv + 2 * (size_t)nblk * NB * NB;
    trsv_kernel<T, false><<<nblk, 256, 0, s>>>(L, Linv, Kf, R, nblk, x, y, sync, stop);
    FST_CHECK_LAUNCH();
    FST_CUDA(cudaMemsetAsync(sync + 1, 0, sizeof(int), s));
    FST_CUDA(cudaMemsetAsync(x, 0xff, sizeof(T) * (size_t)R, s));
    trsv_kernel<T, true><<<nblk, 256, 0, s>>>(LT, Linv, Kb, R, nblk, y, x, sync, stop);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

// x <- (L L^T)^-1 x for every job of a grouped refit (device job array, ticket map of
// `tickets` entries built by solve_tickets); sync: [0] error word, [1] ticket.
template <typename T>
fst_status chol_solve_group(const SolveJob* jobs, int njobs, int maxR, const int* tmap, int tickets, int* sync,
                            cudaStream_t s) {
    const dim3 fg((unsigned)std::min((maxR + 255) / 256, 64), (unsigned)njobs);
    solve_fill_group_kernel<T><<<fg, 256, 0, s>>>(jobs, 0, sync);
    FST_CHECK_LAUNCH();
    trsv_group_kernel<T, false><<<tickets, 256, 0, s>>>(jobs, tmap, sync);
    FST_CHECK_LAUNCH();
    solve_fill_group_kernel<T><<<fg, 256, 0, s>>>(jobs, 1, sync);
    FST_CHECK_LAUNCH();
    trsv_group_kernel<T, true><<<tickets, 256, 0, s>>>(jobs, tmap, sync);
    FST_CHECK_LAUNCH();
    return FST_OK;
}
template fst_status chol_solve_group<float>(const SolveJob*, int, int, const int*, int, int*, cudaStream_t);
template fst_status chol_solve_group<double>(const SolveJob*, int, int, const int*, int, int*, cudaStream_t);

// The ticket map of a grouped solve: step by step (block row in solve order), every matrix
// that has that many block rows.
std::vector<int> solve_tickets(const std::vector<int>& R) {
    int maxb = 0;
    for (int r : R) maxb = std::max(maxb, (r + NB - 1) / NB);
    std::vector<int> t;
    for (int b = 0; b < maxb; ++b)
        for (size_t j = 0; j < R.size(); ++j)
            if (b < (R[j] + NB - 1) / NB) t.push_back((int)(j << 16) | b);
    return t;
}

template fst_status cholesky_lower<float>(float*, int, int*, DevBuf&, cudaStream_t);
template fst_status cholesky_lower<double>(double*, int, int*, DevBuf&, cudaStream_t);
template <typename T>
fst_status chol_solve_graph(SolveGraph& g, const T* L, const T* LT, const T* Linv, int R, T* x, T* y,
                            cudaStream_t s, const int* stop) {
    if (!g.exec || g.L != L || g.LT != LT || g.Linv != Linv || g.x != x || g.R != R || g.elem != (int)sizeof(T) ||
        g.stop != stop) {
        if (g.exec) {
            FST_CUDA(cudaStreamSynchronize(s));
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        if (!g.cap) FST_CUDA(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
        FST_TRY(g.sync.ensure(4 * sizeof(int)));
        FST_CUDA(cudaMemsetAsync(g.sync.ptr, 0, sizeof(int), s));
        FST_CUDA(cudaStreamSynchronize(s));
        FST_CUDA(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = fst_kernel_launches();
        fst_status st = chol_solve<T>(L, LT, Linv, R, x, y, g.sync.as<int>(), g.cap, stop);
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
        g.LT = LT;
        g.Linv = Linv;
        g.x = x;
        g.R = R;
        g.elem = (int)sizeof(T);
        g.stop = stop;
    }
    FST_CUDA(cudaGraphLaunch(g.exec, s));
    count_launches(g.nodes);
    return FST_OK;
}

template fst_status chol_solve_graph<float>(SolveGraph&, const float*, const float*, const float*, int, float*,
                                            float*, cudaStream_t, const int*);
template fst_status chol_solve_graph<double>(SolveGraph&, const double*, const double*, const double*, int, double*,
                                             double*, cudaStream_t, const int*);

template fst_status chol_invert_diag<float>(const float*, int, float*, cudaStream_t);
template fst_status chol_invert_diag<double>(const double*, int, double*, cudaStream_t);
template fst_status chol_solve<float>(const float*, const float*, const float*, int, float*, float*, int*, cudaStream_t,
                                      const int*);
template fst_status chol_solve<double>(const double*, const double*, const double*, int, double*, double*, int*,
                                       cudaStream_t, const int*);

}  // namespace fst

extern "C" fst_status fst_cholesky_f32(float* G, int32_t R, fst_stream stream) {
    using namespace fst;
    FST_REQUIRE(G != nullptr && R > 0, "G is NULL or R <= 0");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(pointer_device(G) == dev, "G must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf flag, ws;
    struct Release {
        DevBuf *a, *b;
        ~Release() {
            a->release();
            b->release();
        }
    } rel{&flag, &ws};
    FST_TRY(flag.ensure(4 * sizeof(int)));
    FST_CUDA(cudaMemsetAsync(flag.ptr, 0, 2 * sizeof(int), s));
    FST_TRY(cholesky_lower<float>(G, R, flag.as<int>(), ws, s));
    int h[2] = {0, 0};
    FST_CUDA(cudaMemcpyAsync(h, flag.ptr, sizeof h, cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    if (h[1]) {
        set_error("Cholesky: a bounded device wait expired (code %d)", h[1]);
        return FST_ETIMEOUT;
    }
    if (h[0]) {
        set_error("matrix is not positive definite in FP32 (pivot below 16 eps max diag)");
        return FST_ENOTSPD;
    }
    return FST_OK;
}

extern "C" fst_status fst_set_wait_limit(int64_t cycles) {
    using namespace fst;
    FST_REQUIRE(cycles >= 0, "cycles < 0");
    const long long v = (long long)cycles;
    FST_CUDA(cudaMemcpyToSymbol(g_solve_wait_limit, &v, sizeof v));
    return FST_OK;
}
