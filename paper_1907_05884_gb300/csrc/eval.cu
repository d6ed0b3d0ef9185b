// eval.cu -- evaluation of a functional sparse Tucker model on the CUDA cores
// (FP64 and FP32), and the fst_eval / fst_eval_f64 entry points.
//
// u~(y) = sum_{j1 j2 j3} alpha_{j1 j2 j3} w1_{j1}(y1) w2_{j2}(y2) w3_{j3}(y3)   (Sec. 2, eq. func_tuck)
// w^(k)_j(y) = sum_n W^k_{n,j} sqrt(2n+1) L_n(t(y))                              (Sec. 2, eq. sparse)
//
// One thread per point (PPT points per thread), persistent grid.  Per block the
// shared memory holds the Legendre recurrence coefficients, the dense coefficient
// matrices (rows n < p_eff, zero rows skipped) and the core padded along j3 to RM.
// Per thread, w1 and w2 go to a private column of shared memory and w3 stays in
// registers; the core is then contracted as sum_i w1_i sum_j w2_j (alpha_ij. . w3).
#include "basis.cuh"

namespace fst {

template <typename T, int RM>
static size_t eval_smem_bytes(const EvalArgs<T>& a, int B, int PPT) {
    size_t e = 2 * (size_t)a.pm + (size_t)(a.pe[0] + a.pe[1] + a.pe[2]) * RM +
               (size_t)a.r[0] * a.r[1] * RM + 2 * (size_t)RM * B * PPT;
    return e * sizeof(T) + 3 * (size_t)a.pm;
}

template <typename T, int RM, int PPT>
__global__ void __launch_bounds__(128) eval_simt_kernel(const EvalArgs<T> a, const T* __restrict__ xyz,
                                                        int64_t n, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = blockDim.x, tid = threadIdx.x;
    const int BP = B * PPT;
    const int r1 = a.r[0], r2 = a.r[1], r3 = a.r[2];
    T* ra = reinterpret_cast<T*>(smem);
    T* rb = ra + a.pm;
    T* Ws[3];
    Ws[0] = rb + a.pm;
    Ws[1] = Ws[0] + a.pe[0] * RM;
    Ws[2] = Ws[1] + a.pe[1] * RM;
    T* As = Ws[2] + a.pe[2] * RM;
    T* u1s = As + r1 * r2 * RM;
    T* u2s = u1s + RM * BP;
    uint8_t* mk = reinterpret_cast<uint8_t*>(u2s + RM * BP);

    for (int i = tid; i < a.pm; i += B) {
        ra[i] = T(2 * i + 1) / T(i + 1);
        rb[i] = T(i) / T(i + 1);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int rk = a.r[k];
        for (int e = tid; e < a.pe[k] * RM; e += B) {
            const int nn = e / RM, j = e - nn * RM;
            Ws[k][e] = j < rk ? a.W[k][nn * rk + j] : T(0);
        }
        for (int e = tid; e < a.pm; e += B) mk[k * a.pm + e] = e < a.pe[k] ? a.mask[k][e] : 0;
    }
    for (int e = tid; e < r1 * r2 * RM; e += B) {
        const int ij = e / RM, kk = e - ij * RM;
        As[e] = kk < r3 ? a.alpha[ij * r3 + kk] : T(0);
    }
    __syncthreads();

    const int64_t stride = (int64_t)gridDim.x * BP;
    for (int64_t base = (int64_t)blockIdx.x * BP; base < n; base += stride) {
        T t[3][PPT], yv[3][PPT];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
            const int64_t q = base + pp * B + tid;
            const bool ok = q < n;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T y = ok ? xyz[k * n + q] : T(0);
                yv[k][pp] = y;
                t[k][pp] = fma(y, a.sc[k], a.of[k]);
            }
        }
        T acc[PPT][RM];
        factor_values<T, RM, PPT>(t[0], Ws[0], mk, a.pe[0], ra, rb, acc);
        piecewise_values<T, RM, PPT>(yv[0], t[0], a, 0, acc);
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp)
#pragma unroll
            for (int j = 0; j < RM; ++j) u1s[j * BP + pp * B + tid] = acc[pp][j];
        factor_values<T, RM, PPT>(t[1], Ws[1], mk + a.pm, a.pe[1], ra, rb, acc);
        piecewise_values<T, RM, PPT>(yv[1], t[1], a, 1, acc);
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp)
#pragma unroll
            for (int j = 0; j < RM; ++j) u2s[j * BP + pp * B + tid] = acc[pp][j];
        factor_values<T, RM, PPT>(t[2], Ws[2], mk + 2 * a.pm, a.pe[2], ra, rb, acc);  // w3 in registers
        piecewise_values<T, RM, PPT>(yv[2], t[2], a, 2, acc);

        T f[PPT];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) f[pp] = T(0);
        for (int i = 0; i < r1; ++i) {
            T s[PPT];
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) s[pp] = T(0);
            for (int j = 0; j < r2; ++j) {
                const T* arow = As + (i * r2 + j) * RM;
                T t0[PPT], t1[PPT];
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) { t0[pp] = T(0); t1[pp] = T(0); }
#pragma unroll
                for (int k = 0; k < RM; k += 4) {
                    T a0, a1, a2, a3;
                    load4(arow + k, a0, a1, a2, a3);
#pragma unroll
                    for (int pp = 0; pp < PPT; ++pp) {
                        t0[pp] = fma(a0, acc[pp][k], t0[pp]);
                        t1[pp] = fma(a1, acc[pp][k + 1], t1[pp]);
                        t0[pp] = fma(a2, acc[pp][k + 2], t0[pp]);
                        t1[pp] = fma(a3, acc[pp][k + 3], t1[pp]);
                    }
                }
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp)
                    s[pp] = fma(t0[pp] + t1[pp], u2s[j * BP + pp * B + tid], s[pp]);
            }
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) f[pp] = fma(s[pp], u1s[i * BP + pp * B + tid], f[pp]);
        }
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
            const int64_t q = base + pp * B + tid;
            if (q < n) out[q] = f[pp];
        }
    }
}

template <typename T, int RM, int PPT>
static fst_status launch_rm(const EvalArgs<T>& a, const T* xyz, int64_t n, T* out, cudaStream_t s) {
    auto kern = eval_simt_kernel<T, RM, PPT>;
    int B = 128;
    size_t smem = eval_smem_bytes<T, RM>(a, B, PPT);
    while (smem > 227 * 1024 && B > 32) {
        B /= 2;
        smem = eval_smem_bytes<T, RM>(a, B, PPT);
    }
    if (smem > 227 * 1024) {
        set_error("model too large for the CUDA-core evaluator (%zu bytes of shared memory)", smem);
        return FST_EUNSUPPORTED;
    }
    FST_TRY(allow_smem(kern, smem));
    int per_sm = 0;
    FST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t need = (n + (int64_t)B * PPT - 1) / ((int64_t)B * PPT);
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (need < grid) grid = need;
    kern<<<(unsigned)grid, B, smem, s>>>(a, xyz, n, out);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <typename T>
fst_status eval_simt_launch(const fst_model* m, const T* xyz, int64_t n, T* out, cudaStream_t s) {
    if (n == 0) return FST_OK;
    EvalArgs<T> a = make_args<T>(m);
    bind(a, m);
    int rmax = m->r[0];
    for (int k = 1; k < 3; ++k) rmax = m->r[k] > rmax ? m->r[k] : rmax;
    constexpr int PPT = sizeof(T) == 4 ? 2 : 1;
    if (rmax <= 8) return launch_rm<T, 8, PPT>(a, xyz, n, out, s);
    if (rmax <= 16) return launch_rm<T, 16, PPT>(a, xyz, n, out, s);
    if (rmax <= 24) return launch_rm<T, 24, PPT>(a, xyz, n, out, s);
    return launch_rm<T, 32, PPT>(a, xyz, n, out, s);
}

template fst_status eval_simt_launch<float>(const fst_model*, const float*, int64_t, float*, cudaStream_t);
template fst_status eval_simt_launch<double>(const fst_model*, const double*, int64_t, double*, cudaStream_t);

static fst_status check_eval_args(const fst_model* m, const void* xyz, int64_t n, const void* out) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    FST_REQUIRE(n >= 0, "n = %lld is negative", (long long)n);
    if (n == 0) return FST_OK;
    FST_REQUIRE(xyz != nullptr && out != nullptr, "xyz or out is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == m->device, "model lives on device %d, current device is %d", m->device, dev);
    FST_REQUIRE(pointer_device(xyz) == dev && pointer_device(out) == dev,
                "xyz and out must be device memory of device %d", dev);
    return FST_OK;
}

}  // namespace fst

using namespace fst;

extern "C" fst_status fst_eval(const fst_model* m, const float* xyz, int64_t n, float* out, fst_prec prec,
                               fst_stream stream) {
    FST_TRY(check_eval_args(m, xyz, n, out));
    if (n == 0) return FST_OK;
    switch (prec) {
        case FST_FP32: return eval_simt_launch<float>(m, xyz, n, out, (cudaStream_t)stream);
        case FST_TF32:
        case FST_BF16:
        case FST_BF16X3:
            return eval_tc_launch(const_cast<fst_model*>(m), xyz, n, out, prec, (cudaStream_t)stream);
        default:
            set_error("fst_eval takes FST_FP32, FST_TF32, FST_BF16 or FST_BF16X3; use fst_eval_f64 for FP64");
            return FST_EINVAL;
    }
}

extern "C" fst_status fst_eval_f64(const fst_model* m, const double* xyz, int64_t n, double* out,
                                   fst_stream stream) {
    FST_TRY(check_eval_args(m, xyz, n, out));
    if (n == 0) return FST_OK;
    return eval_simt_launch<double>(m, xyz, n, out, (cudaStream_t)stream);
}
