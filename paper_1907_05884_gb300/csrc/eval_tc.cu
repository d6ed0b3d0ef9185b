// eval_tc.cu -- evaluation of a functional sparse Tucker model with the core contraction
// on the tcgen05 tensor cores (Sec. 2, eq. func_tuck; Sec. 6, reconstruction):
//
//   u~(y_b) = sum_j w2_j(y_b) sum_k T_{b,(j,k)} w3_k(y_b),   T = U1 C_(1)
//
// with U1[b][i] = w1_i(y_b1) (a 128-point tile x r1) and C_(1) the mode-1 unfolding of the
// core (r1 x r2 r3).  Per 128-point tile:
//   * worker warps (two groups of 4, alternating tiles) evaluate the Legendre factor values
//     of their point on the CUDA cores in FP32 (w1 to shared memory as the MMA A operand in
//     TF32 / BF16 / BF16 hi+lo, w2 and w3 kept in registers);
//   * one thread issues T = U1 C_(1) in column chunks of JC whole j-slices (N = JC * R3P
//     columns) into a 256-column tensor-memory buffer per group;
//   * the workers read each chunk back (tcgen05.ld, thread = point = TMEM lane) and reduce
//     it against w2 and w3 (the Khatri-Rao epilogue), then release the buffer.
// C_(1) is held in shared memory for the whole (persistent) kernel, as N x K K-major
// operand tiles built once per model and precision.  r3 is padded to R3P (8/16/24/32) and
// r1 to the MMA K granule with zeros, which contribute nothing.  Waits are bounded.
#include <cuda_bf16.h>

#include <vector>

#include "basis.cuh"
#include "tc_ptx.cuh"

namespace fst {

fst_status prepare_core_image(fst_model* m, int mode, int r3p);

namespace {

constexpr int kGroups = 2;
constexpr int kWorkers = 4 * kGroups;             // worker warps
constexpr int kThreadsE = (kWorkers + 1) * 32;    // + MMA warp
constexpr long long kWaitLimitE = 2000000000LL;

enum EMode { eTF32 = 0, eBF16 = 1, eBF16X3 = 2 };

__host__ __device__ constexpr int jc_for(int r3p) { return 256 / r3p; }

// Host-side description of the shared-memory image of C_(1).
struct CoreImage {
    int mode, r3p, jc, nc, ncp, kp, kb, nchunks, parts;
    size_t chunk_bytes, bytes;
};

CoreImage core_image_shape(const fst_model* m, int mode, int r3p) {
    CoreImage c;
    c.mode = mode;
    c.r3p = r3p;
    c.jc = jc_for(r3p);
    c.nc = c.jc * r3p;
    c.ncp = (c.nc + 15) / 16 * 16;
    const int gran = mode == eTF32 ? 8 : 16;
    c.kp = (m->r[0] + gran - 1) / gran * gran;
    c.kb = c.kp * (mode == eTF32 ? 4 : 2);
    c.nchunks = (m->r[1] + c.jc - 1) / c.jc;
    c.parts = mode == eBF16X3 ? 2 : 1;
    c.chunk_bytes = (size_t)c.ncp * c.kb;
    c.bytes = c.chunk_bytes * c.nchunks * c.parts;
    return c;
}

uint16_t bf16_bits(float x) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&h);
}
float bf16_val(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
uint32_t tf32_bits(float x) {
    // round to nearest (ties away) at 10 mantissa bits, like cvt.rna.tf32.f32
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    return u;
}

// Build the image: chunk c, part p at ((p * nchunks) + c) * chunk_bytes; row n of a chunk
// is core column (j, k) = (c*jc + n / r3p, n % r3p); K index = i.
std::vector<unsigned char> build_core_image(const fst_model* m, const CoreImage& c) {
    std::vector<unsigned char> img(c.bytes, 0);
    const int r1 = m->r[0], r2 = m->r[1], r3 = m->r[2];
    for (int ch = 0; ch < c.nchunks; ++ch)
        for (int n = 0; n < c.nc; ++n) {
            const int j = ch * c.jc + n / c.r3p, k = n % c.r3p;
            if (j >= r2 || k >= r3) continue;
            for (int i = 0; i < r1; ++i) {
                const float v = (float)m->alpha[((size_t)i * r2 + j) * r3 + k];
                const uint32_t es = c.mode == eTF32 ? 4 : 2;
                const uint32_t off = tc::kmajor_offset(n, i * es, c.kb);
                unsigned char* base = img.data() + (size_t)ch * c.chunk_bytes;
                if (c.mode == eTF32) {
                    const uint32_t b = tf32_bits(v);
                    memcpy(base + off, &b, 4);
                } else {
                    const uint16_t hi = bf16_bits(v);
                    memcpy(base + off, &hi, 2);
                    if (c.mode == eBF16X3) {
                        const uint16_t lo = bf16_bits(v - bf16_val(v));
                        memcpy(base + (size_t)c.nchunks * c.chunk_bytes + off, &lo, 2);
                    }
                }
            }
        }
    return img;
}

struct EvalTcArgs {
    EvalArgs<float> a;
    const unsigned char* core_img;
    int img_bytes;
    int nchunks;
    int kp;
    int err_code;
};

__device__ __forceinline__ uint32_t tf32_dev(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ uint32_t pack2_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int MODE, int R3P, int RM>
__global__ void __launch_bounds__(kThreadsE, 1)
eval_tc_kernel(const EvalTcArgs P, const float* __restrict__ xyz, int64_t n, float* __restrict__ out,
               int* __restrict__ err) {
    constexpr int ES = MODE == eTF32 ? 4 : 2;
    constexpr int JC = jc_for(R3P);
    constexpr int NC = JC * R3P;
    constexpr int NCP = (NC + 15) / 16 * 16;
    constexpr int MAXCH = (FST_MAX_RANK + JC - 1) / JC;
    constexpr int PARTS = MODE == eBF16X3 ? 2 : 1;
    const EvalArgs<float>& a = P.a;
    const int KP = P.kp, KB = KP * ES;
    const int SBO_A = (KB / 16) * 128;
    const int r1 = a.r[0];

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* core = smem;                                           // P.img_bytes
    unsigned char* abuf = core + ((P.img_bytes + 1023) & ~1023);          // kGroups x PARTS x 128 x KB
    const int abytes = 128 * KB;
    float* fsm = reinterpret_cast<float*>(abuf + kGroups * PARTS * abytes);   // recurrence + W tables
    float* ra = fsm;
    float* rb = ra + a.pm;
    float* Ws[3];
    Ws[0] = rb + a.pm;
    Ws[1] = Ws[0] + a.pe[0] * RM;
    Ws[2] = Ws[1] + a.pe[1] * RM;
    uint8_t* mk = reinterpret_cast<uint8_t*>(Ws[2] + a.pe[2] * RM);
    uint64_t* bars = reinterpret_cast<uint64_t*>(((uintptr_t)(mk + 3 * a.pm) + 15) & ~(uintptr_t)15);
    uint64_t* a_full = bars;                 // [kGroups] workers -> MMA: A tile written
    uint64_t* a_empty = bars + kGroups;      // [kGroups] MMA -> workers: A tile consumed
    uint64_t* d_full = bars + 2 * kGroups;   // [kGroups] MMA -> workers: chunk in TMEM
    uint64_t* d_empty = bars + 3 * kGroups;  // [kGroups] workers -> MMA: chunk read
    uint64_t* drain = bars + 4 * kGroups;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
    // shared tables: core image, recurrence, dense coefficient rows
    {
        const uint4* src = reinterpret_cast<const uint4*>(P.core_img);
        uint4* dst = reinterpret_cast<uint4*>(core);
        for (int e = tid; e < P.img_bytes / 16; e += blockDim.x) dst[e] = src[e];
        for (int i = tid; i < a.pm; i += blockDim.x) {
            ra[i] = float(2 * i + 1) / float(i + 1);
            rb[i] = float(i) / float(i + 1);
        }
        for (int k = 0; k < 3; ++k) {
            const int rk = a.r[k];
            for (int e = tid; e < a.pe[k] * RM; e += blockDim.x) {
                const int nn = e / RM, j = e - nn * RM;
                Ws[k][e] = j < rk ? a.W[k][nn * rk + j] : 0.f;
            }
            for (int e = tid; e < a.pm; e += blockDim.x) mk[k * a.pm + e] = e < a.pe[k] ? a.mask[k][e] : 0;
        }
    }
    if (tid == 0) {
        for (int g = 0; g < kGroups; ++g) {
            tc::mbar_init(&a_full[g], 4);
            tc::mbar_init(&a_empty[g], 1);
            tc::mbar_init(&d_full[g], 1);
            tc::mbar_init(&d_empty[g], 4);
        }
        tc::mbar_init(drain, 1);
        tc::fence_mbar_init();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const long long ntiles = (n + 127) / 128;
    const int nch = P.nchunks;

    if (warp < kWorkers) {
        // ------------------------------------------------------------------ workers
        const int g = warp >> 2, sub = warp & 3, row = sub * 32 + lane;   // TMEM lane = row
        unsigned char* A = abuf + g * PARTS * abytes;
        int lt = 0;            // tiles of this group
        int cc = 0;            // chunks of this group
        bool dead = false;
        for (long long t = blockIdx.x + (long long)g * gridDim.x; t < ntiles;
             t += (long long)kGroups * gridDim.x, ++lt) {
            const int64_t q = t * 128 + row;
            const bool ok = q < n;
            float tt[3][1];
#pragma unroll
            for (int k = 0; k < 3; ++k) tt[k][0] = fmaf(ok ? xyz[k * n + q] : 0.f, a.sc[k], a.of[k]);
            float w[1][RM], u2[RM], u3[RM];
            factor_values<float, RM, 1>(tt[1], Ws[1], mk + a.pm, a.pe[1], ra, rb, w);
#pragma unroll
            for (int j = 0; j < RM; ++j) u2[j] = w[0][j];
            factor_values<float, RM, 1>(tt[2], Ws[2], mk + 2 * a.pm, a.pe[2], ra, rb, w);
#pragma unroll
            for (int j = 0; j < RM; ++j) u3[j] = j < a.r[2] ? w[0][j] : 0.f;
            factor_values<float, RM, 1>(tt[0], Ws[0], mk, a.pe[0], ra, rb, w);   // w1 -> A operand
            if (!tc::mbar_wait(&a_empty[g], (uint32_t)(lt & 1) ^ 1u, kWaitLimitE)) {
                atomicOr(err, 1);
                dead = true;
            }
            if (!dead) {
                // row `row` of the A tile: KP values of w1 (zero beyond r1), 16 bytes at a time
#pragma unroll
                for (int c16 = 0; c16 < (RM * ES + 15) / 16 + 1; ++c16) {
                    if (c16 * 16 >= KB) break;
                    const uint32_t off = tc::kmajor_offset(row, c16 * 16, KB);
                    if (MODE == eTF32) {
                        uint32_t v4[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int i = c16 * 4 + e;
                            v4[e] = tf32_dev(i < RM && i < r1 ? w[0][i < RM ? i : 0] : 0.f);
                        }
                        *reinterpret_cast<uint4*>(A + off) = make_uint4(v4[0], v4[1], v4[2], v4[3]);
                    } else {
                        float h[8], l[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int i = c16 * 8 + e;
                            const float x = (i < RM && i < r1) ? w[0][i < RM ? i : 0] : 0.f;
                            h[e] = x;
                            l[e] = x - __bfloat162float(__float2bfloat16_rn(x));
                        }
                        *reinterpret_cast<uint4*>(A + off) =
                            make_uint4(pack2_bf16(h[0], h[1]), pack2_bf16(h[2], h[3]), pack2_bf16(h[4], h[5]),
                                       pack2_bf16(h[6], h[7]));
                        if (MODE == eBF16X3)
                            *reinterpret_cast<uint4*>(A + abytes + off) =
                                make_uint4(pack2_bf16(l[0], l[1]), pack2_bf16(l[2], l[3]), pack2_bf16(l[4], l[5]),
                                           pack2_bf16(l[6], l[7]));
                    }
                }
                tc::fence_async_smem();
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&a_full[g]);
            // Khatri-Rao epilogue, chunk by chunk
            float f = 0.f;
            const uint32_t tbase = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(g * 256);
#pragma unroll
            for (int ch = 0; ch < MAXCH; ++ch) {
                if (ch < nch) {
                    if (!tc::mbar_wait(&d_full[g], (uint32_t)(cc & 1), kWaitLimitE)) {
                        atomicOr(err, 2);
                        dead = true;
                    }
                    tc::fence_after_sync();
                    float s = 0.f;
#pragma unroll
                    for (int c0 = 0; c0 < NC; c0 += 16) {
                        float v[16];
                        tc::tmem_ld16(tbase + c0, v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int col = c0 + e;
                            if (col < NC) {
                                const int jl = col / R3P, k = col % R3P;
                                s = fmaf(v[e], u3[k], s);
                                if (k == R3P - 1) {
                                    const int j = ch * JC + jl;
                                    if (j < RM) f = fmaf(s, u2[j < RM ? j : 0], f);
                                    s = 0.f;
                                }
                            }
                        }
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&d_empty[g]);
                    ++cc;
                }
            }
            if (ok) out[q] = f;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA issuer
        constexpr uint32_t idesc = MODE == eTF32 ? tc::idesc_tf32(128, NCP) : tc::idesc_bf16(128, NCP);
        const int kst = KB / 32;                   // MMAs (32 bytes of K each) per product
        const uint32_t SBO_B = SBO_A;              // same K extent
        const uint32_t core_u32 = tc::smem_u32(core);
        const uint32_t chunk_bytes = (uint32_t)(NCP * KB);
        int lt[kGroups] = {0, 0}, cc[kGroups] = {0, 0};
        bool issued = false, dead = false;
        for (long long t = blockIdx.x; t < ntiles && !dead; t += gridDim.x) {
            const int g = (int)(((t - blockIdx.x) / gridDim.x) % kGroups);
            const uint32_t abase = tc::smem_u32(abuf + g * PARTS * abytes);
            if (!tc::mbar_wait(&a_full[g], (uint32_t)(lt[g] & 1), kWaitLimitE)) {
                atomicOr(err, 4);
                break;
            }
            tc::fence_after_sync();
            for (int ch = 0; ch < nch; ++ch) {
                if (!tc::mbar_wait(&d_empty[g], (uint32_t)(cc[g] & 1) ^ 1u, kWaitLimitE)) {
                    atomicOr(err, 8);
                    dead = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(g * 256);
                const uint32_t bb = core_u32 + ch * chunk_bytes;
                for (int ks = 0; ks < kst; ++ks) {
                    const uint32_t ko = ks * 256;
                    const uint64_t ad = tc::make_desc(abase + ko, 128, SBO_A);
                    const uint64_t bd = tc::make_desc(bb + ko, 128, SBO_B);
                    if (MODE == eTF32) {
                        tc::mma_tf32(d, ad, bd, idesc, ks > 0);
                    } else {
                        tc::mma_bf16(d, ad, bd, idesc, ks > 0);
                        if (MODE == eBF16X3) {
                            const uint64_t al = tc::make_desc(abase + abytes + ko, 128, SBO_A);
                            const uint64_t bl = tc::make_desc(bb + nch * chunk_bytes + ko, 128, SBO_B);
                            tc::mma_bf16(d, ad, bl, idesc, 1u);
                            tc::mma_bf16(d, al, bd, idesc, 1u);
                        }
                    }
                }
                tc::mma_commit(&d_full[g]);
                issued = true;
                ++cc[g];
            }
            if (dead) break;
            tc::mma_commit(&a_empty[g]);
            ++lt[g];
        }
        if (issued) {
            tc::mma_commit(drain);
            if (!tc::mbar_wait(drain, 0u, kWaitLimitE)) atomicOr(err, 16);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

struct EvalErr {
    std::mutex mu;
    DevBuf flag;
};
EvalErr g_eval_err[64];

}  // namespace

// Tensor-core operand image of the core for (mode, r3 padding), cached in the model.
fst_status prepare_core_image(fst_model* m, int mode, int r3p) {
    const CoreImage ci = core_image_shape(m, mode, r3p);
    const int kind = mode * 64 + r3p;
    if (m->tc_core_kind == kind && m->tc_core) return FST_OK;
    std::vector<unsigned char> img = build_core_image(m, ci);
    if (m->tc_core_bytes < img.size()) {
        if (m->tc_core) cudaFree(m->tc_core);
        m->tc_core = nullptr;
        m->tc_core_bytes = 0;
        FST_CUDA(cudaMalloc(&m->tc_core, img.size()));
        m->tc_core_bytes = img.size();
    }
    FST_CUDA(cudaMemcpy(m->tc_core, img.data(), img.size(), cudaMemcpyHostToDevice));
    m->tc_core_kind = kind;
    return FST_OK;
}

namespace {

template <int MODE, int R3P, int RM>
fst_status launch_eval_tc(fst_model* m, const float* xyz, int64_t n, float* out, cudaStream_t s, int* err) {
    const CoreImage ci = core_image_shape(m, MODE, R3P);
    FST_TRY(prepare_core_image(m, MODE, R3P));
    EvalTcArgs P;
    P.a = make_args<float>(m);
    bind(P.a, m);
    P.core_img = static_cast<const unsigned char*>(m->tc_core);
    P.img_bytes = (int)ci.bytes;
    P.nchunks = ci.nchunks;
    P.kp = ci.kp;
    P.err_code = 0;
    const int ES = MODE == eTF32 ? 4 : 2;
    const int PARTS = MODE == eBF16X3 ? 2 : 1;
    const size_t smem = 1024 + (((size_t)ci.bytes + 1023) & ~(size_t)1023) + (size_t)kGroups * PARTS * 128 * ci.kp * ES +
                        (2 * (size_t)P.a.pm + (size_t)(P.a.pe[0] + P.a.pe[1] + P.a.pe[2]) * RM) * 4 + 3 * P.a.pm +
                        16 + 8 * (4 * kGroups + 2);
    if (smem > 227 * 1024) {
        set_error("model too large for the tensor-core evaluator (%zu bytes of shared memory)", smem);
        return FST_EUNSUPPORTED;
    }
    auto kern = eval_tc_kernel<MODE, R3P, RM>;
    FST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long ntiles = (n + 127) / 128;
    long long grid = sm_count();
    if (ntiles < grid) grid = ntiles;
    kern<<<(unsigned)grid, kThreadsE, smem, s>>>(P, xyz, n, out, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <int MODE>
fst_status dispatch_r3(fst_model* m, const float* xyz, int64_t n, float* out, cudaStream_t s, int* err) {
    int rmax = m->r[0] > m->r[1] ? m->r[0] : m->r[1];
    rmax = m->r[2] > rmax ? m->r[2] : rmax;
    const int r3 = m->r[2];
    // RM bounds all three ranks (register arrays); R3P pads r3 for the chunk layout
    if (rmax <= 8) return launch_eval_tc<MODE, 8, 8>(m, xyz, n, out, s, err);
    if (rmax <= 16) return r3 <= 8 ? launch_eval_tc<MODE, 8, 16>(m, xyz, n, out, s, err)
                                   : launch_eval_tc<MODE, 16, 16>(m, xyz, n, out, s, err);
    if (rmax <= 24) return r3 <= 8    ? launch_eval_tc<MODE, 8, 24>(m, xyz, n, out, s, err)
                           : r3 <= 16 ? launch_eval_tc<MODE, 16, 24>(m, xyz, n, out, s, err)
                                      : launch_eval_tc<MODE, 24, 24>(m, xyz, n, out, s, err);
    return r3 <= 8    ? launch_eval_tc<MODE, 8, 32>(m, xyz, n, out, s, err)
           : r3 <= 16 ? launch_eval_tc<MODE, 16, 32>(m, xyz, n, out, s, err)
           : r3 <= 24 ? launch_eval_tc<MODE, 24, 32>(m, xyz, n, out, s, err)
                      : launch_eval_tc<MODE, 32, 32>(m, xyz, n, out, s, err);
}

}  // namespace

fst_status eval_tc_launch(fst_model* m, const float* xyz, int64_t n, float* out, fst_prec prec, cudaStream_t s) {
    if (n == 0) return FST_OK;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    EvalErr& ee = g_eval_err[dev & 63];
    std::lock_guard<std::mutex> lk(m->mu);
    {
        std::lock_guard<std::mutex> lk2(ee.mu);
        if (!ee.flag.ptr) {
            FST_TRY(ee.flag.ensure(sizeof(int)));
            FST_CUDA(cudaMemset(ee.flag.ptr, 0, sizeof(int)));
        }
    }
    int* err = ee.flag.as<int>();
    switch (prec) {
        case FST_TF32: return dispatch_r3<eTF32>(m, xyz, n, out, s, err);
        case FST_BF16: return dispatch_r3<eBF16>(m, xyz, n, out, s, err);
        case FST_BF16X3: return dispatch_r3<eBF16X3>(m, xyz, n, out, s, err);
        default:
            set_error("tensor-core evaluation takes TF32, BF16 or BF16X3");
            return FST_EINVAL;
    }
}

// Device error word of the tensor-core evaluator (bounded waits that expired), read and
// cleared by fst_eval_check.
fst_status eval_tc_check(cudaStream_t s) {
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    EvalErr& ee = g_eval_err[dev & 63];
    std::lock_guard<std::mutex> lk(ee.mu);
    if (!ee.flag.ptr) return FST_OK;
    int h = 0;
    FST_CUDA(cudaMemcpyAsync(&h, ee.flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    if (h) {
        FST_CUDA(cudaMemsetAsync(ee.flag.ptr, 0, sizeof(int), s));
        set_error("tensor-core evaluation: a bounded device wait expired (code %d)", h);
        return FST_ETIMEOUT;
    }
    return FST_OK;
}

}  // namespace fst

extern "C" fst_status fst_eval_check(fst_stream stream) { return fst::eval_tc_check((cudaStream_t)stream); }

extern "C" fst_status fst_eval_prepare(fst_model* m, fst_prec prec) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    if (prec == FST_FP32 || prec == FST_FP64) return FST_OK;
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3, "unknown precision %d", (int)prec);
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == m->device, "model lives on device %d, current device is %d", m->device, dev);
    // a zero-length evaluation on the legacy stream builds the operand image
    cudaStream_t s = 0;
    std::lock_guard<std::mutex> lk(m->mu);
    const int mode = prec == FST_TF32 ? 0 : prec == FST_BF16 ? 1 : 2;
    int rmax = m->r[0] > m->r[1] ? m->r[0] : m->r[1];
    rmax = m->r[2] > rmax ? m->r[2] : rmax;
    const int r3 = m->r[2];
    const int r3p = r3 <= 8 ? 8 : r3 <= 16 ? 16 : r3 <= 24 ? 24 : 32;
    (void)rmax;
    (void)s;
    return fst::prepare_core_image(m, mode, r3p);
}
