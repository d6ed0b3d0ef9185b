// gram_tc.cu -- normal matrix G = A^T A of the sampled least-squares problem on the
// tcgen05 tensor cores (Sec. 5, eq. rand_core; Algorithm 2, solve step), FP32 accumulation
// in tensor memory.
//
// A_{s,a} = w1_i(y_s) w2_j(y_s) w3_k(y_s), a = (i j k) in C order, is never stored: its
// operand tiles are generated on the fly from the factor values U_1..U_3 of the m sampled
// rows (m x 72 FP32 values at r = 24: L2-resident).
//
// Work unit: a 256 x 256 super-tile (ti >= tj) of the lower triangle, as two M = 128,
// N = 256 accumulators (all 512 TMEM columns).  Persistent grid, one CTA per SM:
//   warps 0-7  producers: per K stage (KC sampled rows) stage U_1..U_3 of those rows in
//              shared memory (transposed), build the 256-row A and B operand tiles in the
//              K-major no-swizzle layout (see tc_ptx.cuh), signal `full`; after a
//              super-tile's last stage they read the accumulators back (tcgen05.ld) and
//              store G, then signal `tmem_empty`;
//   warp 8     one thread issues the MMAs of each stage and commits to `empty` (stage
//              reusable) and, after the last stage, to `tmem_full`.
// Precisions: TF32 (kind::tf32, K = 8 per MMA), BF16 (kind::f16), and BF16X3, where
// A = A_hi + A_lo in BF16 and G ~ A_hi^T A_hi + A_hi^T A_lo + A_lo^T A_hi.
// Every wait is bounded (~1 s); on expiry the kernel records an error and drains.
#include <cuda_bf16.h>

#include "fst_internal.cuh"
#include "tc_ptx.cuh"

namespace fst {

namespace {

constexpr int kProducerWarps = 8;
constexpr int kThreads = (kProducerWarps + 1) * 32;
constexpr int kStages = 2;
constexpr int kTile = 256;              // super-tile edge
constexpr long long kWaitLimit = 2000000000LL;

enum Mode { kTF32 = 0, kBF16 = 1, kBF16X3 = 2 };

template <int MODE>
struct Cfg {
    static constexpr int ES = MODE == kTF32 ? 4 : 2;                 // operand element bytes
    static constexpr int KB = MODE == kBF16X3 ? 64 : 128;            // operand row bytes per stage
    static constexpr int KC = KB / ES;                                // sampled rows per stage
    static constexpr int QPC = 16 / ES;                               // rows per 16-byte chunk
    static constexpr int NG = KC / QPC;                               // chunks per operand row
    static constexpr int PARTS = MODE == kBF16X3 ? 2 : 1;             // hi (+ lo)
    static constexpr int TILE_BYTES = kTile * KB;                     // one 256-row operand tile
    static constexpr int USTRIDE = KC + 4;                            // padded row of the U stage
    static constexpr int U_FLOATS = 3 * FST_MAX_RANK * USTRIDE;
    static constexpr int STAGE_BYTES = 2 * PARTS * TILE_BYTES + U_FLOATS * 4;
    static constexpr int ROWTAB = 2 * 2 * kTile * 8;                  // per-tile row table, 2 buffers
    static constexpr int SMEM = kStages * STAGE_BYTES + ROWTAB + 2048; // + barriers, alignment slack
    static constexpr int KSTEPS = KB / 32;                            // MMAs per stage per product
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Barrier 1 over the producer warps that also ORs a flag across them: every producer
// thread gets the same answer, so abort decisions never split the producer group.
__device__ __forceinline__ bool producers_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kProducerWarps * 32)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const float* __restrict__ U1, const float* __restrict__ U2, const float* __restrict__ U3,
               int64_t m, int r1, int r2, int r3, float* __restrict__ G, int* __restrict__ err) {
    using C = Cfg<MODE>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * C::STAGE_BYTES);
    uint64_t* empty = full + kStages;
    uint64_t* tmem_full = empty + kStages;
    uint64_t* tmem_empty = tmem_full + 1;
    uint64_t* drain = tmem_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // rowtab[buf][row] = {off(w1_i) | off(w2_j) << 16, off(w3_k) | valid << 31}: shared-memory
    // offsets of the factor rows of operand row `row` (0..255 super-tile rows, 256..511 columns)
    int2* rowtab = reinterpret_cast<int2*>(smem + kStages * C::STAGE_BYTES + 1024);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = r1 * r2 * r3;
    const int nT = (R + kTile - 1) / kTile;
    const long long ntiles = (long long)nT * (nT + 1) / 2;
    const long long nK = (m + C::KC - 1) / C::KC;

    if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], kProducerWarps);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tmem_full, 1);
        tc::mbar_init(tmem_empty, kProducerWarps);
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

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers + epilogue
        long long gs = 0;   // global stage counter
        int tcount = 0;
        bool stop = false;
        // Factor values of the next stage are loaded into registers one stage ahead
        // (every tile walks the same sampled rows, so the prefetch ignores tile bounds).
        constexpr int kPer = C::KC * 3 * FST_MAX_RANK / (kProducerWarps * 32);
        float pre[kPer];
        auto load_stage = [&](long long kc) {
            const long long q0 = kc * C::KC;
#pragma unroll
            for (int it = 0; it < kPer; ++it) {
                const int e = tid + it * kProducerWarps * 32;
                const int q = e / (3 * FST_MAX_RANK), c = e - q * (3 * FST_MAX_RANK);
                const int mode = c / FST_MAX_RANK, col = c - mode * FST_MAX_RANK;
                const long long srow = q0 + q;
                const int rk = mode == 0 ? r1 : mode == 1 ? r2 : r3;
                const float* Uk = mode == 0 ? U1 : mode == 1 ? U2 : U3;
                pre[it] = (col < rk && srow < m) ? __ldg(Uk + srow * rk + col) : 0.f;
            }
        };
        load_stage(0);
        for (long long t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++tcount) {
            int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
            while ((long long)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while ((long long)ti * (ti + 1) / 2 > t) --ti;
            const int tj = (int)(t - (long long)ti * (ti + 1) / 2);
            int2* tab = rowtab + (tcount & 1) * 2 * kTile;
            for (int row = tid; row < 2 * kTile; row += kProducerWarps * 32) {
                const int a = (row >= kTile ? tj : ti) * kTile + (row & (kTile - 1));
                int2 e = make_int2(0, 0);
                if (a < R) {
                    const int i = a / (r2 * r3), j = (a / r3) % r2, k = a % r3;
                    e = make_int2((i * C::USTRIDE) | ((FST_MAX_RANK + j) * C::USTRIDE) << 16,
                                  ((2 * FST_MAX_RANK + k) * C::USTRIDE) | (int)0x80000000);
                }
                tab[row] = e;
            }
            // (the first stage's producer barrier orders these writes before their use; the
            //  other buffer may still be read by a slower warp finishing the previous tile)
            for (long long kc = 0; kc < nK; ++kc, ++gs) {
                const int st = (int)(gs % kStages);
                const uint32_t ph = (uint32_t)((gs / kStages) & 1);
                const bool ok = tc::mbar_wait(&empty[st], ph ^ 1u, kWaitLimit);
                if (!ok) fail(1);
                const bool skip = !ok || *abort_flag;
                unsigned char* sbase = smem + st * C::STAGE_BYTES;
                float* us = reinterpret_cast<float*>(sbase + 2 * C::PARTS * C::TILE_BYTES);
                float* u1T = us;
                float* u2T = us + FST_MAX_RANK * C::USTRIDE;
                float* u3T = us + 2 * FST_MAX_RANK * C::USTRIDE;
                // store this stage's factor values (transposed), then start loading the next
                if (!skip) {
#pragma unroll
                    for (int it = 0; it < kPer; ++it) {
                        const int e = tid + it * kProducerWarps * 32;
                        const int q = e / (3 * FST_MAX_RANK), c = e - q * (3 * FST_MAX_RANK);
                        const int mode = c / FST_MAX_RANK, col = c - mode * FST_MAX_RANK;
                        us[mode * FST_MAX_RANK * C::USTRIDE + col * C::USTRIDE + q] = pre[it];
                    }
                }
                load_stage(kc + 1 < nK ? kc + 1 : 0);
                if (producers_any(skip)) { stop = true; break; }
                // operand rows: 0..255 -> A (super-tile rows), 256..511 -> B (super-tile columns)
                constexpr int kTasks = (2 * kTile / 8) * (C::NG / 4);   // warp tasks of 8 rows x 4 chunks
                for (int task = warp; task < kTasks; task += kProducerWarps) {
                    const int rowblk = task / (C::NG / 4);
                    const int g = (task % (C::NG / 4)) * 4 + (lane >> 3);
                    const int row = rowblk * 8 + (lane & 7);
                    const bool isB = row >= kTile;
                    const int lrow = isB ? row - kTile : row;
                    const int2 te = tab[row];
                    float v[C::QPC];
                    if (te.y < 0) {
                        const float* p1 = us + (te.x & 0xFFFF) + g * C::QPC;
                        const float* p2 = us + ((unsigned)te.x >> 16) + g * C::QPC;
                        const float* p3 = us + (te.y & 0x7FFFFFFF) + g * C::QPC;
#pragma unroll
                        for (int e = 0; e < C::QPC; e += 4) {
                            const float4 x1 = *reinterpret_cast<const float4*>(p1 + e);
                            const float4 x2 = *reinterpret_cast<const float4*>(p2 + e);
                            const float4 x3 = *reinterpret_cast<const float4*>(p3 + e);
                            v[e] = x1.x * x2.x * x3.x;
                            v[e + 1] = x1.y * x2.y * x3.y;
                            v[e + 2] = x1.z * x2.z * x3.z;
                            v[e + 3] = x1.w * x2.w * x3.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < C::QPC; ++e) v[e] = 0.f;
                    }
                    const uint32_t off = tc::kmajor_offset(lrow, g * 16, C::KB);
                    unsigned char* tile = sbase + (isB ? C::PARTS * C::TILE_BYTES : 0);
                    uint4 w;
                    if (MODE == kTF32) {
                        w = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
                        *reinterpret_cast<uint4*>(tile + off) = w;
                    } else {
                        w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                       pack_bf16(v[6], v[7]));
                        *reinterpret_cast<uint4*>(tile + off) = w;
                        if (MODE == kBF16X3) {
                            float lo[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                lo[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
                            const uint4 wl = make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]),
                                                        pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
                            *reinterpret_cast<uint4*>(tile + C::TILE_BYTES + off) = wl;
                        }
                    }
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&full[st]);
                // U stage reuse is ordered by the next `empty` wait of this stage
            }
            if (stop) break;
            // ---------------------------------------------------------- epilogue
            if (!tc::mbar_wait(tmem_full, (uint32_t)(tcount & 1), kWaitLimit)) fail(2);
            tc::fence_after_sync();
            const int half = warp >> 2;                 // accumulator 0: rows 0..127, 1: rows 128..255
            const int sub = warp & 3;                   // TMEM lanes 32*sub .. 32*sub+31
            const int row = ti * kTile + half * 128 + sub * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(half * 256);
            for (int c0 = 0; c0 < kTile; c0 += 16) {
                float v[16];
                tc::tmem_ld16(taddr + c0, v);
                tc::tmem_wait_ld();
                const int col = tj * kTile + c0;
                if (row < R) {
                    float* dst = G + (size_t)row * R + col;
                    if (col + 16 <= R && (R & 3) == 0) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
                        for (int e = 0; e < 16 && col + e < R; ++e) dst[e] = v[e];
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tmem_empty);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        constexpr uint32_t idesc = MODE == kTF32 ? tc::idesc_tf32(128, 256) : tc::idesc_bf16(128, 256);
        constexpr uint32_t SBO = (C::KB / 16) * 128;
        long long gs = 0;
        int tcount = 0;
        bool issued = false;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tcount) {
            if (!tc::mbar_wait(tmem_empty, (uint32_t)(tcount & 1) ^ 1u, kWaitLimit)) { fail(4); break; }
            tc::fence_after_sync();
            for (long long kc = 0; kc < nK; ++kc, ++gs) {
                const int st = (int)(gs % kStages);
                const uint32_t ph = (uint32_t)((gs / kStages) & 1);
                if (!tc::mbar_wait(&full[st], ph, kWaitLimit)) { fail(8); break; }
                tc::fence_after_sync();
                const uint32_t abase = tc::smem_u32(smem + st * C::STAGE_BYTES);
                const uint32_t bbase = abase + C::PARTS * C::TILE_BYTES;
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    const uint32_t ko = ks * 256;
                    const uint64_t b_hi = tc::make_desc(bbase + ko, 128, SBO);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t ao = h * 16 * SBO + ko;      // rows 128h .. 128h+127
                        const uint64_t a_hi = tc::make_desc(abase + ao, 128, SBO);
                        const uint32_t d = tmem + (uint32_t)(h * 256);
                        if (MODE == kTF32) {
                            tc::mma_tf32(d, a_hi, b_hi, idesc, acc);
                        } else {
                            tc::mma_bf16(d, a_hi, b_hi, idesc, acc);
                            if (MODE == kBF16X3) {
                                const uint64_t a_lo = tc::make_desc(abase + C::TILE_BYTES + ao, 128, SBO);
                                const uint64_t b_lo = tc::make_desc(bbase + C::TILE_BYTES + ko, 128, SBO);
                                tc::mma_bf16(d, a_hi, b_lo, idesc, 1u);
                                tc::mma_bf16(d, a_lo, b_hi, idesc, 1u);
                            }
                        }
                    }
                }
                tc::mma_commit(&empty[st]);
                issued = true;
            }
            if (*abort_flag) break;
            tc::mma_commit(tmem_full);
        }
        if (issued) {
            // wait for every MMA of this CTA before tensor memory is released
            tc::mma_commit(drain);
            if (!tc::mbar_wait(drain, 0u, kWaitLimit)) atomicOr(err, 16);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int MODE>
fst_status launch(const float* U1, const float* U2, const float* U3, int64_t m, int r1, int r2, int r3, float* G,
                  int* err, cudaStream_t s) {
    using C = Cfg<MODE>;
    auto kern = gram_tc_kernel<MODE>;
    FST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    const int R = r1 * r2 * r3;
    const long long nT = (R + kTile - 1) / kTile;
    const long long ntiles = nT * (nT + 1) / 2;
    int grid = sm_count();
    if (ntiles < grid) grid = (int)ntiles;
    kern<<<grid, kThreads, C::SMEM, s>>>(U1, U2, U3, m, r1, r2, r3, G, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

struct GramErr {
    std::mutex mu;
    DevBuf flag;
};
GramErr g_gram_err[64];

}  // namespace

fst_status gram_tc_launch(const fst_model* M, const float* U1, const float* U2, const float* U3, int64_t m,
                          float* G, fst_prec prec, cudaStream_t s) {
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    GramErr& ge = g_gram_err[dev & 63];
    std::lock_guard<std::mutex> lk(ge.mu);
    FST_TRY(ge.flag.ensure(sizeof(int)));
    int* err = ge.flag.as<int>();
    FST_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    fst_status st;
    switch (prec) {
        case FST_TF32: st = launch<kTF32>(U1, U2, U3, m, r1, r2, r3, G, err, s); break;
        case FST_BF16: st = launch<kBF16>(U1, U2, U3, m, r1, r2, r3, G, err, s); break;
        case FST_BF16X3: st = launch<kBF16X3>(U1, U2, U3, m, r1, r2, r3, G, err, s); break;
        default:
            set_error("tensor-core Gram takes TF32, BF16 or BF16X3");
            return FST_EINVAL;
    }
    if (st != FST_OK) return st;
    int herr = 0;
    FST_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("tensor-core Gram: a bounded device wait expired (code %d)", herr);
        return FST_ETIMEOUT;
    }
    return FST_OK;
}

}  // namespace fst
