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

constexpr int kProducerWarps = 16;
constexpr int kEpilogueWarps = 8;       // producer warps 0-7 also drain the accumulators
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
    static constexpr int QPC = 16 / ES;                               // sampled rows per 16-byte chunk
    static constexpr int NG = KC / QPC;                               // chunks per operand row
    static constexpr int PARTS = MODE == kBF16X3 ? 2 : 1;             // hi (+ lo)
    static constexpr int TILE_BYTES = kTile * KB;                     // one 256-row operand tile
    static constexpr int STAGE_BYTES = 2 * PARTS * TILE_BYTES;        // A and B operand tiles
    // staging of one stage: pair products of the A and B tiles' pairs, then w3 rows; the
    // number of rows and of staging buffers (the cp.async prefetch depth) is set at launch
    static constexpr int PSTRIDE = KC + 4;                            // floats per staged row
    static constexpr int FIXED = kStages * STAGE_BYTES + 2048;
    static constexpr int KSTEPS = KB / 32;                            // MMAs per stage per product
};

struct TaskInfo {
    int op, k, g, plo, pb, pe, base;
};
// tasks per producer warp: 2 operands x 4 groups of 8 k (r3 <= 32) x 2 chunk groups x 4
// quarters of the pair range, over the producer warps
constexpr int kSplit = 4;
constexpr int kMaxTasks = (2 * 4 * 2 * kSplit) / 16;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
gram_tc_kernel(const float* __restrict__ PT, const float* __restrict__ U3T, int64_t m, int64_t mpad, int r1, int r2,
               int r3, int halfp, int nstg, float* __restrict__ G, int* __restrict__ err) {
    using C = Cfg<MODE>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* stg0 = reinterpret_cast<float*>(smem + kStages * C::STAGE_BYTES);
    const int stg_floats = (2 * halfp + r3) * C::PSTRIDE;
    uint64_t* full = reinterpret_cast<uint64_t*>(stg0 + nstg * stg_floats);
    uint64_t* empty = full + kStages;
    uint64_t* tmem_full = empty + kStages;
    uint64_t* tmem_empty = tmem_full + 1;
    uint64_t* drain = tmem_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = r1 * r2 * r3;
    const int nT = (R + kTile - 1) / kTile;
    const long long ntiles = (long long)nT * (nT + 1) / 2;
    const int nK = (int)((m + C::KC - 1) / C::KC);

    if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], kProducerWarps);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tmem_full, 1);
        tc::mbar_init(tmem_empty, kEpilogueWarps);
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
    auto decode = [&](long long t, int& ti, int& tj) {
        ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((long long)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while ((long long)ti * (ti + 1) / 2 > t) --ti;
        tj = (int)(t - (long long)ti * (ti + 1) / 2);
    };
    // pairs (i, j) whose rows (p r3 .. p r3 + r3 - 1) meet operand tile `tile`
    auto pair_range = [&](int tile, int& plo, int& phi) {
        const int row0 = tile * kTile;
        const int row1 = min(row0 + kTile, R) - 1;
        plo = row0 / r3;
        phi = row1 / r3;
    };

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers + epilogue
        // Stage loads (pair products and w3 rows of KC sampled rows) go through cp.async
        // nstg-1 stages ahead, into a ring of nstg staging buffers (one commit group per stage).
        // prefetch position: tile (decoded once per tile) and stage within it
        long long pf_t = blockIdx.x;
        int pf_kc = 0;
        int pf_alo = 0, pf_ahi = -1, pf_blo = 0, pf_bhi = -1;
        auto pf_decode = [&]() {
            if (pf_t < ntiles) {
                int ti, tj;
                decode(pf_t, ti, tj);
                pair_range(ti, pf_alo, pf_ahi);
                pair_range(tj, pf_blo, pf_bhi);
            }
        };
        pf_decode();
        auto issue_loads = [&](int kc, int buf) {
            const int alo = pf_alo, ahi = pf_ahi, blo = pf_blo, bhi = pf_bhi;
            const int nA = ahi - alo + 1, nB = bhi - blo + 1;
            float* P = stg0 + buf * stg_floats;
            const long long q0 = (long long)kc * C::KC;
            constexpr int CPR = C::KC / 4;                       // 16-byte chunks per row
            const int rows = nA + nB + r3;
            for (int c = tid; c < rows * CPR; c += kProducerWarps * 32) {
                const int r = c / CPR, cc = c - r * CPR;
                const float* src;
                float* dst;
                if (r < nA) {
                    src = PT + (size_t)(alo + r) * mpad;
                    dst = P + r * C::PSTRIDE;
                } else if (r < nA + nB) {
                    src = PT + (size_t)(blo + r - nA) * mpad;
                    dst = P + (halfp + r - nA) * C::PSTRIDE;
                } else {
                    src = U3T + (size_t)(r - nA - nB) * mpad;
                    dst = P + (2 * halfp + r - nA - nB) * C::PSTRIDE;
                }
                cp_async16(dst + cc * 4, src + q0 + cc * 4);
            }
            cp_async_commit();
        };
        int gs = 0;         // global stage counter
        int tcount = 0;
        bool stop = false;
        // stages are prefetched in order; issue_next() loads the next one (or commits an
        // empty group past the last stage, keeping one group per stage)
        auto issue_next = [&](int buf) {
            if (pf_t < ntiles) {
                issue_loads(pf_kc, buf);
                if (++pf_kc == nK) {
                    pf_kc = 0;
                    pf_t += gridDim.x;
                    pf_decode();
                }
            } else {
                cp_async_commit();
            }
        };
        for (int g0 = 0; g0 < nstg - 1; ++g0) issue_next(g0);
        const int KG = (r3 + 7) / 8;
        const int ntasks = 2 * KG * (C::NG / 4) * kSplit;
        for (long long t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++tcount) {
            int ti, tj;
            decode(t, ti, tj);
            // this warp's generation tasks for the tile: (operand, 8 values of k, 4 chunks, half
            // of the pairs), fixed for all of the tile's stages
            TaskInfo tinfo[kMaxTasks];
#pragma unroll
            for (int ti_ = 0; ti_ < kMaxTasks; ++ti_) {
                const int task = warp + ti_ * kProducerWarps;
                int x = task;
                const int part = x % kSplit;
                x /= kSplit;
                const int cgrp = x % (C::NG / 4);
                x /= (C::NG / 4);
                const int kg = x % KG;
                const int op = x / KG;
                TaskInfo& T = tinfo[ti_];
                T.op = op;
                T.k = kg * 8 + (lane & 7);
                T.g = cgrp * 4 + (lane >> 3);
                int plo, phi;
                pair_range(op ? tj : ti, plo, phi);
                const int np = phi - plo + 1;
                T.plo = plo;
                T.pb = plo + (np * part) / kSplit;
                T.pe = plo + (np * (part + 1)) / kSplit;
                T.base = (op ? tj : ti) * kTile;
            }
            for (int kc = 0; kc < nK; ++kc, ++gs) {
                const int st = gs & (kStages - 1);
                const int buf = gs % nstg;
                const uint32_t ph = (uint32_t)((gs / kStages) & 1);
                const bool ok = tc::mbar_wait(&empty[st], ph ^ 1u, kWaitLimit);
                if (!ok) fail(1);
                // this stage's group is the oldest of the nstg-1 in flight
                if (nstg >= 4) asm volatile("cp.async.wait_group 2;" ::: "memory");
                else if (nstg == 3) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else cp_async_wait_all();
                if (producers_any(!ok || *abort_flag)) { stop = true; break; }
                // the buffer of stage gs+nstg-1 was last read by stage gs-1's generation,
                // which every producer finished before the barrier above
                issue_next((gs + nstg - 1) % nstg);
                const float* P = stg0 + buf * stg_floats;
                const float* U3s = P + 2 * halfp * C::PSTRIDE;
                unsigned char* sbase = smem + st * C::STAGE_BYTES;
                for (int ti_ = 0; ti_ < kMaxTasks; ++ti_) {
                    const int task = warp + ti_ * kProducerWarps;
                    if (task >= ntasks) break;
                    const TaskInfo& T = tinfo[ti_];
                    const int op = T.op, k = T.k, g = T.g, plo = T.plo, pb = T.pb, pe = T.pe, base = T.base;
                    float u3v[C::QPC];
#pragma unroll
                    for (int e = 0; e < C::QPC; e += 4) {
                        const float4 x4 = k < r3 ? *reinterpret_cast<const float4*>(U3s + k * C::PSTRIDE + g * C::QPC + e)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                        u3v[e] = x4.x; u3v[e + 1] = x4.y; u3v[e + 2] = x4.z; u3v[e + 3] = x4.w;
                    }
                    unsigned char* tile = sbase + op * C::PARTS * C::TILE_BYTES;
                    const float* Pop = P + (op ? halfp : 0) * C::PSTRIDE;
                    for (int p = pb; p < pe; ++p) {
                        const int row = p * r3 + k - base;
                        if (k >= r3 || row < 0 || row >= kTile) continue;
                        const float* pr = Pop + (p - plo) * C::PSTRIDE + g * C::QPC;
                        float v[C::QPC];
#pragma unroll
                        for (int e = 0; e < C::QPC; e += 4) {
                            const float4 x4 = *reinterpret_cast<const float4*>(pr + e);
                            v[e] = x4.x * u3v[e];
                            v[e + 1] = x4.y * u3v[e + 1];
                            v[e + 2] = x4.z * u3v[e + 2];
                            v[e + 3] = x4.w * u3v[e + 3];
                        }
                        const uint32_t off = tc::kmajor_offset(row, g * 16, C::KB);
                        if (MODE == kTF32) {
                            *reinterpret_cast<uint4*>(tile + off) =
                                make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
                        } else {
                            *reinterpret_cast<uint4*>(tile + off) =
                                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                           pack_bf16(v[6], v[7]));
                            if (MODE == kBF16X3) {
                                float lo[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) lo[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
                                *reinterpret_cast<uint4*>(tile + C::TILE_BYTES + off) =
                                    make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                                               pack_bf16(lo[6], lo[7]));
                            }
                        }
                    }
                }
                // operand rows beyond R (last tiles only) are zero in every stage
                for (int op = 0; op < 2; ++op) {
                    const int base = (op ? tj : ti) * kTile;
                    const int first = R - base;
                    if (first >= kTile) continue;
                    unsigned char* tile = sbase + op * C::PARTS * C::TILE_BYTES;
                    const int nz = (kTile - (first > 0 ? first : 0)) * C::NG;
                    for (int e = tid; e < nz; e += kProducerWarps * 32) {
                        const int row = (first > 0 ? first : 0) + e / C::NG, g = e % C::NG;
                        const uint32_t off = tc::kmajor_offset(row, g * 16, C::KB);
                        *reinterpret_cast<uint4*>(tile + off) = make_uint4(0, 0, 0, 0);
                        if (MODE == kBF16X3) *reinterpret_cast<uint4*>(tile + C::TILE_BYTES + off) = make_uint4(0, 0, 0, 0);
                    }
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&full[st]);
            }
            if (stop) break;
            // ---------------------------------------------------------- epilogue
            if (warp >= kEpilogueWarps) continue;
            if (!tc::mbar_wait(tmem_full, (uint32_t)(tcount & 1), kWaitLimit)) fail(2);
            tc::fence_after_sync();
            const int hh = warp >> 2;                   // accumulator 0: rows 0..127, 1: rows 128..255
            const int sub = warp & 3;                   // TMEM lanes 32*sub .. 32*sub+31
            const int row = ti * kTile + hh * 128 + sub * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(hh * 256);
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
        cp_async_wait_all();
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        constexpr uint32_t idesc = MODE == kTF32 ? tc::idesc_tf32(128, 256) : tc::idesc_bf16(128, 256);
        constexpr uint32_t SBO = (C::KB / 16) * 128;
        int gs = 0;
        int tcount = 0;
        bool issued = false;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tcount) {
            if (!tc::mbar_wait(tmem_empty, (uint32_t)(tcount & 1) ^ 1u, kWaitLimit)) { fail(4); break; }
            tc::fence_after_sync();
            for (int kc = 0; kc < nK; ++kc, ++gs) {
                const int st = gs & (kStages - 1);
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

// PT[(i r2 + j) mpad + q] = w1_i(q) w2_j(q) and U3T[k mpad + q] = w3_k(q) (zero for q >= m):
// the factor values of the sampled rows rearranged pair-major for 16-byte stage copies.
__global__ void pair_products_kernel(const float* __restrict__ U1, const float* __restrict__ U2,
                                     const float* __restrict__ U3, int64_t m, int64_t mpad, int r1, int r2, int r3,
                                     float* __restrict__ PT, float* __restrict__ U3T) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < mpad; q += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = q < m;
        for (int k = 0; k < r3; ++k) U3T[(size_t)k * mpad + q] = ok ? U3[q * r3 + k] : 0.f;
        for (int i = 0; i < r1; ++i) {
            const float a = ok ? U1[q * r1 + i] : 0.f;
            for (int j = 0; j < r2; ++j) PT[(size_t)(i * r2 + j) * mpad + q] = ok ? a * U2[q * r2 + j] : 0.f;
        }
    }
}

template <int MODE>
fst_status launch(const float* PT, const float* U3T, int64_t m, int64_t mpad, int r1, int r2, int r3, float* G,
                  int* err, cudaStream_t s) {
    using C = Cfg<MODE>;
    auto kern = gram_tc_kernel<MODE>;
    const int halfp = (kTile - 1) / r3 + 2;                  // pairs one 256-row tile can span
    const size_t stg_bytes = (size_t)(2 * halfp + r3) * C::PSTRIDE * 4;
    const size_t limit = 227 * 1024;
    int nstg = 4;
    while (nstg > 2 && C::FIXED + nstg * stg_bytes > limit) --nstg;
    const size_t smem = C::FIXED + nstg * stg_bytes;
    if (smem > limit) {
        set_error("tensor-core Gram: ranks need %zu bytes of shared memory", smem);
        return FST_EUNSUPPORTED;
    }
    FST_TRY(allow_smem(kern, smem));
    const int R = r1 * r2 * r3;
    const long long nT = (R + kTile - 1) / kTile;
    const long long ntiles = nT * (nT + 1) / 2;
    int grid = sm_count();
    if (ntiles < grid) grid = (int)ntiles;
    kern<<<grid, kThreads, smem, s>>>(PT, U3T, m, mpad, r1, r2, r3, halfp, nstg, G, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

ScratchPool g_gram_tc[64];   // per device: PT, U3T

}  // namespace

fst_status pair_products(const float* U1, const float* U2, const float* U3, int64_t m, int64_t mpad, int r1, int r2,
                         int r3, float* PT, float* U3T, cudaStream_t s) {
    int grid = (int)((mpad + 255) / 256);
    if (grid > 8 * sm_count()) grid = 8 * sm_count();
    pair_products_kernel<<<grid, 256, 0, s>>>(U1, U2, U3, m, mpad, r1, r2, r3, PT, U3T);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

fst_status gram_tc_launch(const fst_model* M, const float* U1, const float* U2, const float* U3, int64_t m,
                          float* G, fst_prec prec, cudaStream_t s) {
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    const int r1 = M->r[0], r2 = M->r[1], r3 = M->r[2];
    if (r3 < 4) {
        set_error("tensor-core Gram needs r3 >= 4");
        return FST_EUNSUPPORTED;
    }
    // the error word is the model's (the caller holds the model's lock)
    DevBuf& eb = const_cast<fst_model*>(M)->rs.gram_err;
    FST_TRY(eb.ensure(sizeof(int)));
    int* err = eb.as<int>();
    {
        SlotLease lease(g_gram_tc[dev & 63]);
        FST_TRY(lease.begin(s));
        FST_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        const int64_t mpad = (m + 63) / 64 * 64;
        FST_TRY(lease.ensure(0, sizeof(float) * (size_t)r1 * r2 * mpad));
        FST_TRY(lease.ensure(1, sizeof(float) * (size_t)r3 * mpad));
        float* PT = lease.as<float>(0);
        float* U3T = lease.as<float>(1);
        FST_TRY(pair_products(U1, U2, U3, m, mpad, r1, r2, r3, PT, U3T, s));
        fst_status st;
        switch (prec) {
            case FST_TF32: st = launch<kTF32>(PT, U3T, m, mpad, r1, r2, r3, G, err, s); break;
            case FST_BF16: st = launch<kBF16>(PT, U3T, m, mpad, r1, r2, r3, G, err, s); break;
            case FST_BF16X3: st = launch<kBF16X3>(PT, U3T, m, mpad, r1, r2, r3, G, err, s); break;
            default:
                set_error("tensor-core Gram takes TF32, BF16 or BF16X3");
                return FST_EINVAL;
        }
        if (st != FST_OK) return st;
    }   // the lease records this stream's use of the slot
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
