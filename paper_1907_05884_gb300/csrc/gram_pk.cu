// gram_pk.cu -- normal matrix G = A^T A of the sampled least-squares problem (Sec. 5,
// eq. rand_core; Algorithm 2, solve step) from a packed copy of the Khatri-Rao operand.
//
// A_{s,a} = w1_i(y_s) w2_j(y_s) w3_k(y_s), a = (i j k) in C order.  Two launches:
//   1. pack: A^T is written once in the tensor-core operand format, as tiles of 128 rows
//      (a) x KT sampled rows (s) in the K-major no-swizzle core-matrix layout (tc_ptx.cuh):
//      BF16 (KT = 64), TF32 (KT = 32), or BF16 high and low planes (KT = 32 each) for the
//      BF16x3 products hi*hi + hi*lo + lo*hi.  Tile (plane p, chunk kc, row tile rt) sits at
//      ((p * nkc + kc) * nrt + rt) * TILE, so the two row tiles of a 256-row operand are one
//      contiguous block; rows a >= R and sampled rows s >= m are zero.
//   2. GEMM: persistent, one CTA per SM, 256 x 256 lower super-tiles (two M = 128, N = 256
//      accumulators = all 512 TMEM columns).  Warp 0 moves each stage's operands with bulk
//      copies (one per operand and plane), warp 1 issues the MMAs, warps 2-5 read the
//      accumulators back and store G.  Every CTA walks its n-th tile at the same time as the
//      others and streams the sampled rows in the same order, so each K-chunk of the packed
//      operand (nrt tiles) is read from DRAM once and then served from L2.
// Every wait is bounded (~1 s); on expiry the kernel records an error and drains.
#include <cuda_bf16.h>

#include "fst_internal.cuh"
#include "tc_ptx.cuh"

namespace fst {

namespace {

constexpr int kStagesP = 3;
constexpr int kThreadsP = 6 * 32;                  // producer, MMA, 4 epilogue warps
constexpr uint32_t kStageBytesP = 65536;           // A pair + B pair, all planes
constexpr long long kWaitLimitP = 2000000000LL;

enum PMode { pTF32 = 0, pBF16 = 1, pBF16X3 = 2 };

template <int MODE>
struct PCfg {
    static constexpr int PLANES = MODE == pBF16X3 ? 2 : 1;
    static constexpr int RB = MODE == pBF16X3 ? 64 : 128;          // row bytes of a tile (per plane)
    static constexpr int ES = MODE == pTF32 ? 4 : 2;               // element bytes
    static constexpr int KT = RB / ES;                              // sampled rows per tile
    static constexpr int EPC = 16 / ES;                             // elements per 16-byte chunk
    static constexpr int NCH = RB / 16;                             // chunks per tile row
    static constexpr uint32_t TILE = 128 * RB;                      // bytes of one tile (plane)
    static constexpr uint32_t SBO = (RB / 16) * 128;                // row-group stride
    static constexpr int KSTEPS = RB / 32;                          // MMAs per tile per product
};

__device__ __forceinline__ uint32_t pk_bf16x2(float a, float b) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
}
__device__ __forceinline__ uint32_t pk_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// One thread per 16-byte chunk of a tile, in memory order.  PT[(i r2 + j) mpad + s] =
// w1_i w2_j and U3T[k mpad + s] = w3_k of sampled row s (zero for s >= m).
template <int MODE>
__global__ void __launch_bounds__(256) pack_kr_kernel(const float* __restrict__ PT, const float* __restrict__ U3T,
                                                      int64_t mpad, int r3, int R, int nrt, int nkc,
                                                      unsigned char* __restrict__ out) {
    using C = PCfg<MODE>;
    const int64_t per_tile = 128 * C::NCH;
    const int64_t total = (int64_t)nkc * nrt * per_tile;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = e / per_tile;            // kc * nrt + rt
        const int u = (int)(e - tile * per_tile);
        const int kc = (int)(tile / nrt), rt = (int)(tile - (int64_t)kc * nrt);
        const int rr = u & 7, c = (u >> 3) % C::NCH, g = (u >> 3) / C::NCH;
        const int a = rt * 128 + g * 8 + rr;
        const int64_t s0 = (int64_t)kc * C::KT + c * C::EPC;
        float v[C::EPC];
        if (a < R) {
            const int pair = a / r3, k = a - pair * r3;
            const float* p = PT + (size_t)pair * mpad + s0;
            const float* w = U3T + (size_t)k * mpad + s0;
#pragma unroll
            for (int q = 0; q < C::EPC; ++q) v[q] = p[q] * w[q];
        } else {
#pragma unroll
            for (int q = 0; q < C::EPC; ++q) v[q] = 0.f;
        }
        const size_t off = (size_t)tile * C::TILE + (size_t)u * 16;
        if (MODE == pTF32) {
            *reinterpret_cast<uint4*>(out + off) = make_uint4(pk_tf32(v[0]), pk_tf32(v[1]), pk_tf32(v[2]), pk_tf32(v[3]));
        } else {
            *reinterpret_cast<uint4*>(out + off) =
                make_uint4(pk_bf16x2(v[0], v[1]), pk_bf16x2(v[2], v[3]), pk_bf16x2(v[4], v[5]), pk_bf16x2(v[6], v[7]));
            if (MODE == pBF16X3) {
                float l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) l[q] = v[q] - __bfloat162float(__float2bfloat16_rn(v[q]));
                const size_t plane = (size_t)nkc * nrt * C::TILE;
                *reinterpret_cast<uint4*>(out + plane + off) =
                    make_uint4(pk_bf16x2(l[0], l[1]), pk_bf16x2(l[2], l[3]), pk_bf16x2(l[4], l[5]), pk_bf16x2(l[6], l[7]));
            }
        }
    }
}

constexpr int kStripP = 12;   // super-tile columns of a strip (about sqrt of the CTA count)

template <int MODE>
__global__ void __launch_bounds__(kThreadsP, 1)
gram_pk_kernel(const unsigned char* __restrict__ pk, int R, int nrt, int nkc, float* __restrict__ G,
               int* __restrict__ err) {
    using C = PCfg<MODE>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStagesP * kStageBytesP);
    uint64_t* empty = full + kStagesP;
    uint64_t* tmem_full = empty + kStagesP;
    uint64_t* tmem_empty = tmem_full + 1;
    uint64_t* drain = tmem_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nT = nrt / 2;
    const long long ntiles = (long long)nT * (nT + 1) / 2;
    const size_t plane_bytes = (size_t)nkc * nrt * C::TILE;

    if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
    if (tid == 0) {
        for (int s = 0; s < kStagesP; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tmem_full, 1);
        tc::mbar_init(tmem_empty, 4);
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
    // Super-tile t of the lower triangle, in strips of kStripP columns: strip s holds the tiles
    // with tj in [s S, s S + W), first its triangle (rows s S .. s S + W - 1), then W tiles a
    // row below.  The 152 tiles a wave of CTAs works on then span about 12 rows and 12 columns,
    // so a wave streams about half of the operand's row blocks instead of all of them.
    auto tile_of = [&](long long t, int& ti, int& tj) {
        int s0 = 0;
        for (;;) {
            const int W = nT - s0 < kStripP ? nT - s0 : kStripP;
            const long long tri = (long long)W * (W + 1) / 2;
            const long long cnt = tri + (long long)(nT - s0 - W) * W;
            if (t < cnt) {
                if (t < tri) {
                    int x = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
                    while ((long long)(x + 1) * (x + 2) / 2 <= t) ++x;
                    while ((long long)x * (x + 1) / 2 > t) --x;
                    ti = s0 + x;
                    tj = s0 + (int)(t - (long long)x * (x + 1) / 2);
                } else {
                    const long long u = t - tri;
                    ti = s0 + W + (int)(u / W);
                    tj = s0 + (int)(u % W);
                }
                return;
            }
            t -= cnt;
            s0 += W;
        }
    };

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                int ti, tj;
                tile_of(t, ti, tj);
                const bool diag = ti == tj;
                const uint32_t half = 2 * C::TILE;           // one 256-row operand in one plane
                const uint32_t bytes = (diag ? 1u : 2u) * C::PLANES * half;
                for (int kc = 0; kc < nkc; ++kc, ++it) {
                    const int s = it % kStagesP;
                    const uint32_t ph = (uint32_t)((it / kStagesP) & 1);
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, kWaitLimitP)) {
                        fail(1);
                        break;
                    }
                    unsigned char* st = smem + s * kStageBytesP;
                    tc::mbar_arrive_expect_tx(&full[s], bytes);
                    const size_t a_off = ((size_t)kc * nrt + 2 * ti) * C::TILE;
                    const size_t b_off = ((size_t)kc * nrt + 2 * tj) * C::TILE;
#pragma unroll
                    for (int p = 0; p < C::PLANES; ++p) {
                        tc::bulk_g2s(st + p * half, pk + p * plane_bytes + a_off, half, &full[s]);
                        if (!diag)
                            tc::bulk_g2s(st + (C::PLANES + p) * half, pk + p * plane_bytes + b_off, half, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = MODE == pTF32 ? tc::idesc_tf32(128, 256) : tc::idesc_bf16(128, 256);
            int it = 0, tcount = 0;
            bool issued = false;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tcount) {
                int ti, tj;
                tile_of(t, ti, tj);
                const bool diag = ti == tj;
                if (!tc::mbar_wait(tmem_empty, (uint32_t)(tcount & 1) ^ 1u, kWaitLimitP)) {
                    fail(4);
                    break;
                }
                tc::fence_after_sync();
                bool ok = true;
                for (int kc = 0; kc < nkc; ++kc, ++it) {
                    const int s = it % kStagesP;
                    const uint32_t ph = (uint32_t)((it / kStagesP) & 1);
                    if (!tc::mbar_wait(&full[s], ph, kWaitLimitP)) {
                        fail(8);
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t half = 2 * C::TILE;
                    const uint32_t abase = tc::smem_u32(smem + s * kStageBytesP);
                    const uint32_t bbase = diag ? abase : abase + C::PLANES * half;
#pragma unroll
                    for (int ks = 0; ks < C::KSTEPS; ++ks) {
                        const uint32_t ko = ks * 256;
                        const uint64_t bh = tc::make_desc(bbase + ko, 128, C::SBO);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                            const uint64_t ah = tc::make_desc(abase + h * C::TILE + ko, 128, C::SBO);
                            const uint32_t d = tmem + (uint32_t)(h * 256);
                            if (MODE == pTF32) {
                                tc::mma_tf32(d, ah, bh, idesc, acc);
                            } else {
                                tc::mma_bf16(d, ah, bh, idesc, acc);
                                if (MODE == pBF16X3) {
                                    const uint64_t al = tc::make_desc(abase + half + h * C::TILE + ko, 128, C::SBO);
                                    const uint64_t bl = tc::make_desc(bbase + half + ko, 128, C::SBO);
                                    tc::mma_bf16(d, ah, bl, idesc, 1u);
                                    tc::mma_bf16(d, al, bh, idesc, 1u);
                                }
                            }
                        }
                    }
                    tc::mma_commit(&empty[s]);
                    issued = true;
                }
                if (!ok || *abort_flag) break;
                tc::mma_commit(tmem_full);
            }
            if (issued) {
                // every MMA of this CTA completes before tensor memory is released
                tc::mma_commit(drain);
                if (!tc::mbar_wait(drain, 0u, kWaitLimitP)) atomicOr(err, 16);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int quarter = warp & 3;                    // TMEM lanes 32*quarter .. +31
        int tcount = 0;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tcount) {
            int ti, tj;
            tile_of(t, ti, tj);
            const bool diag = ti == tj;
            if (!tc::mbar_wait(tmem_full, (uint32_t)(tcount & 1), kWaitLimitP)) {
                fail(2);
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = ti * 256 + h * 128 + quarter * 32 + lane;
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(h * 256);
                for (int c0 = 0; c0 < 256; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(taddr + c0, v);
                    tc::tmem_wait_ld();
                    const int col = tj * 256 + c0;
                    if (row >= R || (diag && col > row)) continue;
                    float* dst = G + (size_t)row * R + col;
                    if (!diag && col + 16 <= R && (R & 3) == 0) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (col + e < R && (!diag || col + e <= row)) dst[e] = v[e];
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tmem_empty);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

ScratchPool g_pk[64];   // per device: PT, U3T, the packed operand

template <int MODE>
fst_status pack_and_multiply(const float* PT, const float* U3T, int64_t m, int64_t mpad, int r3, int R,
                             SlotLease& lease, float* G, int* err, cudaStream_t s) {
    using C = PCfg<MODE>;
    const int nrt = 2 * ((R + 255) / 256);
    const int nkc = (int)((m + C::KT - 1) / C::KT);
    const size_t bytes = (size_t)C::PLANES * nkc * nrt * C::TILE;
    FST_TRY(lease.ensure(2, bytes));
    unsigned char* packed = lease.as<unsigned char>(2);
    {
        const int64_t total = (int64_t)nkc * nrt * 128 * C::NCH;
        int64_t grid = (total + 255) / 256;
        if (grid > 16LL * sm_count()) grid = 16LL * sm_count();
        pack_kr_kernel<MODE><<<(unsigned)grid, 256, 0, s>>>(PT, U3T, mpad, r3, R, nrt, nkc,
                                                            packed);
        FST_CHECK_LAUNCH();
    }
    auto kern = gram_pk_kernel<MODE>;
    const size_t smem = kStagesP * kStageBytesP + 1024 + 1024;
    FST_TRY(allow_smem(kern, smem));
    const long long nT = nrt / 2;
    const long long ntiles = nT * (nT + 1) / 2;
    int grid = sm_count();
    if (ntiles < grid) grid = (int)ntiles;
    kern<<<grid, kThreadsP, smem, s>>>(packed, R, nrt, nkc, G, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

}  // namespace

// G (lower triangle) of the sampled rows from the packed operand; same contract as
// gram_tc_launch.  FST_ENOMEM if the packed copy does not fit (the caller may then use the
// on-the-fly kernel).
fst_status gram_pk_launch(const fst_model* M, const float* U1, const float* U2, const float* U3, int64_t m,
                          float* G, fst_prec prec, cudaStream_t s) {
    // the error word is the model's (the caller holds the model's lock)
    DevBuf& eb = const_cast<fst_model*>(M)->rs.gram_err;
    FST_TRY(eb.ensure(sizeof(int)));
    return gram_pk_rows(U1, U2, U3, m, M->r[0], M->r[1], M->r[2], G, prec, eb.as<int>(), s);
}

// The same for rows A_s = u1_s (x) u2_s (x) u3_s given as three factor arrays (m x r_k each;
// u3 may itself be a Kronecker product of further factors, as for order-4 models).
fst_status gram_pk_rows(const float* U1, const float* U2, const float* U3, int64_t m, int r1, int r2, int r3,
                        float* G, fst_prec prec, int* err, cudaStream_t s) {
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    {
        SlotLease lease(g_pk[dev & 63]);
        FST_TRY(lease.begin(s));
        FST_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        const int R = r1 * r2 * r3;
        const int64_t mpad = (m + 63) / 64 * 64;
        FST_TRY(lease.ensure(0, sizeof(float) * (size_t)r1 * r2 * mpad));
        FST_TRY(lease.ensure(1, sizeof(float) * (size_t)r3 * mpad));
        float* PT = lease.as<float>(0);
        float* U3T = lease.as<float>(1);
        FST_TRY(pair_products(U1, U2, U3, m, mpad, r1, r2, r3, PT, U3T, s));
        fst_status st;
        switch (prec) {
            case FST_TF32: st = pack_and_multiply<pTF32>(PT, U3T, m, mpad, r3, R, lease, G, err, s); break;
            case FST_BF16: st = pack_and_multiply<pBF16>(PT, U3T, m, mpad, r3, R, lease, G, err, s); break;
            case FST_BF16X3: st = pack_and_multiply<pBF16X3>(PT, U3T, m, mpad, r3, R, lease, G, err, s); break;
            default:
                set_error("packed Gram takes TF32, BF16 or BF16X3");
                return FST_EINVAL;
        }
        if (st != FST_OK) return st;
    }   // the lease records this stream's use of the slot
    int herr = 0;
    FST_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FST_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("packed Gram: a bounded device wait expired (code %d)", herr);
        return FST_ETIMEOUT;
    }
    return FST_OK;
}

}  // namespace fst
