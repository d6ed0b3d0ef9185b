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

#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <memory>
#include <tuple>
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
// factor-step (pipelined) variant: contraction chunks of at most 144 columns
__host__ __device__ constexpr int jc3_for(int r3p) { return 144 / r3p; }
constexpr int kFacRows = 32;           // ranks padded to 32 in each coefficient part of the factor MMA
constexpr int kBarBytes = 1024;

// Host-side description of the shared-memory image of C_(1) (and, for the factor-step
// variant, of the three factor coefficient matrices behind it).
struct CoreImage {
    int mode, r3p, jc, nc, ncp, kp, kb, nchunks, parts;
    size_t chunk_bytes, bytes;
    bool tc3 = false;
    int rm = 8;                  // rank bound of the size class (K stride of the BF16X3 operand)
    int kpf = 0;                 // Legendre K of the factor MMA (multiple of 32)
    size_t fac_off = 0, fac_bytes = 0;
};

int bucket8(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 24 ? 24 : 32; }

int kpf_of(const fst_model* m) {
    const int pe = std::max(m->p_eff[0], std::max(m->p_eff[1], m->p_eff[2]));
    return std::max(32, (pe + 31) / 32 * 32);
}

__host__ __device__ constexpr int pipe_kc(int mode, int rm);
__host__ __device__ constexpr int pipe_kb(int mode, int rm);

CoreImage core_image_shape(const fst_model* m, int mode, int r3p, bool tc3 = false) {
    CoreImage c;
    c.mode = mode;
    c.r3p = r3p;
    c.tc3 = tc3;
    c.jc = tc3 ? jc3_for(r3p) : jc_for(r3p);
    c.nc = c.jc * r3p;
    c.ncp = (c.nc + 15) / 16 * 16;
    c.rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    const int gran = mode == eTF32 ? 8 : 16;
    c.kp = (m->r[0] + gran - 1) / gran * gran;
    c.kb = c.kp * (mode == eTF32 ? 4 : 2);
    c.parts = mode == eBF16X3 ? 2 : 1;
    if (tc3) {
        // one part: BF16X3 concatenates [C hi; C hi; C lo] along K with stride rm
        c.kp = pipe_kc(mode, c.rm);
        c.kb = pipe_kb(mode, c.rm);
        c.parts = 1;
    }
    c.nchunks = (m->r[1] + c.jc - 1) / c.jc;
    c.chunk_bytes = (size_t)c.ncp * c.kb;
    c.bytes = c.chunk_bytes * c.nchunks * c.parts;
    if (tc3) {
        c.kpf = kpf_of(m);
        c.fac_off = (c.bytes + 1023) & ~(size_t)1023;
        c.fac_bytes = (size_t)3 * 3 * kFacRows * c.kpf * 2;      // three modes, hi | mid | lo
        c.bytes = c.fac_off + c.fac_bytes;
    }
    return c;
}

// Shared memory of a pipelined bucket: alignment slack, the control block, the core and factor
// images, nps Legendre half-tile slots (BF16 hi + lo, 128 x 32) per basis group, and the w1
// operand (128 x KB).
size_t tc3_smem(size_t core_max, int kb_max, int nps) {
    return 1024 + kBarBytes + core_max + (size_t)2 * nps * (2 * 128 * 32 * 2) + (size_t)128 * kb_max;
}
// Two half-tile slots per basis group when they fit.
int tc3_nps(size_t core_max, int kb_max) { return tc3_smem(core_max, kb_max, 2) <= 227 * 1024 ? 2 : 1; }

// The factor-step variant can serve contractions (TF32, BF16, BF16X3) with degrees below 64
// whose images fit the shared memory.
bool tc3_feasible(const fst_model* m, int mode, int r3p) {
    if (kpf_of(m) > 64 || m->wav_s >= 0) return false;   // wavelet columns: factor values on the CUDA cores
    const CoreImage c = core_image_shape(m, mode, r3p, true);
    return tc3_smem((c.bytes + 1023) & ~(size_t)1023, c.kb, 1) <= 227 * 1024;
}

// Autotune table: per device and size class (mode, rank bound, r3 padding, Legendre K) the
// evaluator variant measured fastest (0: factor values on the CUDA cores, 1: on the tensor
// cores).  Classes not measured take the factor-step variant when it is feasible.
struct TuneKey {
    int mode, rm, r3p, kpf;
    bool operator<(const TuneKey& o) const {
        return std::tie(mode, rm, r3p, kpf) < std::tie(o.mode, o.rm, o.r3p, o.kpf);
    }
};
struct TuneTable {
    std::mutex mu;
    std::map<TuneKey, int> choice;
};
TuneTable g_tune[64];
thread_local int t_force_variant = -1;   // set while the autotuner probes a variant

TuneKey tune_key(const fst_model* m, int mode, int r3p) {
    const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    return TuneKey{mode, rm, r3p, kpf_of(m)};
}

bool use_tc3(const fst_model* m, int mode, int r3p) {
    if (!tc3_feasible(m, mode, r3p)) return false;
    if (t_force_variant >= 0) return t_force_variant == 1;
    int dev = 0;
    cudaGetDevice(&dev);
    TuneTable& T = g_tune[dev & 63];
    std::lock_guard<std::mutex> lk(T.mu);
    auto it = T.choice.find(tune_key(m, mode, r3p));
    return it == T.choice.end() ? true : it->second == 1;
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
    if (c.tc3) {
        // pipelined variant: one part; BF16X3 holds C hi at K = i and rm + i, C lo at 2 rm + i
        for (int ch = 0; ch < c.nchunks; ++ch)
            for (int n = 0; n < c.nc; ++n) {
                const int j = ch * c.jc + n / c.r3p, k = n % c.r3p;
                if (j >= r2 || k >= r3) continue;
                unsigned char* base = img.data() + (size_t)ch * c.chunk_bytes;
                for (int i = 0; i < r1; ++i) {
                    const double v = m->alpha[((size_t)i * r2 + j) * r3 + k];
                    if (c.mode == eTF32) {
                        const uint32_t b = tf32_bits((float)v);
                        memcpy(base + tc::kmajor_offset(n, i * 4, c.kb), &b, 4);
                        continue;
                    }
                    const uint16_t hi = bf16_bits((float)v);
                    memcpy(base + tc::kmajor_offset(n, i * 2, c.kb), &hi, 2);
                    if (c.mode == eBF16X3) {
                        const uint16_t lo = bf16_bits((float)(v - (double)bf16_val((float)v)));
                        memcpy(base + tc::kmajor_offset(n, (c.rm + i) * 2, c.kb), &hi, 2);
                        memcpy(base + tc::kmajor_offset(n, (2 * c.rm + i) * 2, c.kb), &lo, 2);
                    }
                }
            }
        // factor coefficient matrices with sqrt(2n+1) and the leading coefficient k_n of L_n
        // folded in (the kernel's Legendre tiles hold L_n / k_n), split in three BF16 parts:
        // mode k, row part * 32 + j (rank j), K = degree n (padded to kpf)
        const int KPB = c.kpf * 2;
        const size_t wbytes = (size_t)3 * kFacRows * KPB;
        std::vector<double> lead(c.kpf, 1.0);     // k_n = prod_{i <= n} (2i - 1) / i
        for (int nn = 1; nn < c.kpf; ++nn) lead[nn] = lead[nn - 1] * (2.0 * nn - 1.0) / nn;
        for (int k = 0; k < 3; ++k) {
            unsigned char* base = img.data() + c.fac_off + (size_t)k * wbytes;
            for (int j = 0; j < m->r[k]; ++j)
                for (int e = m->colptr[k][j]; e < m->colptr[k][j + 1]; ++e) {
                    const int nn = m->rowidx[k][e];
                    if (nn >= c.kpf) continue;
                    double w = m->val[k][e] * sqrt(2.0 * nn + 1.0) * lead[nn];
                    for (int part = 0; part < 3; ++part) {
                        const uint16_t b = bf16_bits((float)w);
                        memcpy(base + tc::kmajor_offset(part * kFacRows + j, nn * 2, KPB), &b, 2);
                        w -= (double)bf16_val((float)w);
                    }
                }
        }
        return img;
    }
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

// One evaluation instance as the kernel sees it.
struct TcItem {
    EvalArgs<float> a;
    const unsigned char* core_img;   // operand image of C_(1) (device)
    int img_bytes, nchunks, kp, tab_bytes;
    int fac_off, kpf;                // factor-step variant: offset of the Wc images, Legendre K
    const float* xyz;
    float* out;
    long long n;
};
// A run of consecutive 128-point tiles of one instance.
struct TcUnit {
    int item, pad;
    long long tile0, ntiles;
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

// BF16 hi and lo words of the pair (a, b): hi = bf16(a, b), lo = bf16(a - hi_a, b - hi_b);
// the differences are exact in FP32 and taken two at a time.
__device__ __forceinline__ void split2_bf16(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pack2_bf16(a, b);
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), make_float2(a, b));
    lo = pack2_bf16(l.x, l.y);
}


// Persistent kernel over a work list of units (instance, tile range).  Block b takes the
// contiguous unit range [cta_start[b], cta_start[b+1]) (cut by estimated cost on the host);
// it reloads the core image and the factor tables into shared memory only when the
// instance changes.
template <int MODE, int R3P, int RM>
__global__ void __launch_bounds__(kThreadsE, 1)
eval_tc_kernel(const TcItem* __restrict__ items, const TcUnit* __restrict__ units, const int* __restrict__ cta_start,
               int core_max, int kb_max, const float* __restrict__ xyz_ov, float* __restrict__ out_ov,
               int* __restrict__ err) {
    constexpr int ES = MODE == eTF32 ? 4 : 2;
    constexpr int JC = jc_for(R3P);
    constexpr int NC = JC * R3P;
    constexpr int NCP = (NC + 15) / 16 * 16;
    constexpr int MAXCH = (FST_MAX_RANK + JC - 1) / JC;
    constexpr int PARTS = MODE == eBF16X3 ? 2 : 1;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint64_t* a_full = bars;                 // [kGroups] workers -> MMA: A tile written
    uint64_t* a_empty = bars + kGroups;      // [kGroups] MMA -> workers: A tile consumed
    uint64_t* d_full = bars + 2 * kGroups;   // [kGroups] MMA -> workers: chunk in TMEM
    uint64_t* d_empty = bars + 3 * kGroups;  // [kGroups] workers -> MMA: chunk read
    uint64_t* drain = bars + 4 * kGroups;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    unsigned char* core = smem + kBarBytes;
    unsigned char* abuf = core + core_max;                       // kGroups x PARTS x 128 x kb_max
    float* fsm = reinterpret_cast<float*>(abuf + kGroups * PARTS * 128 * kb_max);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
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
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int u0 = cta_start[blockIdx.x], u1 = cta_start[blockIdx.x + 1];
    int cur = -1;
    // per-role phase counters run across units
    int lt = 0, cc = 0;                          // worker group
    int mlt[kGroups] = {0, 0}, mcc[kGroups] = {0, 0};
    bool issued = false, dead = false;
    float *ra = nullptr, *rb = nullptr, *Ws0 = nullptr, *Ws1 = nullptr, *Ws2 = nullptr;
    uint8_t* mk = nullptr;
    for (int u = u0; u < u1; ++u) {
        const TcUnit U = units[u];
        const TcItem& I = items[U.item];
        const EvalArgs<float>& a = I.a;
        if (U.item != cur) {
            // every role has finished the previous instance: its MMAs completed before the
            // workers' last chunk wait, so shared memory can be refilled
            tc::fence_before_sync();
            __syncthreads();
            const uint4* src = reinterpret_cast<const uint4*>(I.core_img);
            uint4* dst = reinterpret_cast<uint4*>(core);
            for (int e = tid; e < I.img_bytes / 16; e += blockDim.x) dst[e] = src[e];
            ra = fsm;
            rb = ra + a.pm;
            Ws0 = rb + a.pm;
            Ws1 = Ws0 + a.pe[0] * RM;
            Ws2 = Ws1 + a.pe[1] * RM;
            mk = reinterpret_cast<uint8_t*>(Ws2 + a.pe[2] * RM);
            for (int i = tid; i < a.pm; i += blockDim.x) {
                ra[i] = float(2 * i + 1) / float(i + 1);
                rb[i] = float(i) / float(i + 1);
            }
            float* Wk[3] = {Ws0, Ws1, Ws2};
            for (int k = 0; k < 3; ++k) {
                const int rk = a.r[k];
                for (int e = tid; e < a.pe[k] * RM; e += blockDim.x) {
                    const int nn = e / RM, j = e - nn * RM;
                    Wk[k][e] = j < rk ? a.W[k][nn * rk + j] : 0.f;
                }
                for (int e = tid; e < a.pm; e += blockDim.x) mk[k * a.pm + e] = e < a.pe[k] ? a.mask[k][e] : 0;
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            cur = U.item;
        }
        const int KB = I.kp * ES;
        const int SBO = (KB / 16) * 128;
        const int abytes = 128 * KB;
        const int r1 = a.r[0];
        const int nch = I.nchunks;
        const long long n = I.n;
        if (warp < kWorkers) {
            // -------------------------------------------------------------- workers
            const int g = warp >> 2, sub = warp & 3, row = sub * 32 + lane;   // TMEM lane = row
            unsigned char* A = abuf + g * PARTS * 128 * kb_max;
            const float* X = xyz_ov ? xyz_ov : I.xyz;
            // coordinates of this group's next tile are loaded one tile ahead
            float nxt[3];
            {
                const long long q = (U.tile0 + g) * 128 + row;
                const bool ok = U.tile0 + g < U.tile0 + U.ntiles && q < n;
#pragma unroll
                for (int k = 0; k < 3; ++k) nxt[k] = ok ? X[k * n + q] : 0.f;
            }
            for (long long t = U.tile0 + g; t < U.tile0 + U.ntiles; t += kGroups, ++lt) {
                const long long q = t * 128 + row;
                const bool ok = q < n;
                float tt[3][1], yy[3][1];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    yy[k][0] = nxt[k];
                    tt[k][0] = fmaf(nxt[k], a.sc[k], a.of[k]);
                }
                {
                    const long long q2 = q + kGroups * 128;
                    const bool ok2 = t + kGroups < U.tile0 + U.ntiles && q2 < n;
#pragma unroll
                    for (int k = 0; k < 3; ++k) nxt[k] = ok2 ? X[k * n + q2] : 0.f;
                }
                float w[1][RM], u2[RM], u3[RM];
                factor_values<float, RM, 1>(tt[1], Ws1, mk + a.pm, a.pe[1], ra, rb, w);
                piecewise_values<float, RM, 1>(yy[1], tt[1], a, 1, w);
#pragma unroll
                for (int j = 0; j < RM; ++j) u2[j] = w[0][j];
                factor_values<float, RM, 1>(tt[2], Ws2, mk + 2 * a.pm, a.pe[2], ra, rb, w);
                piecewise_values<float, RM, 1>(yy[2], tt[2], a, 2, w);
#pragma unroll
                for (int j = 0; j < RM; ++j) u3[j] = j < a.r[2] ? w[0][j] : 0.f;
                factor_values<float, RM, 1>(tt[0], Ws0, mk, a.pe[0], ra, rb, w);   // w1 -> A operand
                piecewise_values<float, RM, 1>(yy[0], tt[0], a, 0, w);
                if (!tc::mbar_wait(&a_empty[g], (uint32_t)(lt & 1) ^ 1u, kWaitLimitE)) {
                    atomicOr(err, 1);
                    dead = true;
                }
                if (!dead) {
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
                            float h[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int i = c16 * 8 + e;
                                h[e] = (i < RM && i < r1) ? w[0][i < RM ? i : 0] : 0.f;
                            }
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) split2_bf16(h[2 * e], h[2 * e + 1], hw[e], lw[e]);
                            *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            if (MODE == eBF16X3)
                                *reinterpret_cast<uint4*>(A + abytes + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                    tc::fence_async_smem();
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&a_full[g]);
                const uint32_t tbase = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(g * 256);
                // Khatri-Rao epilogue, chunk by chunk: per j-slice s_j = sum_k T_(j,k) w3_k in
                // packed pairs of k (two independent accumulators), then f += s_j w2_j
                float2 u3p[RM / 2];
#pragma unroll
                for (int e = 0; e < RM / 2; ++e) u3p[e] = make_float2(u3[2 * e], u3[2 * e + 1]);
                float f = 0.f;
#pragma unroll
                for (int ch = 0; ch < MAXCH; ++ch) {
                    if (ch < nch) {
                        if (!tc::mbar_wait(&d_full[g], (uint32_t)(cc & 1), kWaitLimitE)) {
                            atomicOr(err, 2);
                            dead = true;
                        }
                        tc::fence_after_sync();
                        float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c0 = 0; c0 < NC; c0 += 48) {
                            float v[3][16];
#pragma unroll
                            for (int b = 0; b < 3; ++b)
                                if (c0 + 16 * b < NC) tc::tmem_ld16(tbase + c0 + 16 * b, v[b]);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int e = 0; e < 48; e += 2) {
                                const int col = c0 + e;
                                if (col < NC) {
                                    const int jl = col / R3P, k = col % R3P;
                                    const float2 vv = make_float2(v[e / 16][e % 16], v[e / 16][e % 16 + 1]);
                                    const float2 ww = u3p[k / 2 < RM / 2 ? k / 2 : 0];
                                    if ((k & 2) == 0)
                                        sa = __ffma2_rn(vv, ww, sa);
                                    else
                                        sb = __ffma2_rn(vv, ww, sb);
                                    if (k == R3P - 2) {
                                        const int j = ch * JC + jl;
                                        if (j < RM) f = fmaf((sa.x + sa.y) + (sb.x + sb.y), u2[j < RM ? j : 0], f);
                                        sa = make_float2(0.f, 0.f);
                                        sb = make_float2(0.f, 0.f);
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
                if (ok) (out_ov ? out_ov : I.out)[q] = f;
            }
        } else if (lane == 0 && !dead) {
            // -------------------------------------------------------------- MMA issuer
            constexpr uint32_t idesc = MODE == eTF32 ? tc::idesc_tf32(128, NCP) : tc::idesc_bf16(128, NCP);
            const int kst = KB / 32;
            const uint32_t core_u32 = tc::smem_u32(core);
            const uint32_t chunk_bytes = (uint32_t)(NCP * KB);
            for (long long t = U.tile0; t < U.tile0 + U.ntiles && !dead; ++t) {
                const int g = (int)((t - U.tile0) & 1);
                const uint32_t abase = tc::smem_u32(abuf + g * PARTS * 128 * kb_max);
                if (!tc::mbar_wait(&a_full[g], (uint32_t)(mlt[g] & 1), kWaitLimitE)) {
                    atomicOr(err, 4);
                    dead = true;
                    break;
                }
                tc::fence_after_sync();
                for (int ch = 0; ch < nch; ++ch) {
                    if (!tc::mbar_wait(&d_empty[g], (uint32_t)(mcc[g] & 1) ^ 1u, kWaitLimitE)) {
                        atomicOr(err, 8);
                        dead = true;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)(g * 256);
                    const uint32_t bb = core_u32 + ch * chunk_bytes;
                    for (int ks = 0; ks < kst; ++ks) {
                        const uint32_t ko = ks * 256;
                        const uint64_t ad = tc::make_desc(abase + ko, 128, SBO);
                        const uint64_t bd = tc::make_desc(bb + ko, 128, SBO);
                        if (MODE == eTF32) {
                            tc::mma_tf32(d, ad, bd, idesc, ks > 0);
                        } else {
                            tc::mma_bf16(d, ad, bd, idesc, ks > 0);
                            if (MODE == eBF16X3) {
                                const uint64_t al = tc::make_desc(abase + abytes + ko, 128, SBO);
                                const uint64_t bl = tc::make_desc(bb + nch * chunk_bytes + ko, 128, SBO);
                                tc::mma_bf16(d, ad, bl, idesc, 1u);
                                tc::mma_bf16(d, al, bd, idesc, 1u);
                            }
                        }
                    }
                    tc::mma_commit(&d_full[g]);
                    issued = true;
                    ++mcc[g];
                }
                if (dead) break;
                tc::mma_commit(&a_empty[g]);
                ++mlt[g];
            }
        }
    }
    if (warp == kWorkers && lane == 0 && issued) {
        tc::mma_commit(drain);
        if (!tc::mbar_wait(drain, 0u, kWaitLimitE)) atomicOr(err, 16);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- pipelined factor-step evaluator
// Variant for TF32 / BF16 / BF16X3 contractions with degrees below 64: the factor values are
// an MMA too, and the work of a 128-point tile flows through warp-specialised stages so that
// the Legendre arithmetic, the tensor cores and the Khatri-Rao epilogue of different tiles
// overlap:
//   * a scheduler warp publishes the CTA's tiles into a ring of descriptors (and loads the
//     core and factor images into shared memory when the instance changes);
//   * two basis groups of four warps (alternate tiles, thread = point) write the monic
//     Legendre values q_0..q_{pe-1} of every mode, 32 degrees at a time, as BF16 high and low
//     parts into half-tile slots;
//   * one thread issues the MMAs: per mode U_k = P_k Wc_k^T with Wc_k split in three BF16
//     parts side by side (N = 96: hi | mid | lo), so the hi and lo Legendre parts meet every
//     coefficient part (six products, FP32-class factor values), into a two-slot ring of
//     tensor-memory blocks; and T = U1 C_(1) in chunks of whole j-slices into two chunk
//     buffers.  It issues whichever job is ready first;
//   * four epilogue warps (thread = point = TMEM lane) add the three parts of each U block,
//     write w1 as the contraction's A operand (BF16X3: [hi | lo | hi] along K against
//     [C hi; C hi; C lo], one MMA chain for the three products), keep w2 and w3 in registers
//     and reduce each chunk against them.
// Every wait is bounded; on expiry a role records an error code and leaves its loop, and the
// others time out in turn.
constexpr int kPipeWarps = 15;                 // 0-7 basis, 8-11 epilogue, 12 factor MMAs, 13 scheduler, 14 contraction MMAs
constexpr int kThreadsP = kPipeWarps * 32;
constexpr int kND = 8;                         // tile descriptors in flight
constexpr int kUCols = 96;                     // factor MMA N: coefficient hi | mid | lo
constexpr int kChunkCols = 144;                // tensor-memory columns of a contraction chunk buffer
constexpr int kUBase = 2 * kChunkCols;         // the two U blocks follow the two chunk buffers
constexpr int kPHalf = 32;                     // Legendre degrees per half tile
constexpr int kPSlotBytes = 2 * 128 * kPHalf * 2;   // one half tile, BF16 hi + lo
constexpr int kEpiBatch = 3;                   // 16-column TMEM reads in flight per wait in the epilogue
// Register split: launched at 128 a thread (15 warps, 61,440 registers); the two basis
// warpgroups drop to 96 and the epilogue warpgroup rises to 176, warps 12-14 keep 128:
// 256 x 96 + 128 x 176 + 96 x 128 = 59,392 <= 61,440, and per SM sub-partition (warps w, w+4,
// w+8, w+12) at most 32 x (96 + 96 + 176 + 128) = 15,872 <= 16,384.
constexpr int kRegsLaunch = 128, kRegsBasis = 96, kRegsEpi = 176;
static_assert(256 * kRegsBasis + 128 * kRegsEpi + 96 * kRegsLaunch <= kThreadsP * kRegsLaunch, "register split");
static_assert(32 * (2 * kRegsBasis + kRegsEpi + kRegsLaunch) <= 16384, "register split per sub-partition");

struct PipeDesc {
    int item;            // < 0: no more tiles
    int pad;
    long long tile;
};
struct PipeCtl {
    uint64_t desc_full[kND], desc_empty[kND];
    uint64_t p_full[4], p_empty[4];
    uint64_t u_full[2], u_empty[2];
    uint64_t w1_full, w1_empty;
    uint64_t c_full[2], c_empty[2];
    uint64_t drain[2];                   // one per MMA thread
    PipeDesc desc[kND];
    TcItem item;         // the instance being evaluated (copied with its images)
    uint32_t tmem_base;
    int tiles_done;      // epilogue warps finished (one count per warp and tile)
};
static_assert(sizeof(PipeCtl) <= kBarBytes, "control block fits");

// N (a multiple of 8) consecutive TMEM columns of this warp's lanes into v; complete after
// tc::tmem_wait_ld()
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float* v) {
#pragma unroll
    for (int h = 0; h + 16 <= N; h += 16) {
        float t[16];
        tc::tmem_ld16(taddr + h, t);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[h + e] = t[e];
    }
    if (N % 16) {
        float t[8];
        tc::tmem_ld8(taddr + N / 16 * 16, t);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[N / 16 * 16 + e] = t[e];
    }
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc::smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// contraction K of the operand image: BF16X3 [hi | lo | hi] x [C hi; C hi; C lo] with rank
// stride RM, BF16 RM, TF32 RM; in elements, padded to the MMA's K granule
__host__ __device__ constexpr int pipe_kc(int mode, int rm) {
    return mode == eBF16X3 ? (3 * rm + 15) / 16 * 16 : mode == eBF16 ? (rm + 15) / 16 * 16 : (rm + 7) / 8 * 8;
}
__host__ __device__ constexpr int pipe_kb(int mode, int rm) { return pipe_kc(mode, rm) * (mode == eTF32 ? 4 : 2); }

template <int MODE, int R3P, int RM>
__global__ void __launch_bounds__(kThreadsP, 1)
eval_pipe_kernel(const TcItem* __restrict__ items, const TcUnit* __restrict__ units, const int* __restrict__ cta_start,
                 int nunits, int* unit_ctr, int core_max, int nps, const float* __restrict__ xyz_ov,
                 float* __restrict__ out_ov, int* __restrict__ err) {
    constexpr int JC = kChunkCols / R3P;
    constexpr int NC = JC * R3P;
    constexpr int NCP = (NC + 15) / 16 * 16;
    constexpr int MAXCH = (FST_MAX_RANK + JC - 1) / JC;
    constexpr int KB = pipe_kb(MODE, RM);
    constexpr uint32_t SBO_A = (KB / 16) * 128;
    static_assert(NCP <= kChunkCols, "a chunk fits its tensor-memory buffer");
    static_assert(kUBase + 2 * kUCols <= 512, "tensor-memory budget");

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    PipeCtl& C = *reinterpret_cast<PipeCtl*>(smem);
    unsigned char* core = smem + kBarBytes;
    unsigned char* pbuf = core + core_max;
    unsigned char* w1buf = pbuf + (size_t)2 * nps * kPSlotBytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 12) tc::tmem_alloc(&C.tmem_base, 512);
    if (tid == 0) {
        for (int e = 0; e < kND; ++e) {
            tc::mbar_init(&C.desc_full[e], 1);
            tc::mbar_init(&C.desc_empty[e], 10);   // basis group (4 warps), epilogue (4 warps), two MMA threads
        }
        for (int e = 0; e < 4; ++e) {
            tc::mbar_init(&C.p_full[e], 4);
            tc::mbar_init(&C.p_empty[e], 1);
        }
        for (int e = 0; e < 2; ++e) {
            tc::mbar_init(&C.u_full[e], 1);
            tc::mbar_init(&C.u_empty[e], 4);
            tc::mbar_init(&C.c_full[e], 1);
            tc::mbar_init(&C.c_empty[e], 4);
        }
        tc::mbar_init(&C.w1_full, 4);
        tc::mbar_init(&C.w1_empty, 1);
        tc::mbar_init(&C.drain[0], 1);
        tc::mbar_init(&C.drain[1], 1);
        C.tiles_done = 0;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = C.tmem_base;

    if (warp == 13) {
        // ------------------------------------------------------------ scheduler
        const int u0 = unit_ctr ? 0 : cta_start[blockIdx.x], u1 = unit_ctr ? nunits : cta_start[blockIdx.x + 1];
        int cur = -1;
        long long sd = 0;
        bool dead = false;
        for (int us = u0; !dead; ++us) {
            int u = us;
            if (unit_ctr) {
                if (lane == 0) u = atomicAdd(unit_ctr, 1);
                u = __shfl_sync(0xffffffffu, u, 0);
            }
            if (u >= u1) break;
            const TcUnit U = units[u];
            if (U.item != cur) {
                if (cur >= 0) {
                    // every tile of the previous instance is finished (its MMAs complete)
                    // before the images in shared memory are replaced
                    int ok = 1;
                    if (lane == 0) {
                        const long long t0 = clock64();
                        while (*reinterpret_cast<volatile int*>(&C.tiles_done) < 4 * sd) {
                            if (clock64() - t0 > kWaitLimitE) {
                                ok = 0;
                                break;
                            }
                            __nanosleep(256);
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, ok, 0)) {
                        if (lane == 0) atomicOr(err, 128);
                        dead = true;
                        break;
                    }
                }
                const TcItem& I = items[U.item];
                const uint4* src = reinterpret_cast<const uint4*>(I.core_img);
                uint4* dst = reinterpret_cast<uint4*>(core);
                for (int e = lane; e < I.img_bytes / 16; e += 32) dst[e] = src[e];
                // the instance's parameters next to the images: every role reads them from
                // shared memory (the descriptors published after this release them)
                static_assert(sizeof(TcItem) % 4 == 0, "item copied in words");
                for (int e = lane; e < (int)(sizeof(TcItem) / 4); e += 32)
                    reinterpret_cast<int*>(&C.item)[e] = reinterpret_cast<const int*>(&I)[e];
                tc::fence_async_smem();
                __syncwarp();
                cur = U.item;
            }
            for (long long t = U.tile0; t < U.tile0 + U.ntiles; ++t, ++sd) {
                const int slot = (int)(sd % kND);
                const uint32_t par = (uint32_t)((sd / kND) & 1) ^ 1u;
                int ok = 1;
                if (lane == 0) {
                    if (tc::mbar_wait(&C.desc_empty[slot], par, kWaitLimitE)) {
                        C.desc[slot].item = U.item;
                        C.desc[slot].tile = t;
                        tc::mbar_arrive(&C.desc_full[slot]);
                    } else {
                        atomicOr(err, 256);
                        ok = 0;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    dead = true;
                    break;
                }
            }
        }
        // two end markers: one for each basis group (the MMA thread and the epilogue stop at
        // the first)
        for (int e = 0; e < 2 && !dead && lane == 0; ++e, ++sd) {
            const int slot = (int)(sd % kND);
            if (tc::mbar_wait(&C.desc_empty[slot], (uint32_t)((sd / kND) & 1) ^ 1u, kWaitLimitE)) {
                C.desc[slot].item = -1;
                tc::mbar_arrive(&C.desc_full[slot]);
            } else {
                atomicOr(err, 256);
                dead = true;
            }
        }
    } else if (warp < 8) {
        // ------------------------------------------------------------ basis groups
        tc::setmaxnreg_dec<kRegsBasis>();
        const int g = warp >> 2, row = (warp & 3) * 32 + lane;
        int pi = 0;                    // this group's next half-tile slot (of nps) and its use parity
        uint32_t pph = 0;
        float nxt[3] = {0.f, 0.f, 0.f};
        long long nxt_seq = -1;
        for (long long sd = g;; sd += 2) {
            const int slot = (int)(sd % kND);
            if (!tc::mbar_wait(&C.desc_full[slot], (uint32_t)((sd / kND) & 1), kWaitLimitE)) {
                atomicOr(err, 1);
                break;
            }
            const PipeDesc d = C.desc[slot];
            if (d.item < 0) break;
            const TcItem& I = C.item;
            const EvalArgs<float>& a = I.a;
            const float* X = xyz_ov ? xyz_ov : I.xyz;
            const long long n = I.n;
            float x[3];
            if (nxt_seq == sd) {
#pragma unroll
                for (int k = 0; k < 3; ++k) x[k] = nxt[k];
            } else {
                const long long q = d.tile * 128 + row;
#pragma unroll
                for (int k = 0; k < 3; ++k) x[k] = q < n ? X[k * n + q] : 0.f;
            }
            // coordinates of this group's next tile, if the scheduler has published it
            {
                const long long s2 = sd + 2;
                const int sl2 = (int)(s2 % kND);
                if (mbar_test(&C.desc_full[sl2], (uint32_t)((s2 / kND) & 1))) {
                    const PipeDesc d2 = C.desc[sl2];
                    if (d2.item >= 0) {
                        const TcItem& I2 = C.item;
                        const float* X2 = xyz_ov ? xyz_ov : I2.xyz;
                        const long long q2 = d2.tile * 128 + row;
#pragma unroll
                        for (int k = 0; k < 3; ++k) nxt[k] = q2 < I2.n ? X2[k * I2.n + q2] : 0.f;
                        nxt_seq = s2;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&C.desc_empty[slot]);
            bool dead = false;
#pragma unroll 1
            for (int k = 0; k < 3 && !dead; ++k) {
                const float xt = fmaf(x[k], a.sc[k], a.of[k]);
                const int pe = a.pe[k];
                float Lm = 1.f, L = xt;
                // monic Legendre polynomials q_d = L_d / k_d (the leading coefficients k_d are
                // folded into the factor coefficients): q_d = x q_{d-1} - (d-1)^2 / ((2d-1)(2d-3))
                // q_{d-2}, two operations a degree, 32 degrees a half tile
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h * kPHalf >= pe) break;
                    const int ps = g * nps + pi;
                    if (!tc::mbar_wait(&C.p_empty[ps], pph ^ 1u, kWaitLimitE)) {
                        atomicOr(err, 2);
                        dead = true;
                        break;
                    }
                    unsigned char* Pb = pbuf + (size_t)ps * kPSlotBytes;
                    // degrees at or beyond pe are zeroed (their coefficient rows are zero, and
                    // far outside the box the recurrence could overflow); a half tile wholly
                    // below pe needs no mask
                    auto half = [&](auto masked) {
#pragma unroll
                        for (int c8 = 0; c8 < 4; ++c8) {
                            float v[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int dg = h * kPHalf + c8 * 8 + e;
                                float val;
                                if (dg == 0) {
                                    val = 1.f;
                                } else if (dg == 1) {
                                    val = xt;
                                } else {
                                    const float gd = float((dg - 1) * (dg - 1)) / float((2 * dg - 1) * (2 * dg - 3));
                                    const float Ln = fmaf(xt, L, -gd * Lm);
                                    Lm = L;
                                    L = Ln;
                                    val = Ln;
                                }
                                v[e] = (decltype(masked)::value && dg >= pe) ? 0.f : val;
                            }
                            const uint32_t off = tc::kmajor_offset(row, c8 * 16, kPHalf * 2);
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) split2_bf16(v[2 * e], v[2 * e + 1], hw[e], lw[e]);
                            *reinterpret_cast<uint4*>(Pb + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            *reinterpret_cast<uint4*>(Pb + 128 * kPHalf * 2 + off) =
                                make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    };
                    if ((h + 1) * kPHalf <= pe)
                        half(std::false_type{});
                    else
                        half(std::true_type{});
                    tc::fence_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&C.p_full[ps]);
                    if (++pi == nps) {
                        pi = 0;
                        pph ^= 1u;
                    }
                }
            }
            if (dead) break;
        }
    } else if (warp < 12) {
        // ------------------------------------------------------------ epilogue
        tc::setmaxnreg_inc<kRegsEpi>();
        const int ew = warp & 3, row = ew * 32 + lane;
        const uint32_t lanes = (uint32_t)(ew * 32) << 16;
        long long cm = 0, qc = 0;      // factor blocks and contraction chunks consumed
        bool dead = false;
        auto wait = [&](uint64_t* bar, uint32_t par, int code) {
            if (!dead && !tc::mbar_wait(bar, par, kWaitLimitE)) {
                atomicOr(err, code);
                dead = true;
            }
            tc::fence_after_sync();
            dead = __any_sync(0xffffffffu, dead);
        };
        for (long long sd = 0; !dead; ++sd) {
            const int slot = (int)(sd % kND);
            wait(&C.desc_full[slot], (uint32_t)((sd / kND) & 1), 4);
            if (dead) break;
            const PipeDesc d = C.desc[slot];
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&C.desc_empty[slot]);
            if (d.item < 0) break;
            const TcItem& I = C.item;
            const int r1 = I.a.r[0], r3 = I.a.r[2];
            const int nch = I.nchunks;
            float u2[RM], u3[RM];
#pragma unroll 1
            for (int k = 0; k < 3 && !dead; ++k, ++cm) {
                const int us = (int)(cm & 1);
                wait(&C.u_full[us], (uint32_t)((cm >> 1) & 1), 8);
                if (dead) break;
                // the three coefficient parts of the block (all loads in flight, one wait), added
                // low to high
                float uk[RM];
                const uint32_t ub = tmem + lanes + (uint32_t)(kUBase + us * kUCols);
#pragma unroll
                for (int c = 0; c < RM; c += 8) {
                    float th[8], tm[8], tl[8];
                    tc::tmem_ld8(ub + c, th);
                    tc::tmem_ld8(ub + 32 + c, tm);
                    tc::tmem_ld8(ub + 64 + c, tl);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const float2 t = __fadd2_rn(__fadd2_rn(make_float2(tl[e], tl[e + 1]), make_float2(tm[e], tm[e + 1])),
                                                    make_float2(th[e], th[e + 1]));
                        uk[c + e] = t.x;
                        uk[c + e + 1] = t.y;
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&C.u_empty[us]);
                if (k == 0) {
                    // w1 as the contraction's A operand (the previous tile's chunks are done)
                    wait(&C.w1_empty, (uint32_t)(sd & 1) ^ 1u, 16);
                    if (dead) break;
                    if (MODE == eTF32) {
#pragma unroll
                        for (int c16 = 0; c16 < KB / 16; ++c16) {
                            uint32_t v4[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int i = c16 * 4 + e;
                                v4[e] = tf32_dev(i < RM && i < r1 ? uk[i < RM ? i : 0] : 0.f);
                            }
                            *reinterpret_cast<uint4*>(w1buf + tc::kmajor_offset(row, c16 * 16, KB)) =
                                make_uint4(v4[0], v4[1], v4[2], v4[3]);
                        }
                    } else {
                        // BF16 words of the K-concatenated row [hi | lo | hi] (RM is even, so
                        // every word is one split pair): word w < RM/2 is hi pair w, then the lo
                        // pairs, then the hi pairs again, then zeros
                        static_assert(RM % 2 == 0, "rank bound is even");
                        uint32_t hw[RM / 2], lw[RM / 2];
#pragma unroll
                        for (int e = 0; e < RM / 2; ++e) {
                            const float a0 = 2 * e < r1 ? uk[2 * e] : 0.f, a1 = 2 * e + 1 < r1 ? uk[2 * e + 1] : 0.f;
                            split2_bf16(a0, a1, hw[e], lw[e]);
                        }
                        constexpr int H = RM / 2;
#pragma unroll
                        for (int c16 = 0; c16 < KB / 16; ++c16) {
                            uint32_t w4[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int w = c16 * 4 + e;
                                w4[e] = w < H ? hw[w < H ? w : 0]
                                        : (MODE == eBF16X3 && w < 2 * H) ? lw[w >= H && w < 2 * H ? w - H : 0]
                                        : (MODE == eBF16X3 && w < 3 * H) ? hw[w >= 2 * H && w < 3 * H ? w - 2 * H : 0]
                                                                         : 0u;
                            }
                            *reinterpret_cast<uint4*>(w1buf + tc::kmajor_offset(row, c16 * 16, KB)) =
                                make_uint4(w4[0], w4[1], w4[2], w4[3]);
                        }
                    }
                    tc::fence_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&C.w1_full);
                } else if (k == 1) {
#pragma unroll
                    for (int e = 0; e < RM; ++e) u2[e] = uk[e];
                } else {
#pragma unroll
                    for (int e = 0; e < RM; ++e) u3[e] = e < r3 ? uk[e] : 0.f;
                }
            }
            if (dead) break;
            // Khatri-Rao epilogue, chunk by chunk: per j-slice s_j = sum_k T_(j,k) w3_k in packed
            // pairs of k (two independent accumulators), then f += s_j w2_j
            float2 u3p[RM / 2];
#pragma unroll
            for (int e = 0; e < RM / 2; ++e) u3p[e] = make_float2(u3[2 * e], u3[2 * e + 1]);
            float f = 0.f;
#pragma unroll 1
            for (int ch = 0; ch < MAXCH; ++ch) {
                if (ch >= nch) break;
                const int cb = (int)(qc & 1);
                wait(&C.c_full[cb], (uint32_t)((qc >> 1) & 1), 32);
                if (dead) break;
                const uint32_t cbase = tmem + lanes + (uint32_t)(cb * kChunkCols);
                float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 16 * kEpiBatch) {
                    float v[kEpiBatch][16];
#pragma unroll
                    for (int b = 0; b < kEpiBatch; ++b)
                        if (c0 + 16 * b < NC) tc::tmem_ld16(cbase + c0 + 16 * b, v[b]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16 * kEpiBatch; e += 2) {
                        const int col = c0 + e;
                        if (col < NC) {
                            const int jl = col / R3P, k = col % R3P;
                            const float2 vv = make_float2(v[e / 16][e % 16], v[e / 16][e % 16 + 1]);
                            const float2 ww = u3p[k / 2 < RM / 2 ? k / 2 : 0];
                            if ((k & 2) == 0)
                                sa = __ffma2_rn(vv, ww, sa);
                            else
                                sb = __ffma2_rn(vv, ww, sb);
                            if (k == R3P - 2) {
                                const float2 s2 = __fadd2_rn(sa, sb);
                                if (jl < RM) f = fmaf(s2.x + s2.y, u2[jl < RM ? jl : 0], f);
                                sa = make_float2(0.f, 0.f);
                                sb = make_float2(0.f, 0.f);
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&C.c_empty[cb]);
                ++qc;
                // w2_{ch JC + jl} is u2[jl] in chunk ch (zero past the rank bound)
#pragma unroll
                for (int e = 0; e < RM; ++e) u2[e] = e + JC < RM ? u2[e + JC < RM ? e + JC : 0] : 0.f;
            }
            if (dead) break;
            const long long q = d.tile * 128 + row;
            if (q < I.n) (out_ov ? out_ov : I.out)[q] = f;
            __syncwarp();
            if (lane == 0) atomicAdd(&C.tiles_done, 1);
        }
    } else if ((warp == 12 || warp == 14) && lane == 0) {
        // ------------------------------------------------------------ MMA issuers
        // Two threads on different schedulers: warp 12 issues the factor MMAs of every tile in
        // order (modes 0, 1, 2), warp 14 the contraction chunks in order.  Each waits only on
        // the barriers of its own jobs (suspending, bounded waits), and the matrix descriptors
        // are formed once and advanced by adding offsets (the start address is their low field).
        const bool fac = warp == 12;
        const uint32_t core_u32 = tc::smem_u32(core), p_u32 = tc::smem_u32(pbuf), w1_u32 = tc::smem_u32(w1buf);
        constexpr uint32_t idesc_c = MODE == eTF32 ? tc::idesc_tf32(128, NCP) : tc::idesc_bf16(128, NCP);
        constexpr uint32_t idesc_f = tc::idesc_bf16(128, kUCols);
        long long cf = 0, qc = 0;      // factor blocks and chunks issued
        int pig[2] = {0, 0};           // next half-tile slot of each basis group and its use parity
        uint32_t pphg[2] = {0u, 0u};
        bool dead = false, issued = false;
        auto wait = [&](uint64_t* bar, uint32_t par, int code) -> bool {
            if (dead) return false;
            if (!tc::mbar_wait(bar, par, kWaitLimitE)) {
                atomicOr(err, code);
                dead = true;
                return false;
            }
            tc::fence_after_sync();
            return true;
        };
        const uint64_t pdesc0 = tc::make_desc(p_u32, 128, 512);            // half-tile slot 0, hi part
        const uint64_t adesc0 = tc::make_desc(w1_u32, 128, SBO_A);
        for (long long sd = 0; !dead; ++sd) {
            const int slot = (int)(sd % kND);
            if (!wait(&C.desc_full[slot], (uint32_t)((sd / kND) & 1), 512)) break;
            const int it = C.desc[slot].item;
            tc::mbar_arrive(&C.desc_empty[slot]);
            if (it < 0) break;
            const TcItem& I = C.item;
            if (fac) {
                const int g = (int)(sd & 1);
                const uint32_t kpb = (uint32_t)I.kpf * 2u;
                const uint64_t wdesc0 = tc::make_desc(core_u32 + (uint32_t)I.fac_off, 128, (kpb / 16u) * 128u);
#pragma unroll 1
                for (int k = 0; k < 3 && !dead; ++k) {
                    const int us = (int)(cf & 1);
                    if (!wait(&C.u_empty[us], (uint32_t)((cf >> 1) & 1) ^ 1u, 1024)) break;
                    const uint32_t dcol = tmem + (uint32_t)(kUBase + us * kUCols);
                    const uint64_t wk = wdesc0 + (((uint64_t)k * kUCols * kpb) >> 4);
                    const int nh = (I.a.pe[k] + kPHalf - 1) / kPHalf;
#pragma unroll 1
                    for (int hf = 0; hf < nh; ++hf) {
                        const int ps = g * nps + pig[g];
                        if (!wait(&C.p_full[ps], pphg[g], 2048)) break;
                        const uint64_t pa = pdesc0 + (((uint64_t)ps * kPSlotBytes) >> 4);
                        const uint64_t wb = wk + (uint64_t)(hf * 32);              // 512 bytes on
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                            for (int part = 0; part < 2; ++part)
                                tc::mma_bf16(dcol, pa + (uint64_t)(part * (128 * kPHalf * 2 / 16) + ks * 16),
                                             wb + (uint64_t)(ks * 16), idesc_f,
                                             (hf > 0 || ks > 0 || part > 0) ? 1u : 0u);
                        tc::mma_commit(&C.p_empty[ps]);
                        issued = true;
                        if (++pig[g] == nps) {
                            pig[g] = 0;
                            pphg[g] ^= 1u;
                        }
                    }
                    if (dead) break;
                    tc::mma_commit(&C.u_full[us]);
                    ++cf;
                }
            } else {
                if (!wait(&C.w1_full, (uint32_t)(sd & 1), 4096)) break;
#pragma unroll 1
                for (int ch = 0; ch < I.nchunks; ++ch) {
                    const int cb = (int)(qc & 1);
                    if (!wait(&C.c_empty[cb], (uint32_t)((qc >> 1) & 1) ^ 1u, 8192)) break;
                    const uint64_t bd0 = tc::make_desc(core_u32 + (uint32_t)ch * (uint32_t)(NCP * KB), 128, SBO_A);
                    const uint32_t dcol = tmem + (uint32_t)(cb * kChunkCols);
#pragma unroll
                    for (int ks = 0; ks < KB / 32; ++ks) {
                        if (MODE == eTF32)
                            tc::mma_tf32(dcol, adesc0 + (uint64_t)(ks * 16), bd0 + (uint64_t)(ks * 16), idesc_c, ks > 0);
                        else
                            tc::mma_bf16(dcol, adesc0 + (uint64_t)(ks * 16), bd0 + (uint64_t)(ks * 16), idesc_c, ks > 0);
                    }
                    tc::mma_commit(&C.c_full[cb]);
                    issued = true;
                    ++qc;
                }
                if (dead) break;
                tc::mma_commit(&C.w1_empty);     // the tile's A operand is read
            }
        }
        if (issued) {
            // every MMA of this thread completes before tensor memory is released
            tc::mma_commit(&C.drain[fac ? 0 : 1]);
            if (!tc::mbar_wait(&C.drain[fac ? 0 : 1], 0u, kWaitLimitE)) atomicOr(err, 16);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 12) tc::tmem_dealloc(tmem, 512);
}

struct EvalErr {
    std::mutex mu;
    DevBuf flag;
};
EvalErr g_eval_err[64];

struct HostItem {
    fst_model* m;
    const float* xyz;
    long long n;
    float* out;
};


// One size class of a batch: instances sharing the (rank, r3) padding, one launch.
struct Bucket {
    int mode = 0, r3p = 8, rm = 8;
    bool tc3 = false;            // factor step on the tensor cores (eval_pipe_kernel)
    int kpf_max = 32;
    int nps = 1;                 // Legendre half-tile slots per basis group (pipelined variant)
    std::vector<TcItem> items;
    std::vector<TcUnit> units;
    std::vector<int> cta_start;
    int core_max = 0, kb_max = 32, grid = 1;
    size_t smem = 0;
    size_t items_off = 0, units_off = 0, cta_off = 0, ctr_off = 0, bytes = 0;   // device image layout
};

fst_status build_buckets(const std::vector<HostItem>& hitems, int mode, std::vector<Bucket>& out) {
    out.clear();
    const int PARTS = mode == eBF16X3 ? 2 : 1;
    const int sms = sm_count();
    std::vector<std::vector<size_t>> members;
    std::vector<std::array<int, 3>> keys;
    for (size_t i = 0; i < hitems.size(); ++i) {
        const fst_model* m = hitems[i].m;
        const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
        const int r3p = std::min(bucket8(m->r[2]), rm);
        const std::array<int, 3> key{rm, r3p, use_tc3(m, mode, r3p) ? 1 : 0};
        size_t b = 0;
        while (b < keys.size() && keys[b] != key) ++b;
        if (b == keys.size()) {
            keys.push_back(key);
            members.emplace_back();
        }
        members[b].push_back(i);
    }
    for (size_t b = 0; b < keys.size(); ++b) {
        Bucket B;
        B.mode = mode;
        B.rm = keys[b][0];
        B.r3p = keys[b][1];
        B.tc3 = keys[b][2] != 0;
        std::vector<double> tile_cost;
        int tab_max = 0;
        for (size_t idx : members[b]) {
            fst_model* m = hitems[idx].m;
            TcItem it;
            {
                // one model's lock at a time (never two held together): the image slots and
                // tc_core are shared with single-instance evaluations on other threads
                std::lock_guard<std::recursive_mutex> lk(m->mu);
                FST_TRY(prepare_core_image(m, mode, B.r3p));
                it.core_img = static_cast<const unsigned char*>(m->tc_core);   // this kind's image
            }
            const CoreImage ci = core_image_shape(m, mode, B.r3p, B.tc3);
            it.a = make_args<float>(m);
            bind(it.a, m);
            it.img_bytes = (int)ci.bytes;
            it.nchunks = ci.nchunks;
            it.kp = ci.kp;
            it.tab_bytes = (int)((2 * (size_t)it.a.pm + (size_t)(it.a.pe[0] + it.a.pe[1] + it.a.pe[2]) * B.rm) * 4 +
                                 3 * it.a.pm);
            it.fac_off = (int)ci.fac_off;
            it.kpf = ci.kpf;
            it.xyz = hitems[idx].xyz;
            it.out = hitems[idx].out;
            it.n = hitems[idx].n;
            B.core_max = std::max(B.core_max, (int)((ci.bytes + 1023) & ~(size_t)1023));
            B.kb_max = std::max(B.kb_max, ci.kb);
            B.kpf_max = std::max(B.kpf_max, ci.kpf);
            tab_max = std::max(tab_max, it.tab_bytes);
            // per-tile cost: factor values (CUDA cores, or Legendre tiles + factor MMAs) +
            // contraction and epilogue per chunk
            const double fac = B.tc3 ? 1.0 + 3.0 * ci.kpf / 32.0
                                     : 1.0 + (double)B.rm * (it.a.pe[0] + it.a.pe[1] + it.a.pe[2]) / 64.0;
            tile_cost.push_back(fac + (double)ci.nchunks * ci.ncp * (PARTS == 2 ? 1.5 : 1.0) / 64.0);
            B.items.push_back(it);
        }
        if (B.tc3) B.nps = tc3_nps(B.core_max, B.kb_max);
        B.smem = B.tc3 ? tc3_smem(B.core_max, B.kb_max, B.nps)
                       : 1024 + kBarBytes + B.core_max + (size_t)kGroups * PARTS * 128 * B.kb_max + tab_max + 16;
        if (B.smem > 227 * 1024) {
            set_error("model too large for the tensor-core evaluator (%zu bytes of shared memory)", B.smem);
            return FST_EUNSUPPORTED;
        }
        long long total_tiles = 0;
        double total_cost = 0;
        for (size_t i = 0; i < B.items.size(); ++i) {
            const long long nt = (B.items[i].n + 127) / 128;
            total_tiles += nt;
            total_cost += nt * tile_cost[i];
        }
        if (total_tiles == 0) continue;
        // units of ~1/4 of a CTA's share (taken dynamically by the factor-step kernel, cut
        // into static per-CTA ranges by cost for the other); at least one tile per worker group
        long long run = (total_tiles + 4LL * sms - 1) / (4LL * sms);
        if (run < 3) run = 3;
        std::vector<double> unit_cost;
        for (size_t i = 0; i < B.items.size(); ++i) {
            const long long nt = (B.items[i].n + 127) / 128;
            for (long long t0 = 0; t0 < nt; t0 += run) {
                TcUnit u;
                u.item = (int)i;
                u.pad = 0;
                u.tile0 = t0;
                u.ntiles = std::min(run, nt - t0);
                B.units.push_back(u);
                unit_cost.push_back(u.ntiles * tile_cost[i]);
            }
        }
        B.grid = (int)std::min<long long>(sms, (long long)B.units.size());
        B.cta_start.assign(B.grid + 1, (int)B.units.size());
        B.cta_start[0] = 0;
        double acc = 0;
        int c = 1;
        for (size_t u = 0; u < B.units.size() && c < B.grid; ++u) {
            acc += unit_cost[u];
            while (c < B.grid && acc >= total_cost * c / B.grid) B.cta_start[c++] = (int)u + 1;
        }
        for (; c < B.grid; ++c) B.cta_start[c] = (int)B.units.size();
        B.items_off = 0;
        B.units_off = (B.items.size() * sizeof(TcItem) + 15) & ~(size_t)15;
        B.cta_off = (B.units_off + B.units.size() * sizeof(TcUnit) + 15) & ~(size_t)15;
        B.ctr_off = (B.cta_off + B.cta_start.size() * sizeof(int) + 15) & ~(size_t)15;   // unit counter
        B.bytes = B.ctr_off + 16;
        out.push_back(std::move(B));
    }
    return FST_OK;
}

void bucket_image(const Bucket& B, std::vector<unsigned char>& img) {
    img.assign(B.bytes, 0);
    memcpy(img.data() + B.items_off, B.items.data(), B.items.size() * sizeof(TcItem));
    memcpy(img.data() + B.units_off, B.units.data(), B.units.size() * sizeof(TcUnit));
    memcpy(img.data() + B.cta_off, B.cta_start.data(), B.cta_start.size() * sizeof(int));
}

struct Overrides {
    const float* xyz = nullptr;
    float* out = nullptr;
};

template <int MODE, int R3P, int RM>
fst_status launch_bucket_t(const Bucket& B, const unsigned char* dimg, int* err, cudaStream_t s, Overrides ov) {
    auto kern = eval_tc_kernel<MODE, R3P, RM>;
    FST_TRY(allow_smem(kern, B.smem));
    kern<<<B.grid, kThreadsE, B.smem, s>>>(reinterpret_cast<const TcItem*>(dimg + B.items_off),
                                           reinterpret_cast<const TcUnit*>(dimg + B.units_off),
                                           reinterpret_cast<const int*>(dimg + B.cta_off), B.core_max, B.kb_max,
                                           ov.xyz, ov.out, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <int MODE>
fst_status launch_bucket_m(const Bucket& B, const unsigned char* dimg, int* err, cudaStream_t s, Overrides ov) {
#define FST_EB(R3, RMV) \
    if (B.r3p == R3 && B.rm == RMV) return launch_bucket_t<MODE, R3, RMV>(B, dimg, err, s, ov);
    FST_EB(8, 8) FST_EB(8, 16) FST_EB(16, 16) FST_EB(8, 24) FST_EB(16, 24) FST_EB(24, 24)
    FST_EB(8, 32) FST_EB(16, 32) FST_EB(24, 32) FST_EB(32, 32)
#undef FST_EB
    set_error("no evaluator instance for r3 padding %d, rank bound %d", B.r3p, B.rm);
    return FST_EUNSUPPORTED;
}

template <int MODE, int R3P, int RM>
fst_status launch_bucket_tc3_t(const Bucket& B, const unsigned char* dimg, int* err, cudaStream_t s, Overrides ov) {
    auto kern = eval_pipe_kernel<MODE, R3P, RM>;
    FST_TRY(allow_smem(kern, B.smem));
    // several instances: units from a counter; one: the static per-CTA ranges
    int* ctr = nullptr;
    if (B.items.size() > 1) {
        ctr = reinterpret_cast<int*>(const_cast<unsigned char*>(dimg) + B.ctr_off);
        FST_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int), s));
    }
    kern<<<B.grid, kThreadsP, B.smem, s>>>(reinterpret_cast<const TcItem*>(dimg + B.items_off),
                                           reinterpret_cast<const TcUnit*>(dimg + B.units_off),
                                           reinterpret_cast<const int*>(dimg + B.cta_off), (int)B.units.size(), ctr,
                                           B.core_max, B.nps, ov.xyz, ov.out, err);
    FST_CHECK_LAUNCH();
    return FST_OK;
}

template <int MODE>
fst_status launch_bucket_tc3_m(const Bucket& B, const unsigned char* dimg, int* err, cudaStream_t s, Overrides ov) {
#define FST_EB(R3, RMV) \
    if (B.r3p == R3 && B.rm == RMV) return launch_bucket_tc3_t<MODE, R3, RMV>(B, dimg, err, s, ov);
    FST_EB(8, 8) FST_EB(8, 16) FST_EB(16, 16) FST_EB(8, 24) FST_EB(16, 24) FST_EB(24, 24)
    FST_EB(8, 32) FST_EB(16, 32) FST_EB(24, 32) FST_EB(32, 32)
#undef FST_EB
    set_error("no evaluator instance for r3 padding %d, rank bound %d", B.r3p, B.rm);
    return FST_EUNSUPPORTED;
}

fst_status launch_bucket(const Bucket& B, const unsigned char* dimg, int* err, cudaStream_t s, Overrides ov) {
    if (B.tc3) {
        if (B.mode == eTF32) return launch_bucket_tc3_m<eTF32>(B, dimg, err, s, ov);
        if (B.mode == eBF16) return launch_bucket_tc3_m<eBF16>(B, dimg, err, s, ov);
        return launch_bucket_tc3_m<eBF16X3>(B, dimg, err, s, ov);
    }
    switch (B.mode) {
        case eTF32: return launch_bucket_m<eTF32>(B, dimg, err, s, ov);
        case eBF16: return launch_bucket_m<eBF16>(B, dimg, err, s, ov);
        default: return launch_bucket_m<eBF16X3>(B, dimg, err, s, ov);
    }
}

int mode_of(fst_prec p) { return p == FST_TF32 ? eTF32 : p == FST_BF16 ? eBF16 : eBF16X3; }

fst_status error_word(int** out) {
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    EvalErr& ee = g_eval_err[dev & 63];
    std::lock_guard<std::mutex> lk(ee.mu);
    if (!ee.flag.ptr) {
        FST_TRY(ee.flag.ensure(sizeof(int)));
        FST_CUDA(cudaMemset(ee.flag.ptr, 0, sizeof(int)));
    }
    *out = ee.flag.as<int>();
    return FST_OK;
}

}  // namespace

// Tensor-core operand image of the core for (mode, r3 padding), cached in the model.
fst_status prepare_core_image(fst_model* m, int mode, int r3p) {
    const bool tc3 = use_tc3(m, mode, r3p);
    const CoreImage ci = core_image_shape(m, mode, r3p, tc3);
    const int kind = (tc3 ? 512 : 0) + mode * 64 + r3p;
    // the slot of this kind, else a stale or unused one, else the least recently built
    fst_model::TcImage* slot = nullptr;
    for (auto& t : m->tc_img)
        if (t.kind == kind && t.ptr) {
            m->tc_core = t.ptr;
            return FST_OK;
        }
    for (auto& t : m->tc_img)
        if (t.kind < 0) {
            slot = &t;
            break;
        }
    if (!slot) slot = &m->tc_img[0];   // every slot holds a live kind (8 kinds): replace the first
    std::vector<unsigned char> img = build_core_image(m, ci);
    // a stale slot's buffer may still be read by evaluations queued on other (non-blocking)
    // streams before the core changed: the synchronous copy below does not wait for them
    if (slot->ptr) FST_CUDA(cudaDeviceSynchronize());
    if (slot->bytes < img.size()) {
        if (slot->ptr) cudaFree(slot->ptr);
        slot->ptr = nullptr;
        slot->bytes = 0;
        FST_CUDA(cudaMalloc(&slot->ptr, img.size()));
        slot->bytes = img.size();
    }
    FST_CUDA(cudaMemcpy(slot->ptr, img.data(), img.size(), cudaMemcpyHostToDevice));
    slot->kind = kind;
    m->tc_core = slot->ptr;
    ++m->tc_core_kind_version;
    return FST_OK;
}

}  // namespace fst

// A prepared batch: work lists of every size class uploaded once.
struct fst_eval_plan {
    int device = 0;
    std::vector<fst::Bucket> buckets;
    unsigned char* dimg = nullptr;      // work lists and unit counters
    std::vector<size_t> offs;
    // runs of one plan on different streams are ordered on the device (they share the unit
    // counters): each waits for the event of the previous run
    mutable std::mutex mu;
    mutable cudaEvent_t done = nullptr;
    mutable bool used = false;
};

namespace fst {

fst_status plan_build(const std::vector<HostItem>& items, fst_prec prec, fst_eval_plan** out) {
    std::unique_ptr<fst_eval_plan> P(new fst_eval_plan());
    FST_CUDA(cudaGetDevice(&P->device));
    FST_TRY(build_buckets(items, mode_of(prec), P->buckets));
    size_t total = 0;
    for (const Bucket& B : P->buckets) {
        P->offs.push_back(total);
        total += (B.bytes + 255) & ~(size_t)255;
    }
    if (total) {
        FST_CUDA(cudaMalloc(&P->dimg, total));
        std::vector<unsigned char> img;
        for (size_t b = 0; b < P->buckets.size(); ++b) {
            bucket_image(P->buckets[b], img);
            FST_CUDA(cudaMemcpy(P->dimg + P->offs[b], img.data(), img.size(), cudaMemcpyHostToDevice));
        }
    }
    *out = P.release();
    return FST_OK;
}

fst_status plan_run(const fst_eval_plan* P, cudaStream_t s, Overrides ov = Overrides()) {
    int* err = nullptr;
    FST_TRY(error_word(&err));
    std::lock_guard<std::mutex> lk(P->mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FST_CUDA(cudaStreamIsCapturing(s, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;   // a captured run is ordered by its graph
    if (!capturing) {
        if (!P->done) FST_CUDA(cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming));
        if (P->used) FST_CUDA(cudaStreamWaitEvent(s, P->done, 0));
    }
    for (size_t b = 0; b < P->buckets.size(); ++b)
        FST_TRY(launch_bucket(P->buckets[b], P->dimg + P->offs[b], err, s, ov));
    if (!capturing) {
        FST_CUDA(cudaEventRecord(P->done, s));
        P->used = true;
    }
    return FST_OK;
}

void plan_free(fst_eval_plan* P) {
    if (!P) return;
    if (P->dimg) cudaFree(P->dimg);   // cudaFree waits for work in flight on the device
    if (P->done) cudaEventDestroy(P->done);
    delete P;
}

// Asynchronous batch: the size classes are built on the host, their work lists staged in a
// pinned buffer and copied to a device slot of a per-device ring; a slot is reused only
// after the launches that read it have finished (its event).  Buffers only grow, so a
// steady stream of batches allocates nothing.
struct BatchRing {
    std::mutex mu;
    DevBuf dev[8];
    unsigned char* host[8] = {};
    size_t host_bytes[8] = {};
    cudaEvent_t done[8] = {};
    int next = 0;
};
BatchRing g_batch_ring[64];

fst_status eval_tc_batch(const std::vector<HostItem>& items, fst_prec prec, cudaStream_t s) {
    std::vector<Bucket> buckets;
    FST_TRY(build_buckets(items, mode_of(prec), buckets));
    if (buckets.empty()) return FST_OK;
    std::vector<size_t> offs;
    size_t total = 0;
    for (const Bucket& B : buckets) {
        offs.push_back(total);
        total += (B.bytes + 255) & ~(size_t)255;
    }
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    BatchRing& ring = g_batch_ring[dev & 63];
    std::lock_guard<std::mutex> lk(ring.mu);
    const int slot = ring.next;
    ring.next = (ring.next + 1) % 8;
    if (ring.done[slot]) FST_CUDA(cudaEventSynchronize(ring.done[slot]));
    else FST_CUDA(cudaEventCreateWithFlags(&ring.done[slot], cudaEventDisableTiming));
    FST_TRY(ring.dev[slot].ensure(total));
    if (ring.host_bytes[slot] < total) {
        if (ring.host[slot]) cudaFreeHost(ring.host[slot]);
        ring.host[slot] = nullptr;
        ring.host_bytes[slot] = 0;
        FST_CUDA(cudaMallocHost(&ring.host[slot], total));
        ring.host_bytes[slot] = total;
    }
    std::vector<unsigned char> img;
    for (size_t b = 0; b < buckets.size(); ++b) {
        bucket_image(buckets[b], img);
        memcpy(ring.host[slot] + offs[b], img.data(), img.size());
    }
    unsigned char* d = ring.dev[slot].as<unsigned char>();
    FST_CUDA(cudaMemcpyAsync(d, ring.host[slot], total, cudaMemcpyHostToDevice, s));
    int* err = nullptr;
    FST_TRY(error_word(&err));
    for (size_t b = 0; b < buckets.size(); ++b) FST_TRY(launch_bucket(buckets[b], d + offs[b], err, s, Overrides()));
    FST_CUDA(cudaEventRecord(ring.done[slot], s));
    return FST_OK;
}

fst_status eval_tc_launch(fst_model* m, const float* xyz, int64_t n, float* out, fst_prec prec, cudaStream_t s) {
    if (n == 0) return FST_OK;
    std::lock_guard<std::recursive_mutex> lk(m->mu);
    // single instance: the work list depends on n, the precision and the core image only; it
    // is kept in the model, and the point and output buffers are passed at launch
    const int mode = mode_of(prec);
    const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    FST_TRY(prepare_core_image(m, mode, std::min(bucket8(m->r[2]), rm)));
    fst_eval_plan*& P = m->eval_plan;
    if (!P || m->eval_plan_n != (long long)n || m->eval_plan_prec != (int)prec ||
        m->eval_plan_core != m->tc_core_kind_version) {
        if (P) {
            FST_CUDA(cudaStreamSynchronize(s));
            plan_free(P);
            P = nullptr;
        }
        std::vector<HostItem> one{HostItem{m, xyz, (long long)n, out}};
        FST_TRY(plan_build(one, prec, &P));
        m->eval_plan_n = (long long)n;
        m->eval_plan_prec = (int)prec;
        m->eval_plan_core = m->tc_core_kind_version;
    }
    Overrides ov;
    ov.xyz = xyz;
    ov.out = out;
    return plan_run(P, s, ov);
}

// ---------------------------------------------------------------- autotuner
// Probe points: n points spread over the model's box by a counter hash (splitmix64 finaliser
// of the index), reproducible.
__global__ void probe_points_kernel(float* xyz, int64_t n, float lo0, float lo1, float lo2, float hi0, float hi1,
                                    float hi2) {
    const float lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            uint64_t z = (uint64_t)(3 * i + k + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const float u01 = (float)(z >> 40) * (1.0f / 16777216.0f);
            xyz[k * n + i] = lo[k] + (hi[k] - lo[k]) * u01;
        }
}

struct ProbeBufs {
    std::mutex mu;
    DevBuf xyz, out;
};
ProbeBufs g_probe[64];

// Times both evaluator variants of the model's size class on n probe points (one warm-up and
// three timed runs each, CUDA events) and records the faster in the table.  Synchronous.
fst_status eval_autotune(fst_model* m, fst_prec prec, int64_t n, cudaStream_t s, float ms[2], int* choice) {
    ms[0] = ms[1] = -1.f;
    const int mode = mode_of(prec);
    const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    const int r3p = std::min(bucket8(m->r[2]), rm);
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    const TuneKey key = tune_key(m, mode, r3p);
    if (!tc3_feasible(m, mode, r3p)) {
        *choice = 0;
    } else {
        ProbeBufs& pb = g_probe[dev & 63];
        std::lock_guard<std::mutex> lk(pb.mu);
        FST_TRY(pb.xyz.ensure(sizeof(float) * 3 * (size_t)n));
        FST_TRY(pb.out.ensure(sizeof(float) * (size_t)n));
        float* xyz = pb.xyz.as<float>();
        float* out = pb.out.as<float>();
        probe_points_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8LL * sm_count()), 256, 0, s>>>(
            xyz, n, (float)m->lo[0], (float)m->lo[1], (float)m->lo[2], (float)m->hi[0], (float)m->hi[1],
            (float)m->hi[2]);
        FST_CHECK_LAUNCH();
        cudaEvent_t e0, e1;
        FST_CUDA(cudaEventCreate(&e0));
        FST_CUDA(cudaEventCreate(&e1));
        fst_status st = FST_OK;
        for (int v = 0; v < 2 && st == FST_OK; ++v) {
            t_force_variant = v;
            fst_eval_plan* P = nullptr;
            st = prepare_core_image(m, mode, r3p);
            std::vector<HostItem> one{HostItem{m, xyz, (long long)n, out}};
            if (st == FST_OK) st = plan_build(one, prec, &P);
            if (st == FST_OK) st = plan_run(P, s);
            if (st == FST_OK && cudaEventRecord(e0, s) != cudaSuccess) st = FST_ECUDA;
            for (int r = 0; r < 3 && st == FST_OK; ++r) st = plan_run(P, s);
            if (st == FST_OK && cudaEventRecord(e1, s) != cudaSuccess) st = FST_ECUDA;
            if (st == FST_OK && cudaEventSynchronize(e1) != cudaSuccess) st = FST_ECUDA;
            if (st == FST_OK) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                ms[v] = t / 3.f;
            }
            if (P) plan_free(P);
        }
        t_force_variant = -1;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st == FST_ECUDA) set_error("autotune: CUDA event failure");
        FST_TRY(st);
        *choice = ms[1] < ms[0] ? 1 : 0;
    }
    {
        TuneTable& T = g_tune[dev & 63];
        std::lock_guard<std::mutex> lk(T.mu);
        T.choice[key] = *choice;
    }
    return prepare_core_image(m, mode, r3p);   // the image of the chosen variant
}

bool tune_known(const fst_model* m, fst_prec prec) {
    const int mode = mode_of(prec);
    const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    const int r3p = std::min(bucket8(m->r[2]), rm);
    int dev = 0;
    cudaGetDevice(&dev);
    TuneTable& T = g_tune[dev & 63];
    std::lock_guard<std::mutex> lk(T.mu);
    return T.choice.count(tune_key(m, mode, r3p)) != 0;
}

fst_status tune_set(const fst_model* m, fst_prec prec, int choice) {
    const int mode = mode_of(prec);
    const int rm = bucket8(std::max(m->r[0], std::max(m->r[1], m->r[2])));
    const int r3p = std::min(bucket8(m->r[2]), rm);
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    TuneTable& T = g_tune[dev & 63];
    std::lock_guard<std::mutex> lk(T.mu);
    if (choice < 0) T.choice.erase(tune_key(m, mode, r3p));
    else T.choice[tune_key(m, mode, r3p)] = choice;
    return FST_OK;
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
    std::lock_guard<std::recursive_mutex> lk(m->mu);
    const int mode = prec == FST_TF32 ? 0 : prec == FST_BF16 ? 1 : 2;
    int rmax = m->r[0] > m->r[1] ? m->r[0] : m->r[1];
    rmax = m->r[2] > rmax ? m->r[2] : rmax;
    const int r3 = m->r[2];
    const int r3p = std::min(r3 <= 8 ? 8 : r3 <= 16 ? 16 : r3 <= 24 ? 24 : 32, fst::bucket8(rmax));
    if (!fst::tune_known(m, prec)) {
        // first model of this size class on this device: measure the evaluator variants
        float ms[2];
        int choice = 0;
        return fst::eval_autotune(m, prec, 1 << 18, s, ms, &choice);
    }
    return fst::prepare_core_image(m, mode, r3p);
}

extern "C" fst_status fst_eval_autotune(fst_model* m, fst_prec prec, int64_t n_probe, fst_stream stream,
                                        float* ms_cuda_core_factors, float* ms_tensor_core_factors,
                                        int32_t* choice) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "autotuning covers the tensor-core precisions TF32, BF16, BF16X3");
    FST_REQUIRE(n_probe > 0, "n_probe must be positive");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == m->device, "model lives on device %d, current device is %d", m->device, dev);
    std::lock_guard<std::recursive_mutex> lk(m->mu);
    float ms[2];
    int c = 0;
    FST_TRY(fst::eval_autotune(m, prec, n_probe, (cudaStream_t)stream, ms, &c));
    if (ms_cuda_core_factors) *ms_cuda_core_factors = ms[0];
    if (ms_tensor_core_factors) *ms_tensor_core_factors = ms[1];
    if (choice) *choice = c;
    return FST_OK;
}

extern "C" fst_status fst_eval_autotune_set(const fst_model* m, fst_prec prec, int32_t choice) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3, "tensor-core precision expected");
    FST_REQUIRE(choice >= -1 && choice <= 1, "choice must be -1 (forget), 0 or 1");
    return fst::tune_set(m, prec, choice);
}

extern "C" fst_status fst_eval_batched(const fst_eval_item* items, int32_t count, fst_prec prec,
                                       fst_stream stream) {
    using namespace fst;
    FST_REQUIRE(count >= 0 && (count == 0 || items != nullptr), "items is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<HostItem> work;
    for (int i = 0; i < count; ++i) {
        const fst_eval_item& it = items[i];
        FST_REQUIRE(it.model != nullptr && it.n >= 0, "item %d: model NULL or n < 0", i);
        if (it.n == 0) continue;
        FST_REQUIRE(it.xyz && it.out, "item %d: xyz or out is NULL", i);
        FST_REQUIRE(it.model->device == dev, "item %d: model lives on another device", i);
        FST_REQUIRE(pointer_device(it.xyz) == dev && pointer_device(it.out) == dev,
                    "item %d: xyz and out must be device memory of device %d", i, dev);
        work.push_back(HostItem{const_cast<fst_model*>(it.model), it.xyz, (long long)it.n, it.out});
    }
    if (work.empty()) return FST_OK;
    if (prec == FST_FP32) {
        for (const HostItem& h : work) FST_TRY(eval_simt_launch<float>(h.m, h.xyz, h.n, h.out, s));
        return FST_OK;
    }
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "fst_eval_batched takes FP32, TF32, BF16 or BF16X3");
    return eval_tc_batch(work, prec, s);
}

extern "C" fst_status fst_eval_plan_create(const fst_eval_item* items, int32_t count, fst_prec prec,
                                           fst_eval_plan** out) {
    using namespace fst;
    FST_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    FST_REQUIRE(count >= 0 && (count == 0 || items != nullptr), "items is NULL");
    FST_REQUIRE(prec == FST_TF32 || prec == FST_BF16 || prec == FST_BF16X3,
                "evaluation plans take TF32, BF16 or BF16X3");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    std::vector<HostItem> work;
    for (int i = 0; i < count; ++i) {
        const fst_eval_item& it = items[i];
        FST_REQUIRE(it.model != nullptr && it.n >= 0, "item %d: model NULL or n < 0", i);
        if (it.n == 0) continue;
        FST_REQUIRE(it.xyz && it.out, "item %d: xyz or out is NULL", i);
        FST_REQUIRE(it.model->device == dev, "item %d: model lives on another device", i);
        FST_REQUIRE(pointer_device(it.xyz) == dev && pointer_device(it.out) == dev,
                    "item %d: xyz and out must be device memory of device %d", i, dev);
        work.push_back(HostItem{const_cast<fst_model*>(it.model), it.xyz, (long long)it.n, it.out});
    }
    return plan_build(work, prec, out);
}

extern "C" fst_status fst_eval_plan_run(const fst_eval_plan* plan, fst_stream stream) {
    using namespace fst;
    FST_REQUIRE(plan != nullptr, "plan is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev == plan->device, "plan was made on device %d, current device is %d", plan->device, dev);
    return plan_run(plan, (cudaStream_t)stream);
}

extern "C" void fst_eval_plan_free(fst_eval_plan* plan) { fst::plan_free(plan); }
