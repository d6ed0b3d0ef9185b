// sample.cu -- uniform row sampling without replacement (Algorithm 2, sampling step).
//
// Row q carries the key splitmix64(seed, q): the (q+1)-th output of a splitmix64
// stream (Steele, Lea, Flood 2014) seeded with `seed`.  The sample is the set of m
// rows with the smallest keys.  Distinct rows have distinct keys (the splitmix64
// finaliser is a bijection of 64-bit words and the states seed + (q+1)*gamma are
// distinct), so the set is well defined.
//
// GPU algorithm: keys are never stored.  A 6-pass radix select (11-bit digits,
// most significant first) finds the m-th smallest key T by histogramming the keys
// that share the prefix fixed so far; a final two-pass stream compaction writes
// the rows with key <= T in ascending row order.  Every pass recomputes the keys
// from the counter, so the only memory traffic is the output.
#include "fst_internal.cuh"

namespace fst {

struct SelectState {
    unsigned long long prefix;  // fixed high bits of the m-th smallest key
    unsigned long long mask;    // which bits of prefix are fixed
    unsigned long long rank;    // 1-based rank of the wanted key among keys matching prefix
};

constexpr int kDigitBits = 11;
constexpr int kBins = 1 << kDigitBits;
constexpr int kPasses = 6;   // shifts 53, 42, 31, 20, 9, 0 (the last digit has 9 bits)
constexpr int kCompactBlock = 256;

__device__ __forceinline__ int pass_shift(int pass) { return pass < 5 ? 53 - kDigitBits * pass : 0; }

__global__ void select_hist_kernel(uint64_t seed, int64_t Q, int pass, const SelectState* st,
                                   unsigned int* hist) {
    __shared__ unsigned int h[kBins];
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    const int shift = pass_shift(pass);
    const unsigned dmask = pass < 5 ? (kBins - 1) : 511;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = splitmix_key(seed, (uint64_t)q);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One block: find the digit holding the rank-th key, fix it, clear the histogram.
__global__ void select_pick_kernel(int pass, SelectState* st, unsigned int* hist) {
    __shared__ unsigned long long part[32];
    const int t = threadIdx.x;   // launched with 32 threads
    // each thread owns kBins / 32 consecutive bins
    unsigned long long sum = 0;
    for (int i = 0; i < kBins / 32; ++i) sum += hist[t * (kBins / 32) + i];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        unsigned long long rank = st->rank, before = 0;
        int owner = -1;
        for (int w = 0; w < 32; ++w) {
            if (before + part[w] >= rank) { owner = w; break; }
            before += part[w];
        }
        if (owner >= 0) {
            int digit = -1;
            for (int i = 0; i < kBins / 32; ++i) {
                const int b = owner * (kBins / 32) + i;
                if (before + hist[b] >= rank) { digit = b; break; }
                before += hist[b];
            }
            const int shift = pass < 5 ? 53 - kDigitBits * pass : 0;
            const unsigned long long dmask = pass < 5 ? (kBins - 1) : 511;
            st->prefix |= ((unsigned long long)digit) << shift;
            st->mask |= dmask << shift;
            st->rank = rank - before;
        }
    }
    __syncthreads();
    for (int i = 0; i < kBins / 32; ++i) hist[t * (kBins / 32) + i] = 0;
}

__global__ void init_state_kernel(SelectState* st, unsigned long long m, unsigned int* hist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->prefix = 0;
        st->mask = 0;
        st->rank = m;
    }
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
}

// Compaction pass 1: rows with key <= T per block (each block owns a contiguous row range).
__global__ void compact_count_kernel(uint64_t seed, int64_t Q, int64_t rows_per_block,
                                     const SelectState* st, unsigned long long* counts) {
    const uint64_t T = st->prefix;
    const int64_t lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t hi = lo + rows_per_block < Q ? lo + rows_per_block : Q;
    unsigned int c = 0;
    for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x)
        c += splitmix_key(seed, (uint64_t)q) <= T;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned int wsum[kCompactBlock / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
        counts[blockIdx.x] = tot;
    }
}

// Exclusive scan of the per-block counts (one block, sequential chunks).
__global__ void scan_counts_kernel(unsigned long long* counts, int nblocks) {
    __shared__ unsigned long long carry;
    __shared__ unsigned long long buf[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        buf[threadIdx.x] = i < nblocks ? counts[i] : 0;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            unsigned long long v = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += v;
            __syncthreads();
        }
        const unsigned long long incl = buf[threadIdx.x];
        const unsigned long long mine = i < nblocks ? counts[i] : 0;
        __syncthreads();
        if (i < nblocks) counts[i] = carry + incl - mine;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// Compaction pass 2: write selected rows in ascending order.
__global__ void compact_write_kernel(uint64_t seed, int64_t Q, int64_t rows_per_block,
                                     const SelectState* st, const unsigned long long* offsets,
                                     int64_t* idx, int64_t m) {
    const uint64_t T = st->prefix;
    const int64_t lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t hi = lo + rows_per_block < Q ? lo + rows_per_block : Q;
    __shared__ unsigned int wcount[kCompactBlock / 32];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = offsets[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r0 = lo; r0 < hi; r0 += blockDim.x) {
        const int64_t q = r0 + threadIdx.x;
        const bool sel = q < hi && splitmix_key(seed, (uint64_t)q) <= T;
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        __syncthreads();
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        unsigned long long off = base;
        for (int w = 0; w < warp; ++w) off += wcount[w];
        off += __popc(bal & ((1u << lane) - 1u));
        if (sel && off < (unsigned long long)m) idx[off] = q;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wcount[w];
            base += tot;
        }
    }
}

__global__ void iota_kernel(int64_t* idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        idx[i] = i;
}

// Per-device scratch of the sampler (state, histogram, block counts).  Calls on different
// streams are ordered on the device through `done` (the event after the last user's kernels),
// so two samplers never share the scratch at the same time; no host synchronisation.
struct SampleScratch {
    std::mutex mu;
    DevBuf state, hist, counts;
    cudaEvent_t done = nullptr;
    bool used = false;
};
static SampleScratch g_sample_scratch[64];

fst_status sample_rows(uint64_t seed, int64_t Q, int64_t m, int64_t* idx, cudaStream_t s) {
    if (m <= 0 || Q <= 0) return FST_OK;
    if (m >= Q) {
        int grid = (int)((Q + 255) / 256);
        if (grid > 4 * sm_count()) grid = 4 * sm_count();
        iota_kernel<<<grid, 256, 0, s>>>(idx, Q);
        FST_CHECK_LAUNCH();
        return FST_OK;
    }
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    SampleScratch& sc = g_sample_scratch[dev];
    std::lock_guard<std::mutex> lk(sc.mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FST_CUDA(cudaStreamIsCapturing(s, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;   // no cross-stream ordering inside a capture
    if (!capturing) {
        if (!sc.done) FST_CUDA(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming));
        if (sc.used) FST_CUDA(cudaStreamWaitEvent(s, sc.done, 0));
    }
    const int sms = sm_count();
    int64_t nblocks = (Q + 8191) / 8192;
    if (nblocks < 1) nblocks = 1;
    if (nblocks > 16 * sms) nblocks = 16 * sms;
    const int64_t rows_per_block = (Q + nblocks - 1) / nblocks;
    FST_TRY(sc.state.ensure(sizeof(SelectState)));
    FST_TRY(sc.hist.ensure(kBins * sizeof(unsigned int)));
    FST_TRY(sc.counts.ensure((size_t)nblocks * sizeof(unsigned long long)));
    SelectState* st = sc.state.as<SelectState>();
    unsigned int* hist = sc.hist.as<unsigned int>();
    init_state_kernel<<<1, 256, 0, s>>>(st, (unsigned long long)m, hist);
    FST_CHECK_LAUNCH();
    int hgrid = (int)((Q + 1023) / 1024);
    if (hgrid > 4 * sms) hgrid = 4 * sms;
    for (int pass = 0; pass < kPasses; ++pass) {
        select_hist_kernel<<<hgrid, 512, 0, s>>>(seed, Q, pass, st, hist);
        FST_CHECK_LAUNCH();
        select_pick_kernel<<<1, 32, 0, s>>>(pass, st, hist);
        FST_CHECK_LAUNCH();
    }
    unsigned long long* counts = sc.counts.as<unsigned long long>();
    compact_count_kernel<<<(unsigned)nblocks, kCompactBlock, 0, s>>>(seed, Q, rows_per_block, st, counts);
    FST_CHECK_LAUNCH();
    scan_counts_kernel<<<1, 1024, 0, s>>>(counts, (int)nblocks);
    FST_CHECK_LAUNCH();
    compact_write_kernel<<<(unsigned)nblocks, kCompactBlock, 0, s>>>(seed, Q, rows_per_block, st, counts,
                                                                      idx, m);
    FST_CHECK_LAUNCH();
    if (!capturing) {
        FST_CUDA(cudaEventRecord(sc.done, s));
        sc.used = true;
    }
    return FST_OK;
}

}  // namespace fst

using namespace fst;

extern "C" fst_status fst_sample_rows(uint64_t seed, int64_t Q, int64_t m, int64_t* idx, fst_stream stream) {
    FST_REQUIRE(Q >= 0 && m >= 0, "Q and m must be non-negative");
    if (Q == 0 || m == 0) return FST_OK;
    FST_REQUIRE(idx != nullptr, "idx is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(pointer_device(idx) == dev, "idx must be device memory of device %d", dev);
    return sample_rows(seed, Q, m, idx, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ sampling without allocation
// fst_sample_rows_static: the same sampler for callers that must not allocate device
// memory, for example an in-situ visualisation hook running inside a simulation that has
// already handed all device memory to its own pool, or a latency-bound loop that cannot
// afford cudaMalloc's implicit device synchronisation.  Its scratch (selection state,
// digit histogram, per-block counts) lives in one file-scope device array that every GPU
// which loads this library keeps until the process exits.
namespace fst {

constexpr int64_t kStaticRowsPerBlock = 8192;
constexpr int64_t kStaticMaxBlocks = 65536;                 // rows per call <= 2^29
constexpr size_t kStaticStateBytes = 256;
constexpr size_t kStaticScratchBytes =
    kStaticStateBytes + kBins * sizeof(unsigned int) + kStaticMaxBlocks * sizeof(unsigned long long);

static __device__ __align__(256) unsigned char g_sample_static_scratch[kStaticScratchBytes];

// Host code only sees a stand-in for the array's name: the device address is resolved
// once per device, with that device current, and cached.
static void* g_static_scratch_addr[64];
static std::mutex g_static_scratch_mu;

static fst_status static_scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_static_scratch_mu);
    if (!g_static_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sample_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(sampler scratch)", __FILE__, __LINE__);
        g_static_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_static_scratch_addr[dev]);
    return FST_OK;
}

}  // namespace fst

extern "C" fst_status fst_sample_rows_static(uint64_t seed, int64_t Q, int64_t m, int64_t* idx,
                                             fst_stream stream) {
    FST_REQUIRE(Q >= 0 && m >= 0, "Q and m must be non-negative");
    FST_REQUIRE(Q <= kStaticRowsPerBlock * kStaticMaxBlocks,
                "fst_sample_rows_static handles at most %lld rows (Q = %lld); use fst_sample_rows",
                (long long)(kStaticRowsPerBlock * kStaticMaxBlocks), (long long)Q);
    if (Q == 0 || m == 0) return FST_OK;
    FST_REQUIRE(idx != nullptr, "idx is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    FST_REQUIRE(pointer_device(idx) == dev, "idx must be device memory of device %d", dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (m >= Q) {
        int grid = (int)((Q + 255) / 256);
        if (grid > 4 * sm_count()) grid = 4 * sm_count();
        iota_kernel<<<grid, 256, 0, s>>>(idx, Q);
        FST_CHECK_LAUNCH();
        return FST_OK;
    }
    unsigned char* base = nullptr;
    FST_TRY(static_scratch_address(dev, &base));
    SelectState* st = reinterpret_cast<SelectState*>(base);
    unsigned int* hist = reinterpret_cast<unsigned int*>(base + kStaticStateBytes);
    unsigned long long* counts =
        reinterpret_cast<unsigned long long*>(base + kStaticStateBytes + kBins * sizeof(unsigned int));
    const int64_t nblocks = (Q + kStaticRowsPerBlock - 1) / kStaticRowsPerBlock;
    // the state and the histogram start from zero on every call; counts are fully rewritten
    init_state_kernel<<<1, 256, 0, s>>>(st, (unsigned long long)m, hist);
    FST_CHECK_LAUNCH();
    int hgrid = (int)((Q + 1023) / 1024);
    if (hgrid > 4 * sm_count()) hgrid = 4 * sm_count();
    for (int pass = 0; pass < kPasses; ++pass) {
        select_hist_kernel<<<hgrid, 512, 0, s>>>(seed, Q, pass, st, hist);
        FST_CHECK_LAUNCH();
        select_pick_kernel<<<1, 32, 0, s>>>(pass, st, hist);
        FST_CHECK_LAUNCH();
    }
    compact_count_kernel<<<(unsigned)nblocks, kCompactBlock, 0, s>>>(seed, Q, kStaticRowsPerBlock, st, counts);
    FST_CHECK_LAUNCH();
    scan_counts_kernel<<<1, 1024, 0, s>>>(counts, (int)nblocks);
    FST_CHECK_LAUNCH();
    compact_write_kernel<<<(unsigned)nblocks, kCompactBlock, 0, s>>>(seed, Q, kStaticRowsPerBlock, st, counts,
                                                                      idx, m);
    FST_CHECK_LAUNCH();
    return FST_OK;
}
