// fst_internal.cuh -- shared declarations of libfst's translation units.
//
// Device data layout of a model (all on the device the model was created on):
//   W64[k], W32[k]  dense coefficient matrix of mode k, (p_k+1) x r_k row-major,
//                   entry [n][j] = W^k_{n,j} * sqrt(2n+1), i.e. the coefficient of the
//                   plain Legendre polynomial L_n in w^(k)_j (eq. sparse, Sec. 2).
//   rowmask[k]      one byte per degree n: 1 if row n of W^k has a nonzero.
//   alpha64/32      core, C order [j1][j2][j3] (eq. func_tuck).
//   tc_*            tensor-core operand images of the core (see eval_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "fst.h"

namespace fst {

void set_error(const char* fmt, ...);
fst_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define FST_CUDA(expr)                                                                  \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) return ::fst::cuda_fail(_e, #expr, __FILE__, __LINE__);  \
    } while (0)
// Every kernel launch in libfst is followed by FST_CHECK_LAUNCH(), which also counts it;
// graph replays add their kernel nodes with count_launches.
void count_launch();
void count_launches(uint64_t n);
#define FST_CHECK_LAUNCH()          \
    do {                            \
        ::fst::count_launch();      \
        FST_CUDA(cudaGetLastError()); \
    } while (0)
#define FST_TRY(expr)                        \
    do {                                     \
        fst_status _s = (expr);              \
        if (_s != FST_OK) return _s;         \
    } while (0)
#define FST_REQUIRE(cond, ...)                       \
    do {                                             \
        if (!(cond)) {                               \
            ::fst::set_error(__VA_ARGS__);           \
            return FST_EINVAL;                       \
        }                                            \
    } while (0)

// A device buffer that only grows.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    fst_status ensure(size_t need);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Per-device scratch that refits of different models on different streams may need at the
// same time (the Gram's operand copies).  A caller leases the first slot nobody holds (one
// caller alone always gets slot 0), its stream waits on the device for the slot's previous
// user, and the lease records the caller's use once its work is enqueued; the host holds the
// slot only while enqueueing.  Growing a buffer first waits for the previous user to finish.
constexpr int kScratchSlots = 4;
struct ScratchSlot {
    std::mutex mu;
    DevBuf buf[3];
    cudaEvent_t done = nullptr;
    bool used = false;
};
struct ScratchPool {
    ScratchSlot slot[kScratchSlots];
};
class SlotLease {
  public:
    explicit SlotLease(ScratchPool& pool) {
        for (int i = 0; i < kScratchSlots && !sl_; ++i)
            if (pool.slot[i].mu.try_lock()) sl_ = &pool.slot[i];
        if (!sl_) {
            pool.slot[0].mu.lock();
            sl_ = &pool.slot[0];
        }
    }
    // a lease that began records its use even when the caller gave up half-way, since
    // some of its work may already be enqueued
    ~SlotLease() {
        if (began_) {
            if (cudaEventRecord(sl_->done, s_) == cudaSuccess) sl_->used = true;
        }
        sl_->mu.unlock();
    }
    SlotLease(const SlotLease&) = delete;
    SlotLease& operator=(const SlotLease&) = delete;
    fst_status begin(cudaStream_t s) {
        if (!sl_->done) FST_CUDA(cudaEventCreateWithFlags(&sl_->done, cudaEventDisableTiming));
        if (sl_->used) FST_CUDA(cudaStreamWaitEvent(s, sl_->done, 0));
        s_ = s;
        began_ = true;
        return FST_OK;
    }
    fst_status ensure(int i, size_t bytes) {
        if (bytes > sl_->buf[i].bytes && sl_->used) FST_CUDA(cudaEventSynchronize(sl_->done));
        return sl_->buf[i].ensure(bytes);
    }
    template <typename T> T* as(int i) const { return sl_->buf[i].as<T>(); }
  private:
    ScratchSlot* sl_ = nullptr;
    cudaStream_t s_ = nullptr;
    bool began_ = false;
};

// A captured triangular-solve sequence (chol.cu), replayed with one graph launch.
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    const void* L = nullptr;
    const void* LT = nullptr;
    const void* Linv = nullptr;
    void* x = nullptr;
    const int* stop = nullptr;
    int R = 0, elem = 0;
    uint64_t nodes = 0;
    DevBuf sync;                 // error word, ticket, ready flags of the one-launch solves
    void release();
};

// Scratch of the refit, kept inside the model between calls.
struct RefitScratch {
    DevBuf idx, U[3], b, G, G64, res, g, z, delta, alpha, norms, flag, Linv, LT, xw, yw, pcg, chol_ws, atr_part,
        gram_err, pcg_state, mix;
    SolveGraph solve;
};

}  // namespace fst

struct fst_eval_plan;

struct fst_model {
    int device = 0;
    int r[3] = {0, 0, 0};
    int p[3] = {0, 0, 0};
    int p_eff[3] = {0, 0, 0};    // 1 + highest degree with a nonzero coefficient
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    std::vector<int32_t> colptr[3], rowidx[3];
    std::vector<double> val[3];
    std::vector<double> alpha;   // host copy of the core

    double* W64[3] = {nullptr, nullptr, nullptr};
    float* W32[3] = {nullptr, nullptr, nullptr};
    // wavelet columns (Sec. 4.2): the space W_{s,q} (wav_s < 0: none), which columns use it,
    // and their coefficients on the finest cells as local Legendre expansions
    int wav_s = -1, wav_q = 0;
    int wav_cols[3] = {0, 0, 0};
    std::vector<uint8_t> colwav[3];
    double* Wp64[3] = {nullptr, nullptr, nullptr};
    float* Wp32[3] = {nullptr, nullptr, nullptr};
    uint8_t* rowmask[3] = {nullptr, nullptr, nullptr};
    double* alpha64 = nullptr;
    float* alpha32 = nullptr;

    // tensor-core images of the core, built on demand (eval_tc.cu): one slot per kind
    // (precision, evaluator variant, r3 padding), so preparing one kind never rewrites an
    // image that a batch of another kind may still be reading
    struct TcImage {
        void* ptr = nullptr;
        size_t bytes = 0;
        int kind = -1;      // -1: stale (the core changed) or unused
    };
    TcImage tc_img[8];
    const void* tc_core = nullptr;          // the image of the last prepared kind
    long long tc_core_kind_version = 0;     // bumped whenever an image is (re)built
    // cached single-instance tensor-core work list (eval_tc.cu)
    fst_eval_plan* eval_plan = nullptr;
    long long eval_plan_n = -1, eval_plan_core = -1;
    int eval_plan_prec = -1;

    fst::RefitScratch rs;
    std::recursive_mutex mu;   // re-entered by single-instance evaluations that build a work list

    int R() const { return r[0] * r[1] * r[2]; }
};

namespace fst {

void plan_free(fst_eval_plan* p);

// Multiwavelet spaces W_{s,q} (wavelet.cu): Gauss-Legendre rules, the mother wavelets as
// local Legendre expansions on the two halves, the finest-cell expansion of one function of
// W_{s,q}, and the space's design at the fit's grid nodes.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
std::vector<double> mother_wavelets(int q);
void wavelet_piecewise(int s, int q, int idx, const std::vector<double>& mw, std::vector<double>& out);
void wavelet_grid_design(int N, int s, int q, std::vector<double>& Phi);
void function_samples(int p, int s, int q, const std::vector<const int32_t*>& rows, const std::vector<const double*>& vals,
                      const std::vector<int>& len, const std::vector<uint8_t>& is_wav, std::vector<double>& S, int& L);

// Device upload of the derived layouts after the host copy changed.
fst_status model_upload_core(fst_model* m);
fst_status model_invalidate_tc(fst_model* m);

// Raise a kernel's dynamic shared-memory limit on the current device to at least `bytes`.
// The limit is a property of the function, not of a launch, and it only grows here, so
// launches from host threads on different streams never lower it under one another.
fst_status allow_dynamic_smem(const void* func, size_t bytes);
template <typename K>
fst_status allow_smem(K* kernel, size_t bytes) {
    return allow_dynamic_smem(reinterpret_cast<const void*>(kernel), bytes);
}

// Key of row q under a seed: the (q+1)-th output of a splitmix64 stream started at the seed
// (Steele, Lea, Flood, OOPSLA 2014).  The sampler keeps the rows with the smallest keys; the
// mixed refit takes its random signs from the top bit.
__host__ __device__ __forceinline__ uint64_t splitmix_key(uint64_t seed, uint64_t q) {
    uint64_t z = seed + (q + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Number of SMs of the current device (cached).
int sm_count();
// Device of a pointer, or -1 for host memory.
int pointer_device(const void* p);

// Evaluation entry points used by the refit (residual path).
template <typename T>
fst_status eval_simt_launch(const fst_model* m, const T* xyz, int64_t n, T* out, cudaStream_t s);

// Row sampler (sample.cu).
fst_status sample_rows(uint64_t seed, int64_t Q, int64_t m, int64_t* idx, cudaStream_t s);

// Tensor-core eval (eval_tc.cu).
fst_status eval_tc_launch(fst_model* m, const float* xyz, int64_t n, float* out, fst_prec prec,
                          cudaStream_t s);
// Tensor-core Gram (gram_tc.cu): lower triangle of G = A^T A, FP32 accumulation.
fst_status gram_tc_launch(const fst_model* m, const float* U1, const float* U2, const float* U3,
                          int64_t mrows, float* G, fst_prec prec, cudaStream_t s);
// The same G from a packed BF16 / TF32 / BF16 hi+lo copy of the Khatri-Rao operand
// (gram_pk.cu); FST_ENOMEM if that copy cannot be allocated.
fst_status gram_pk_launch(const fst_model* m, const float* U1, const float* U2, const float* U3, int64_t rows,
                          float* G, fst_prec prec, cudaStream_t s);
// The packed-operand Gram of rows u1 (x) u2 (x) u3 (gram_pk.cu): G lower triangle, err the
// expired-wait word; FST_ENOMEM when the packed copy does not fit.
fst_status gram_pk_rows(const float* U1, const float* U2, const float* U3, int64_t m, int r1, int r2, int r3,
                        float* G, fst_prec prec, int* err, cudaStream_t s);
// PT[(i r2 + j) mpad + q] = w1_i(q) w2_j(q), U3T[k mpad + q] = w3_k(q), zero for q >= m.
fst_status pair_products(const float* U1, const float* U2, const float* U3, int64_t m, int64_t mpad, int r1, int r2,
                         int r3, float* PT, float* U3T, cudaStream_t s);

// Cholesky and triangular solves (chol.cu).
template <typename T>
fst_status cholesky_lower(T* G, int R, int* d_flag, DevBuf& ws, cudaStream_t s);
template <typename T>
fst_status chol_invert_diag(const T* L, int R, T* Linv, cudaStream_t s);   // 64x64 diagonal-block inverses, then the forward and backward link matrices (3 x ceil(R/64) x 64^2 values)
template <typename T>
fst_status chol_solve(const T* L, const T* LT, const T* Linv, int R, T* x, T* y, int* sync, cudaStream_t s,
                      const int* stop = nullptr);  // x <- (L L^T)^-1 x; nothing when *stop is set
// The same through a CUDA graph captured on first use for (L, Linv, x, y, R) and replayed.
template <typename T>
fst_status chol_solve_graph(SolveGraph& g, const T* L, const T* LT, const T* Linv, int R, T* x, T* y,
                            cudaStream_t s, const int* stop = nullptr);
// LT = L^T (the strict upper blocks used by the backward solve)
template <typename T>
fst_status chol_transpose(const T* L, int R, T* LT, cudaStream_t s);

// Grouped refits: the factorisations of several FP32 normal matrices in shared launches,
// and the solves of several factored matrices in one launch per direction.
struct CholItem {
    float* G;
    int R;
    int* flag;      // [0] pivot flag
    DevBuf* ws;     // the matrix's factorisation workspace
};
fst_status cholesky_lower_group(const std::vector<CholItem>& items, DevBuf& sched, int* gerr, cudaStream_t s);
struct SolveJob {
    const void* L;
    const void* LT;
    const void* Linv;   // diagonal-block inverses, then the forward and backward link matrices
    void* x;            // right-hand side in, solution out
    void* y;            // scratch
    const int* stop;    // nothing is solved while *stop is set
    int R, nblk;
};
template <typename T>
fst_status chol_solve_group(const SolveJob* jobs, int njobs, int maxR, const int* tmap, int tickets, int* sync,
                            cudaStream_t s);
std::vector<int> solve_tickets(const std::vector<int>& R);

}  // namespace fst
