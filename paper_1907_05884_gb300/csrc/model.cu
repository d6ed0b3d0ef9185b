// model.cu -- model objects, model files, error reporting (C ABI in include/fst.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>

#include "fst_internal.cuh"

#define FST_STR_(x) #x
#define FST_STR(x) FST_STR_(x)

namespace fst {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void SolveGraph::release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    exec = nullptr;
    cap = nullptr;
    L = LT = Linv = nullptr;
    x = nullptr;
    R = elem = 0;
    nodes = 0;
    sync.release();
}

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

fst_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? FST_ENOMEM : FST_ECUDA;
}

fst_status allow_dynamic_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return FST_OK;
    FST_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return FST_OK;
}

fst_status DevBuf::ensure(size_t need) {
    if (need <= bytes) return FST_OK;
    release();
    size_t want = need < 256 ? 256 : need;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        (void)cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
        return FST_ENOMEM;
    }
    bytes = want;
    return FST_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

int sm_count() {
    static int cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

int pointer_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device;
    return -1;
}

static void free_device(fst_model* m) {
    for (int k = 0; k < 3; ++k) {
        if (m->W64[k]) cudaFree(m->W64[k]);
        if (m->W32[k]) cudaFree(m->W32[k]);
        if (m->rowmask[k]) cudaFree(m->rowmask[k]);
        if (m->Wp64[k]) cudaFree(m->Wp64[k]);
        if (m->Wp32[k]) cudaFree(m->Wp32[k]);
        m->W64[k] = nullptr;
        m->W32[k] = nullptr;
        m->rowmask[k] = nullptr;
        m->Wp64[k] = nullptr;
        m->Wp32[k] = nullptr;
    }
    if (m->alpha64) cudaFree(m->alpha64);
    if (m->alpha32) cudaFree(m->alpha32);
    for (auto& t : m->tc_img) {
        if (t.ptr) cudaFree(t.ptr);
        t.ptr = nullptr;
        t.bytes = 0;
        t.kind = -1;
    }
    if (m->eval_plan) plan_free(m->eval_plan);
    m->eval_plan = nullptr;
    m->alpha64 = nullptr;
    m->alpha32 = nullptr;
    m->tc_core = nullptr;
    RefitScratch& s = m->rs;
    s.idx.release();
    for (int k = 0; k < 3; ++k) s.U[k].release();
    s.b.release();
    s.G.release();
    s.G64.release();
    s.res.release();
    s.g.release();
    s.z.release();
    s.delta.release();
    s.alpha.release();
    s.norms.release();
    s.flag.release();
    s.Linv.release();
    s.LT.release();
    s.chol_ws.release();
    s.atr_part.release();
    s.gram_err.release();
    s.pcg_state.release();
    s.mix.release();
    s.xw.release();
    s.yw.release();
    s.pcg.release();
    s.solve.release();
}

fst_status model_invalidate_tc(fst_model* m) {
    // the core changed: every image is stale (its buffer is reused by the next build)
    for (auto& t : m->tc_img) t.kind = -1;
    ++m->tc_core_kind_version;
    return FST_OK;
}

fst_status model_upload_core(fst_model* m) {
    const size_t R = (size_t)m->R();
    std::vector<float> a32(R);
    for (size_t i = 0; i < R; ++i) a32[i] = (float)m->alpha[i];
    FST_CUDA(cudaMemcpy(m->alpha64, m->alpha.data(), R * sizeof(double), cudaMemcpyHostToDevice));
    FST_CUDA(cudaMemcpy(m->alpha32, a32.data(), R * sizeof(float), cudaMemcpyHostToDevice));
    return model_invalidate_tc(m);
}

static bool is_wavelet_col(const fst_wavelet_desc* w, int k, int j) {
    return w && w->col_wavelet[k] && w->col_wavelet[k][j];
}

static fst_status validate_desc(const fst_model_desc* d, const fst_wavelet_desc* w) {
    FST_REQUIRE(d != nullptr, "model description is NULL");
    int nwav = 0;
    if (w) {
        FST_REQUIRE(w->level >= 0 && w->level <= FST_MAX_WAVELET_LEVEL, "wavelet level %d outside [0,%d]", w->level,
                    FST_MAX_WAVELET_LEVEL);
        FST_REQUIRE(w->degree >= 0 && w->degree <= FST_MAX_WAVELET_DEGREE, "wavelet degree %d outside [0,%d]",
                    w->degree, FST_MAX_WAVELET_DEGREE);
        nwav = (w->degree + 1) << w->level;
        FST_REQUIRE(nwav <= 256, "wavelet space of dimension %d above 256", nwav);
    }
    FST_REQUIRE(d->alpha != nullptr, "alpha is NULL");
    for (int k = 0; k < 3; ++k) {
        FST_REQUIRE(d->r[k] >= 1 && d->r[k] <= FST_MAX_RANK, "rank r[%d]=%d outside [1,%d]", k,
                    d->r[k], FST_MAX_RANK);
        FST_REQUIRE(d->p[k] >= 0 && d->p[k] <= FST_MAX_DEGREE, "degree p[%d]=%d outside [0,%d]", k,
                    d->p[k], FST_MAX_DEGREE);
        FST_REQUIRE(d->colptr[k] != nullptr, "colptr[%d] is NULL", k);
        FST_REQUIRE(isfinite(d->lo[k]) && isfinite(d->hi[k]) && d->hi[k] > d->lo[k],
                    "box of mode %d is empty or not finite", k);
        const int32_t* cp = d->colptr[k];
        FST_REQUIRE(cp[0] == 0, "colptr[%d][0] must be 0", k);
        for (int j = 0; j < d->r[k]; ++j) {
            FST_REQUIRE(cp[j + 1] >= cp[j], "colptr[%d] decreases at %d", k, j);
            const bool wc = is_wavelet_col(w, k, j);
            for (int e = cp[j]; e < cp[j + 1]; ++e) {
                FST_REQUIRE(d->rowidx[k] && d->val[k], "rowidx/val[%d] is NULL", k);
                int n = d->rowidx[k][e];
                if (wc)
                    FST_REQUIRE(n >= 0 && n < nwav, "wavelet index %d of mode %d column %d outside [0,%d)", n, k,
                                j, nwav);
                else
                    FST_REQUIRE(n >= 0 && n <= d->p[k], "degree %d of mode %d column %d outside [0,%d]",
                                n, k, j, d->p[k]);
                FST_REQUIRE(e == cp[j] || n > d->rowidx[k][e - 1],
                            "degrees of mode %d column %d not strictly increasing", k, j);
                FST_REQUIRE(isfinite(d->val[k][e]), "non-finite coefficient in mode %d", k);
            }
        }
    }
    return FST_OK;
}

}  // namespace fst

using namespace fst;

static fst_status create_model(const fst_model_desc* desc, const fst_wavelet_desc* wav, fst_model** out) {
    FST_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    FST_TRY(validate_desc(desc, wav));
    std::unique_ptr<fst_model> m(new fst_model());
    FST_CUDA(cudaGetDevice(&m->device));
    for (int k = 0; k < 3; ++k) {
        m->r[k] = desc->r[k];
        m->p[k] = desc->p[k];
        m->lo[k] = desc->lo[k];
        m->hi[k] = desc->hi[k];
        const int nnz = desc->colptr[k][desc->r[k]];
        m->colptr[k].assign(desc->colptr[k], desc->colptr[k] + desc->r[k] + 1);
        m->rowidx[k].assign(desc->rowidx[k], desc->rowidx[k] + nnz);
        m->val[k].assign(desc->val[k], desc->val[k] + nnz);
        m->colwav[k].assign(desc->r[k], 0);
        for (int j = 0; j < desc->r[k]; ++j)
            if (is_wavelet_col(wav, k, j)) {
                m->colwav[k][j] = 1;
                ++m->wav_cols[k];
            }
    }
    if (wav && m->wav_cols[0] + m->wav_cols[1] + m->wav_cols[2] > 0) {
        m->wav_s = wav->level;
        m->wav_q = wav->degree;
    }
    const size_t R = (size_t)m->R();
    m->alpha.assign(desc->alpha, desc->alpha + R);
    for (size_t i = 0; i < R; ++i)
        FST_REQUIRE(isfinite(m->alpha[i]), "non-finite core entry %zu", i);

    fst_status st = FST_OK;
    for (int k = 0; k < 3 && st == FST_OK; ++k) {
        const int np = m->p[k] + 1, rk = m->r[k];
        std::vector<double> W(np * (size_t)rk, 0.0);
        std::vector<float> W32(np * (size_t)rk, 0.0f);
        std::vector<uint8_t> mask(np, 0);
        int pe = 1;
        for (int j = 0; j < rk; ++j)
            for (int e = m->colptr[k][j]; e < m->colptr[k][j + 1] && !m->colwav[k][j]; ++e) {
                const int n = m->rowidx[k][e];
                const double c = m->val[k][e] * sqrt(2.0 * n + 1.0);
                W[(size_t)n * rk + j] = c;
                if (c != 0.0) {
                    mask[n] = 1;
                    if (n + 1 > pe) pe = n + 1;
                }
            }
        for (size_t i = 0; i < W.size(); ++i) W32[i] = (float)W[i];
        m->p_eff[k] = pe;
        cudaError_t e1 = cudaMalloc(&m->W64[k], W.size() * sizeof(double));
        cudaError_t e2 = cudaMalloc(&m->W32[k], W.size() * sizeof(float));
        cudaError_t e3 = cudaMalloc(&m->rowmask[k], mask.size());
        if (e1 || e2 || e3) {
            st = cuda_fail(e1 ? e1 : e2 ? e2 : e3, "cudaMalloc(model)", __FILE__, __LINE__);
            break;
        }
        e1 = cudaMemcpy(m->W64[k], W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice);
        e2 = cudaMemcpy(m->W32[k], W32.data(), W32.size() * sizeof(float), cudaMemcpyHostToDevice);
        e3 = cudaMemcpy(m->rowmask[k], mask.data(), mask.size(), cudaMemcpyHostToDevice);
        if (e1 || e2 || e3) {
            st = cuda_fail(e1 ? e1 : e2 ? e2 : e3, "cudaMemcpy(model)", __FILE__, __LINE__);
            break;
        }
        if (m->wav_cols[k] == 0) continue;
        // wavelet columns: the exact expansion of each on the finest cells, as coefficients of
        // sqrt(2n+1) L_n of the cell's local coordinate (sqrt(2n+1) folded in)
        const int nq = m->wav_q + 1, cells = 1 << m->wav_s;
        const std::vector<double> mw = mother_wavelets(m->wav_q);
        std::vector<double> Wp((size_t)cells * nq * rk, 0.0), pw;
        for (int j = 0; j < rk; ++j) {
            if (!m->colwav[k][j]) continue;
            for (int e = m->colptr[k][j]; e < m->colptr[k][j + 1]; ++e) {
                wavelet_piecewise(m->wav_s, m->wav_q, m->rowidx[k][e], mw, pw);
                for (int f = 0; f < cells; ++f)
                    for (int n = 0; n < nq; ++n)
                        Wp[((size_t)f * nq + n) * rk + j] += m->val[k][e] * pw[(size_t)f * nq + n];
            }
        }
        std::vector<float> Wp32(Wp.size());
        for (int f = 0; f < cells; ++f)
            for (int n = 0; n < nq; ++n)
                for (int j = 0; j < rk; ++j) {
                    double& v = Wp[((size_t)f * nq + n) * rk + j];
                    v *= sqrt(2.0 * n + 1.0);
                    Wp32[((size_t)f * nq + n) * rk + j] = (float)v;
                }
        e1 = cudaMalloc(&m->Wp64[k], Wp.size() * sizeof(double));
        e2 = cudaMalloc(&m->Wp32[k], Wp.size() * sizeof(float));
        if (e1 || e2) {
            st = cuda_fail(e1 ? e1 : e2, "cudaMalloc(model)", __FILE__, __LINE__);
            break;
        }
        e1 = cudaMemcpy(m->Wp64[k], Wp.data(), Wp.size() * sizeof(double), cudaMemcpyHostToDevice);
        e2 = cudaMemcpy(m->Wp32[k], Wp32.data(), Wp32.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e1 || e2) st = cuda_fail(e1 ? e1 : e2, "cudaMemcpy(model)", __FILE__, __LINE__);
    }
    if (st == FST_OK) {
        cudaError_t e1 = cudaMalloc(&m->alpha64, R * sizeof(double));
        cudaError_t e2 = cudaMalloc(&m->alpha32, R * sizeof(float));
        if (e1 || e2) st = cuda_fail(e1 ? e1 : e2, "cudaMalloc(core)", __FILE__, __LINE__);
    }
    if (st == FST_OK) st = model_upload_core(m.get());
    if (st != FST_OK) {
        free_device(m.get());
        return st;
    }
    *out = m.release();
    return FST_OK;
}

extern "C" fst_status fst_model_create(const fst_model_desc* desc, fst_model** out) {
    return create_model(desc, nullptr, out);
}

extern "C" fst_status fst_model_create_wavelet(const fst_model_desc* desc, const fst_wavelet_desc* wav,
                                               fst_model** out) {
    FST_REQUIRE(wav != nullptr, "wavelet description is NULL");
    return create_model(desc, wav, out);
}

extern "C" fst_status fst_model_read_wavelet(const fst_model* m, int32_t* level, int32_t* degree,
                                             uint8_t* col_wavelet[3]) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    if (level) *level = m->wav_s;
    if (degree) *degree = m->wav_s >= 0 ? m->wav_q : 0;
    for (int k = 0; k < 3; ++k)
        if (col_wavelet && col_wavelet[k]) memcpy(col_wavelet[k], m->colwav[k].data(), m->r[k]);
    return FST_OK;
}

extern "C" void fst_model_free(fst_model* m) {
    if (!m) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    free_device(m);
    cudaSetDevice(cur);
    delete m;
}

extern "C" fst_status fst_model_shape(const fst_model* m, int32_t r[3], int32_t p[3],
                                      int32_t nnz[3]) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    for (int k = 0; k < 3; ++k) {
        if (r) r[k] = m->r[k];
        if (p) p[k] = m->p[k];
        if (nnz) nnz[k] = (int32_t)m->val[k].size();
    }
    return FST_OK;
}

extern "C" fst_status fst_model_read(const fst_model* m, int32_t* colptr[3], int32_t* rowidx[3],
                                     double* val[3], double* alpha, double lo[3], double hi[3]) {
    FST_REQUIRE(m != nullptr, "model is NULL");
    for (int k = 0; k < 3; ++k) {
        if (colptr && colptr[k])
            memcpy(colptr[k], m->colptr[k].data(), m->colptr[k].size() * sizeof(int32_t));
        if (rowidx && rowidx[k])
            memcpy(rowidx[k], m->rowidx[k].data(), m->rowidx[k].size() * sizeof(int32_t));
        if (val && val[k]) memcpy(val[k], m->val[k].data(), m->val[k].size() * sizeof(double));
        if (lo) lo[k] = m->lo[k];
        if (hi) hi[k] = m->hi[k];
    }
    if (alpha) memcpy(alpha, m->alpha.data(), m->alpha.size() * sizeof(double));
    return FST_OK;
}

extern "C" fst_status fst_model_set_core(fst_model* m, const double* alpha) {
    FST_REQUIRE(m != nullptr && alpha != nullptr, "model or alpha is NULL");
    const size_t R = (size_t)m->R();
    for (size_t i = 0; i < R; ++i) FST_REQUIRE(isfinite(alpha[i]), "non-finite core entry %zu", i);
    std::lock_guard<std::recursive_mutex> lk(m->mu);
    m->alpha.assign(alpha, alpha + R);
    int cur = 0;
    cudaGetDevice(&cur);
    FST_CUDA(cudaSetDevice(m->device));
    fst_status st = model_upload_core(m);
    cudaSetDevice(cur);
    return st;
}

// ------------------------------------------------------------------ model files
static const char kMagic[4] = {'F', 'S', 'T', 'M'};
static const uint32_t kVersion = 2;    // 2 adds the wavelet section; 1 is still read

extern "C" fst_status fst_model_save(const fst_model* m, const char* path) {
    FST_REQUIRE(m != nullptr && path != nullptr, "model or path is NULL");
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return FST_EINVAL;
    }
    bool ok = fwrite(kMagic, 1, 4, f) == 4;
    ok = ok && fwrite(&kVersion, 4, 1, f) == 1;
    int32_t hdr[6] = {m->r[0], m->r[1], m->r[2], m->p[0], m->p[1], m->p[2]};
    ok = ok && fwrite(hdr, 4, 6, f) == 6;
    ok = ok && fwrite(m->lo, 8, 3, f) == 3 && fwrite(m->hi, 8, 3, f) == 3;
    for (int k = 0; k < 3 && ok; ++k) {
        int32_t nnz = (int32_t)m->val[k].size();
        ok = fwrite(&nnz, 4, 1, f) == 1;
        ok = ok && fwrite(m->colptr[k].data(), 4, m->colptr[k].size(), f) == m->colptr[k].size();
        ok = ok && fwrite(m->rowidx[k].data(), 4, nnz, f) == (size_t)nnz;
        ok = ok && fwrite(m->val[k].data(), 8, nnz, f) == (size_t)nnz;
    }
    ok = ok && fwrite(m->alpha.data(), 8, m->alpha.size(), f) == m->alpha.size();
    int32_t wv[2] = {m->wav_s, m->wav_s >= 0 ? m->wav_q : 0};
    ok = ok && fwrite(wv, 4, 2, f) == 2;
    for (int k = 0; k < 3 && ok && m->wav_s >= 0; ++k)
        ok = fwrite(m->colwav[k].data(), 1, m->r[k], f) == (size_t)m->r[k];
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return FST_EINVAL;
    }
    return FST_OK;
}

extern "C" fst_status fst_model_load(const char* path, fst_model** out) {
    FST_REQUIRE(path != nullptr && out != nullptr, "path or out is NULL");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return FST_EINVAL;
    }
    struct Closer { FILE* f; ~Closer() { fclose(f); } } closer{f};
    char magic[4];
    uint32_t ver = 0;
    int32_t hdr[6];
    fst_model_desc d;
    memset(&d, 0, sizeof d);
    if (fread(magic, 1, 4, f) != 4 || memcmp(magic, kMagic, 4) != 0 || fread(&ver, 4, 1, f) != 1 ||
        (ver != 1 && ver != kVersion) || fread(hdr, 4, 6, f) != 6 || fread(d.lo, 8, 3, f) != 3 ||
        fread(d.hi, 8, 3, f) != 3) {
        set_error("%s: not an FSTM v%u file", path, kVersion);
        return FST_EFORMAT;
    }
    for (int k = 0; k < 3; ++k) {
        d.r[k] = hdr[k];
        d.p[k] = hdr[3 + k];
        if (d.r[k] < 1 || d.r[k] > FST_MAX_RANK || d.p[k] < 0 || d.p[k] > FST_MAX_DEGREE) {
            set_error("%s: ranks/degrees out of range", path);
            return FST_EFORMAT;
        }
    }
    std::vector<int32_t> cp[3], ri[3];
    std::vector<double> vv[3];
    for (int k = 0; k < 3; ++k) {
        int32_t nnz = -1;
        if (fread(&nnz, 4, 1, f) != 1 || nnz < 0 || nnz > d.r[k] * std::max(d.p[k] + 1, 256)) {
            set_error("%s: bad coefficient count", path);
            return FST_EFORMAT;
        }
        cp[k].resize(d.r[k] + 1);
        ri[k].resize(nnz);
        vv[k].resize(nnz);
        if (fread(cp[k].data(), 4, cp[k].size(), f) != cp[k].size() ||
            fread(ri[k].data(), 4, nnz, f) != (size_t)nnz || fread(vv[k].data(), 8, nnz, f) != (size_t)nnz ||
            cp[k][d.r[k]] != nnz) {
            set_error("%s: truncated coefficients", path);
            return FST_EFORMAT;
        }
        d.colptr[k] = cp[k].data();
        d.rowidx[k] = ri[k].data();
        d.val[k] = vv[k].data();
    }
    std::vector<double> al((size_t)d.r[0] * d.r[1] * d.r[2]);
    if (fread(al.data(), 8, al.size(), f) != al.size()) {
        set_error("%s: truncated core", path);
        return FST_EFORMAT;
    }
    d.alpha = al.data();
    fst_wavelet_desc w;
    memset(&w, 0, sizeof w);
    std::vector<uint8_t> cw[3];
    bool has_wav = false;
    if (ver >= 2) {
        int32_t wv[2];
        if (fread(wv, 4, 2, f) != 2) {
            set_error("%s: truncated wavelet section", path);
            return FST_EFORMAT;
        }
        if (wv[0] >= 0) {
            has_wav = true;
            w.level = wv[0];
            w.degree = wv[1];
            for (int k = 0; k < 3; ++k) {
                cw[k].resize(d.r[k]);
                if (fread(cw[k].data(), 1, d.r[k], f) != (size_t)d.r[k]) {
                    set_error("%s: truncated wavelet flags", path);
                    return FST_EFORMAT;
                }
                w.col_wavelet[k] = cw[k].data();
            }
        }
    }
    fst_status st = has_wav ? fst_model_create_wavelet(&d, &w, out) : fst_model_create(&d, out);
    if (st == FST_EINVAL) st = FST_EFORMAT;
    return st;
}

// ------------------------------------------------------------------ status strings
extern "C" const char* fst_status_str(fst_status s) {
    switch (s) {
        case FST_OK: return "ok";
        case FST_EINVAL: return "invalid argument";
        case FST_ENOMEM: return "out of memory";
        case FST_ECUDA: return "CUDA error";
        case FST_ENOTSPD: return "normal matrix not positive definite";
        case FST_ERANK: return "fewer sampled rows than unknowns";
        case FST_ETIMEOUT: return "device wait timed out";
        case FST_EFORMAT: return "malformed model file";
        case FST_ENOTCONV: return "refinement did not converge";
        case FST_EUNSUPPORTED: return "unsupported precision or shape";
    }
    return "unknown status";
}

extern "C" const char* fst_last_error(void) { return g_last_error.c_str(); }

extern "C" uint64_t fst_kernel_launches(void) { return g_launches.load(); }

extern "C" const char* fst_build_info(void) {
    return "libfst 0.1 (sm_103a; CUDA " FST_STR(__CUDACC_VER_MAJOR__) "." FST_STR(__CUDACC_VER_MINOR__) ")";
}
