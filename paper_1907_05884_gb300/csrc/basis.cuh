// basis.cuh -- device code shared by the evaluation and refit kernels: the factor values
// of Sec. 2, eq. sparse, for columns in the orthonormal Legendre space P_p,
//   w^(k)_j(y) = sum_n W^k_{n,j} sqrt(2n+1) L_n(t),  t = 2 (y - lo)/(hi - lo) - 1,
// with L_n from the three-term recurrence (n+1) L_{n+1} = (2n+1) t L_n - n L_{n-1}, and for
// columns in a multiwavelet space W_{s,q} (Sec. 4.2, Fig. 3): such a column is a polynomial
// of degree <= q on each of the 2^s equal cells of the box, stored (exactly converted from
// its multiwavelet coefficients) as sqrt(2n+1) L_n of the cell's local coordinate.
#pragma once

#include "fst_internal.cuh"

namespace fst {

template <typename T>
struct EvalArgs {
    int r[3];
    int pe[3];
    int pm;         // max pe rounded up to a multiple of 4
    T sc[3], of[3]; // t = y * sc + of maps the box onto [-1,1]
    const T* W[3];
    const uint8_t* mask[3];
    const T* alpha;
    // wavelet columns: per mode, 2^s cells (0: none) of nq = q + 1 local Legendre rows each,
    // Wp[k][(f nq + n) r_k + j] with sqrt(2n+1) folded in; the box decides the cells
    const T* Wp[3];
    int wcells[3];
    int wq;
    double wlo[3], whi[3];
};

// Finest cell of coordinate y: the number of interior boundaries lo + ((hi - lo) c) 2^-s,
// c = 1 .. cells - 1, at or below y, compared exactly in FP64 (every implementation that
// compares the same values agrees on the cell).
__device__ __forceinline__ int wavelet_cell(double y, double lo, double hi, int cells) {
    const double span = __dadd_rn(hi, -lo), inv = 1.0 / (double)cells;   // inv: a power of two
    int f = 0;
    for (int c = 1; c < cells; ++c) f += y >= __dadd_rn(lo, __dmul_rn(__dmul_rn(span, (double)c), inv)) ? 1 : 0;
    return f;
}

// Adds the wavelet columns' values of mode k to acc: the point's cell f, its local
// coordinate tau = cells (t + 1) - 2f - 1, and sum_n Wp[f][n][j] L_n(tau).
template <typename T, int RM, int PPT>
__device__ __forceinline__ void piecewise_values(const T (&y)[PPT], const T (&t)[PPT], const EvalArgs<T>& a,
                                                 int k, T (&acc)[PPT][RM]) {
    const int cells = a.wcells[k];
    if (cells == 0) return;
    const int nq = a.wq, rk = a.r[k];
#pragma unroll
    for (int pp = 0; pp < PPT; ++pp) {
        const int f = wavelet_cell((double)y[pp], a.wlo[k], a.whi[k], cells);
        const T tau = (T)cells * (t[pp] + T(1)) - (T)(2 * f + 1);
        const T* w = a.Wp[k] + (size_t)f * nq * rk;
        T Lm = T(1), L = tau;
        for (int n = 0; n < nq; ++n) {
            T Ln;
            if (n == 0) {
                Ln = T(1);
            } else if (n == 1) {
                Ln = tau;
            } else {
                Ln = (T(2 * n - 1) * tau * L - T(n - 1) * Lm) / T(n);
                Lm = L;
                L = Ln;
            }
            const T* wr = w + (size_t)n * rk;
#pragma unroll
            for (int j = 0; j < RM; ++j)
                if (j < rk) acc[pp][j] = fma(wr[j], Ln, acc[pp][j]);
        }
    }
}

__device__ __forceinline__ void load4(const float* p, float& a, float& b, float& c, float& d) {
    float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double* p, double& a, double& b, double& c, double& d) {
    double2 v0 = *reinterpret_cast<const double2*>(p);
    double2 v1 = *reinterpret_cast<const double2*>(p + 2);
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}

// Factor values of one mode for PPT points: acc[pp][j] = sum_n Ws[n][j] L_n(t[pp]).
template <typename T, int RM, int PPT>
__device__ __forceinline__ void factor_values(const T (&t)[PPT], const T* Ws, const uint8_t* mk, int pe,
                                              const T* ra, const T* rb, T (&acc)[PPT][RM]) {
#pragma unroll
    for (int j = 0; j < RM; j += 4) {
        T w0, w1, w2, w3;
        load4(Ws + j, w0, w1, w2, w3);
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
            acc[pp][j] = w0; acc[pp][j + 1] = w1; acc[pp][j + 2] = w2; acc[pp][j + 3] = w3;
        }
    }
    if (pe <= 1) return;
    T Lm[PPT], L[PPT];
#pragma unroll
    for (int pp = 0; pp < PPT; ++pp) { Lm[pp] = T(1); L[pp] = t[pp]; }
    for (int nn = 1; nn < pe; ++nn) {
        if (nn >= 2) {
            // (n+1) L_{n+1} = (2n+1) t L_n - n L_{n-1} with n = nn-1
            const T a = ra[nn - 1], b = rb[nn - 1];
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) {
                T Ln = a * t[pp] * L[pp] - b * Lm[pp];
                Lm[pp] = L[pp];
                L[pp] = Ln;
            }
        }
        if (mk[nn]) {
            const T* w = Ws + nn * RM;
#pragma unroll
            for (int j = 0; j < RM; j += 4) {
                T w0, w1, w2, w3;
                load4(w + j, w0, w1, w2, w3);
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    acc[pp][j] = fma(w0, L[pp], acc[pp][j]);
                    acc[pp][j + 1] = fma(w1, L[pp], acc[pp][j + 1]);
                    acc[pp][j + 2] = fma(w2, L[pp], acc[pp][j + 2]);
                    acc[pp][j + 3] = fma(w3, L[pp], acc[pp][j + 3]);
                }
            }
        }
    }
}


template <typename T>
inline EvalArgs<T> make_args(const fst_model* m) {
    EvalArgs<T> a;
    int pm = 1;
    for (int k = 0; k < 3; ++k) {
        a.r[k] = m->r[k];
        a.pe[k] = m->p_eff[k];
        pm = m->p_eff[k] > pm ? m->p_eff[k] : pm;
        a.sc[k] = (T)(2.0 / (m->hi[k] - m->lo[k]));
        a.of[k] = (T)(-(m->hi[k] + m->lo[k]) / (m->hi[k] - m->lo[k]));
        a.mask[k] = m->rowmask[k];
        a.wcells[k] = m->wav_s >= 0 && m->wav_cols[k] > 0 ? 1 << m->wav_s : 0;
        a.wlo[k] = m->lo[k];
        a.whi[k] = m->hi[k];
        a.Wp[k] = nullptr;
    }
    a.wq = m->wav_s >= 0 ? m->wav_q + 1 : 0;
    a.pm = (pm + 3) & ~3;
    return a;
}

inline void bind(EvalArgs<double>& a, const fst_model* m) {
    for (int k = 0; k < 3; ++k) {
        a.W[k] = m->W64[k];
        a.Wp[k] = m->Wp64[k];
    }
    a.alpha = m->alpha64;
}
inline void bind(EvalArgs<float>& a, const fst_model* m) {
    for (int k = 0; k < 3; ++k) {
        a.W[k] = m->W32[k];
        a.Wp[k] = m->Wp32[k];
    }
    a.alpha = m->alpha32;
}

}  // namespace fst
