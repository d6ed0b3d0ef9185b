// basis.cuh -- device code shared by the evaluation and refit kernels: the
// orthonormal Legendre factor values of Sec. 2, eq. sparse,
//   w^(k)_j(y) = sum_n W^k_{n,j} sqrt(2n+1) L_n(t),  t = 2 (y - lo)/(hi - lo) - 1,
// with L_n from the three-term recurrence (n+1) L_{n+1} = (2n+1) t L_n - n L_{n-1}.
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
};

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
    }
    a.pm = (pm + 3) & ~3;
    return a;
}

inline void bind(EvalArgs<double>& a, const fst_model* m) {
    for (int k = 0; k < 3; ++k) a.W[k] = m->W64[k];
    a.alpha = m->alpha64;
}
inline void bind(EvalArgs<float>& a, const fst_model* m) {
    for (int k = 0; k < 3; ++k) a.W[k] = m->W32[k];
    a.alpha = m->alpha32;
}

}  // namespace fst
