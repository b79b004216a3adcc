// Device-side building blocks of the lazy-PCA / Gibbs sweep kernels.
//
// Per-site conditional (Section 5.2, Eq. posterior_pca_transition_matrix;
// Section 5.1, Eq. gibbs_sampler_elementary_step):
//   p_i(s) ~ exp(-E_i(s)),  E_i(s) = sum_j V(s, x_j) + U(g_i, s) + lambda 1{s != x_i}.
//
// GPU formulation (same distribution, different algebra):
//   * Potts V(s,t) = -c 1{s=t} equals c min(|s-t|, 1) up to a constant, so
//     both priors are evaluated as c * P(s), P(s) = sum_j min(|s - x_j|, T)
//     with T = 1 for Potts.  A neighbour outside the image is replaced by
//     label 1024, whose term min(|s - 1024|, T) = T is the same for every s
//     and cancels in the normalisation (free boundary).
//   * Weight w(s) = A(g - s) * 2^(gam * P(s)), gam = -c log2(e), with the
//     data factor A(d) = exp(-(U(g, g - d) - U(g, g))) from a 511-entry table
//     (|A| <= 1 for Gaussian noise).  The inertia multiplies the weight of
//     the single label s = x_i by e^lambda (all others are relatively
//     penalised by e^-lambda): it is applied as one correction
//     delta = w(x_i) (e^lambda - 1) to the CDF at and above x_i.
//   * Parameter limits keep every weight in [e^-80, e^40]: no overflow and
//     no subnormal weight among those that matter.
//   * Inverse-CDF draw: new label = smallest k with u Z < C_k.  The FP32
//     evaluation has a rigorous error bound eta (relative to Z); when the
//     uniform lies within eta of the chosen CDF interval's ends the draw is
//     re-evaluated in FP64 (table products, FP64 sums in label order) and
//     counted.  This makes the FP32 path decide exactly what the FP64
//     definition decides.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcad {

constexpr int kChunk = 8;                 // labels per chunk of the 2-pass CDF
constexpr float kMissingLabel = 1024.0f;  // stand-in for a neighbour outside the image
constexpr int kMissingLabelI = 1024;
constexpr uint32_t kTagPCA = 0u;
constexpr uint32_t kTagGibbs = 1u;
constexpr int kTableOffset = 255;         // data table index = g - s + 255

// Per-model constants consumed by the kernels (built on the host).
struct DevModel {
    int L;             // labels
    int nbhd;          // 4 or 8
    int T;             // truncation (1 for Potts)
    int pmax;          // nbhd * T: largest P(s)
    float gam;         // -c * log2(e)
    float Tf;          // (float)T
    float em1;         // e^lambda - 1 (0: no inertia)
    float eta;         // FP32 error bound of the normalised CDF
    const float *ta32;   // [511] data factor, FP32
    const double *ta64;  // [511] data factor, FP64
    const double *pr64;  // [pmax + 1] exp(-c P), FP64
    double el64;         // e^lambda, FP64
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds of two 32x32->64-bit
// multiplications (multipliers 0xD2511F53, 0xCD9E8D57) with a Weyl key
// schedule (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t &o0,
                                              uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    o0 = c0;
    o1 = c1;
    o2 = c2;
    o3 = c3;
}

// 24-bit uniform numerator of site (row, col) at sweep `sweep`.
__device__ __forceinline__ uint32_t site_u24(uint64_t seed, uint32_t chain, uint32_t tag,
                                             uint32_t sweep, uint32_t row, uint32_t col)
{
    uint32_t o0, o1, o2, o3;
    philox4x32_10(col >> 2, row, sweep, (tag << 24) | (chain & 0xFFFFFFu),
                  (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), o0, o1, o2, o3);
    const uint32_t j = col & 3u;
    const uint32_t w = j == 0 ? o0 : (j == 1 ? o1 : (j == 2 ? o2 : o3));
    return w >> 8;
}

// ------------------------------------------------------- FP32 chunk weights

// Sum of the weights of labels [8c, 8c+8) (labels >= L masked when MASK).
template <int NB, bool MASK>
__device__ __forceinline__ float chunk_sum(const DevModel &m, const float *__restrict__ ta_s,
                                           int g, const float (&xn)[NB], int c)
{
    const float sb = (float)(c * kChunk);
    float xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = xn[j] - sb;
    const float *tap = ta_s + (g - c * kChunk + kTableOffset);
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        float P = fminf(fabsf(xr[0] - (float)k), m.Tf);
#pragma unroll
        for (int j = 1; j < NB; ++j)
            P += fminf(fabsf(xr[j] - (float)k), m.Tf);
        const float e = exp2f(m.gam * P);
        float a = tap[-k];
        if (MASK && (c * kChunk + k >= m.L))
            a = 0.0f;
        S = __fmaf_rn(a, e, S);
    }
    return S;
}

// Inclusive running sums p_k of the weights of chunk c.
template <int NB>
__device__ __forceinline__ void chunk_prefix(const DevModel &m, const float *__restrict__ ta_s,
                                             int g, const float (&xn)[NB], int c,
                                             float (&p)[kChunk])
{
    const float sb = (float)(c * kChunk);
    float xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = xn[j] - sb;
    const float *tap = ta_s + (g - c * kChunk + kTableOffset);
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        float P = fminf(fabsf(xr[0] - (float)k), m.Tf);
#pragma unroll
        for (int j = 1; j < NB; ++j)
            P += fminf(fabsf(xr[j] - (float)k), m.Tf);
        const float e = exp2f(m.gam * P);
        float a = tap[-k];
        if (c * kChunk + k >= m.L)
            a = 0.0f;
        S = __fmaf_rn(a, e, S);
        p[k] = S;
    }
}

template <int NB>
__device__ __forceinline__ float label_weight(const DevModel &m, const float *__restrict__ ta_s,
                                              int g, const float (&xn)[NB], int s)
{
    const float sf = (float)s;
    float P = fminf(fabsf(xn[0] - sf), m.Tf);
#pragma unroll
    for (int j = 1; j < NB; ++j)
        P += fminf(fabsf(xn[j] - sf), m.Tf);
    return ta_s[g - s + kTableOffset] * exp2f(m.gam * P);
}

// FP32 inverse-CDF draw.  Gcol points at this thread's column of a shared
// scratch array (stride gstride floats) holding the chunk prefix sums.
// Returns the label; `certain` is false when the uniform lies within the
// error bound of a boundary of the chosen label's CDF interval.
template <int NC, int NB>
__device__ __forceinline__ int draw_fp32(const DevModel &m, const float *__restrict__ ta_s,
                                         float *Gcol, int gstride, int g, int xi,
                                         const float (&xn)[NB], float u, bool &certain)
{
    // pass 1: chunk prefix sums of the inertia-free weights
    float G = 0.0f;
    const int nfull = m.L / kChunk;  // chunks with no label >= L
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        const float S = (c < nfull) ? chunk_sum<NB, false>(m, ta_s, g, xn, c)
                                    : chunk_sum<NB, true>(m, ta_s, g, xn, c);
        G += S;
        Gcol[c * gstride] = G;
    }
    float delta = 0.0f;
    if (m.em1 != 0.0f)
        delta = label_weight<NB>(m, ta_s, g, xn, xi) * m.em1;
    const float Z = G + delta;
    const float t = u * Z;
    // smallest chunk whose (inertia-corrected) prefix exceeds t
    int lo = 0, hi = NC - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float gm = Gcol[mid * gstride] + ((xi <= mid * kChunk + kChunk - 1) ? delta : 0.0f);
        if (t < gm)
            hi = mid;
        else
            lo = mid + 1;
    }
    const int cs = lo;
    const float Gprev = cs > 0 ? Gcol[(cs - 1) * gstride] : 0.0f;
    float p[kChunk];
    chunk_prefix<NB>(m, ta_s, g, xn, cs, p);
    const int base = cs * kChunk;
    const int kmax = min(kChunk - 1, m.L - 1 - base);
    int k = kmax;
    float hiC = 0.0f;
#pragma unroll
    for (int kk = kChunk - 1; kk >= 0; --kk) {
        const float Ck = (Gprev + p[kk]) + ((base + kk >= xi) ? delta : 0.0f);
        if (kk <= kmax && t < Ck) {
            k = kk;
            hiC = Ck;
        }
    }
    if (k == kmax && !(t < hiC))
        hiC = (Gprev + p[kmax]) + ((base + kmax >= xi) ? delta : 0.0f);
    float loC;
    if (k > 0)
        loC = (Gprev + p[k - 1]) + ((base + k - 1 >= xi) ? delta : 0.0f);
    else
        loC = Gprev + ((base - 1 >= xi) ? delta : 0.0f);
    const int s = base + k;
    const float margin = m.eta * Z;
    const bool ok_hi = (s == m.L - 1) || (hiC - t > margin);
    const bool ok_lo = (s == 0) || (t - loC > margin);
    certain = ok_hi && ok_lo;
    return s;
}

// ------------------------------------------------------------ FP64 re-draw

template <int NB>
__device__ __forceinline__ double weight64(const DevModel &m, int g, int xi, const int (&xni)[NB],
                                           int s)
{
    int P = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int d = abs(s - xni[j]);
        P += d < m.T ? d : m.T;
    }
    double w = __dmul_rn(m.ta64[g - s + kTableOffset], m.pr64[P]);
    if (m.em1 != 0.0f && s == xi)
        w = __dmul_rn(w, m.el64);
    return w;
}

// FP64 evaluation of the same draw: weights in FP64, sums in label order.
template <int NB>
__device__ __noinline__ int draw_fp64(const DevModel &m, int g, int xi, const int (&xni)[NB],
                                      double u)
{
    double Z = 0.0;
    for (int s = 0; s < m.L; ++s)
        Z = __dadd_rn(Z, weight64<NB>(m, g, xi, xni, s));
    const double t = __dmul_rn(u, Z);
    double C = 0.0;
    for (int s = 0; s < m.L; ++s) {
        C = __dadd_rn(C, weight64<NB>(m, g, xi, xni, s));
        if (t < C)
            return s;
    }
    return m.L - 1;
}

}  // namespace pcad
