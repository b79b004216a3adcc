// Weight arithmetic of the windowed lazy-PCA draw (Section 5.2, Eq.
// posterior_pca_transition_matrix) shared by the tensor-core sweep and the
// CUDA-core windowed sweep: weights from exact tent sums
// Pb(s) = sum_j max(T - |x_j - s|, 0), w(s) = 2^(alpha (g - s)^2 + mu Pb(s) + cb),
// the outside-chunk table (Pb = 0) and the exact prefix sums of one chunk.
#pragma once

#include <cuda_fp16.h>

#include "pcad_internal.h"

namespace pcad {
namespace tcm {

// Outside-chunk table of a model: the sum of chunk c for observation g is
// F(g - 8c), F(d) = sum_k 2^(alpha (d - k)^2), at [d + 255] (d in
// [-255, 255]); when L % 8 != 0 the last chunk's masked sums follow at
// [kTabLast + g].  768 floats (3 KB).
constexpr int kTabLast = 512;
constexpr int kTabF = 768;

// Weight of one label from its tent sum Pb (an exact integer):
// 2^(alpha dg^2 + mu Pb + cb).  The common offset cb = -mu nbhd T keeps both
// terms of the exponent non-positive (mu > 0), so its rounding error stays
// proportional to the exponent itself.
__device__ __forceinline__ float label_wb(const DevModel &m, float mu, float Pb, float dg)
{
    const float q = __fmul_rn(dg, dg);
    const float v = __fmaf_rn(m.alpha, q, __fmaf_rn(mu, Pb, m.cb));
    return ex2_ftz(v);
}

// Exact tent sum of label s over the neighbours (missing ones, label 1024,
// and unused outlier slots contribute zero).
template <int N>
__device__ __forceinline__ float tent_sum(const float (&x)[N], float Tf, float s, int n = N)
{
    float P = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j < n)
            P = __fadd_rn(P, fmaxf(__fsub_rn(Tf, fabsf(__fsub_rn(s, x[j]))), 0.0f));
    return P;
}

// Sum of the weights of absolute chunk c (labels 8c .. 8c + 7) outside the
// window, where no in-window neighbour's tent reaches: 2^(alpha (g - s)^2 +
// cb), label_wb at Pb = 0.  LMASK zeroes labels >= L.
template <bool LMASK>
__device__ __forceinline__ float outside_chunk(const DevModel &m, float gf, int c)
{
    const float dgb = __fsub_rn(gf, (float)(c * kChunk));
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        const float dg = __fsub_rn(dgb, (float)k);
        float w = ex2_ftz(__fmaf_rn(m.alpha, __fmul_rn(dg, dg), m.cb));
        if (LMASK && c * kChunk + k >= m.L)
            w = 0.0f;
        S = __fadd_rn(S, w);
    }
    return S;
}

// Entry i of the outside-chunk table (the same operations as outside_chunk,
// hence the same values).
template <bool LMASK>
__device__ __forceinline__ float tab_entry(const DevModel &m, int i)
{
    if (i < 2 * 255 + 1)
        return outside_chunk<false>(m, (float)(i - 255), 0);
    if (LMASK && i >= kTabLast && i < kTabLast + 256)
        return outside_chunk<true>(m, (float)(i - kTabLast), (m.L - 1) / kChunk);
    return 0.0f;
}

// Outside sum of chunk c (of nc) for observation g.
template <bool LMASK>
__device__ __forceinline__ float tab_sum(const float *tab, int g, int c, int nc)
{
    if (LMASK && c == nc - 1)
        return tab[kTabLast + g];
    return tab[g - kChunk * c + 255];
}

// Sum of the weights of window chunk c from 8 tent sums read from TMEM (pb,
// raw FP32 bits).  Two labels per packed FP32x2 instruction (each lane of a
// pair rounds as the scalar operation: the weights equal label_wb's); the
// chunk sum is a pairwise tree (3 roundings per weight).
template <bool LMASK>
__device__ __forceinline__ float window_chunk(const DevModel &m, float mu, float gf,
                                              const uint32_t *pb, int c)
{
    const float dgb = __fsub_rn(gf, (float)(c * kChunk));
    const float2 a2 = make_float2(m.alpha, m.alpha), mu2 = make_float2(mu, mu),
                 cb2 = make_float2(m.cb, m.cb);
    const float2 dgb2 = make_float2(dgb, __fsub_rn(dgb, 1.0f));
    float2 wv[4];
#pragma unroll
    for (int k = 0; k < kChunk; k += 2) {
        const float2 dg = __fadd2_rn(dgb2, make_float2(-(float)k, -(float)k));
        const float2 qq = __fmul2_rn(dg, dg);
        const float2 pb2 = make_float2(__uint_as_float(pb[k]), __uint_as_float(pb[k + 1]));
        const float2 in2 = __ffma2_rn(mu2, pb2, cb2);
        const float2 v = __ffma2_rn(a2, qq, in2);
        float w0 = ex2_ftz(v.x), w1 = ex2_ftz(v.y);
        if (LMASK && c * kChunk + k >= m.L)
            w0 = 0.0f;
        if (LMASK && c * kChunk + k + 1 >= m.L)
            w1 = 0.0f;
        wv[k >> 1] = make_float2(w0, w1);
    }
    const float2 a = __fadd2_rn(make_float2(wv[0].x, wv[2].x), make_float2(wv[0].y, wv[2].y));
    const float2 b = __fadd2_rn(make_float2(wv[1].x, wv[3].x), make_float2(wv[1].y, wv[3].y));
    const float2 t2 = __fadd2_rn(a, b);
    return __fadd_rn(t2.x, t2.y);
}

// Inclusive prefix sums of absolute chunk c's weights from exact tent sums
// (neighbour labels xn, observation gf) on the CUDA cores: bit-identical to
// the pass-1 weights.  The tents of two labels at once in half2 (integers up
// to 2048 are exact: neighbour labels, 1024 for a missing one, less 8c), the
// weights as window_chunk's.
template <int NB>
__device__ __forceinline__ void chunk_prefix_exact(const DevModel &m, float mu,
                                                   const float (&xn)[NB], float gf, int c,
                                                   float (&p)[kChunk])
{
    const float sb = (float)(c * kChunk);
    const __half2 T2 = __float2half2_rn(m.Tf), z2 = __float2half2_rn(0.0f);
    __half2 xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = __float2half2_rn(__fsub_rn(xn[j], sb));
    const float dgb = __fsub_rn(gf, sb);
    const float2 a2 = make_float2(m.alpha, m.alpha), mu2 = make_float2(mu, mu),
                 cb2 = make_float2(m.cb, m.cb);
    const float2 dgb2 = make_float2(dgb, __fsub_rn(dgb, 1.0f));
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; k += 2) {
        const __half2 k2 = __floats2half2_rn((float)k, (float)(k + 1));
        __half2 P2 = z2;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            P2 = __hadd2(P2, __hmax2(__hsub2(T2, __habs2(__hsub2(k2, xr[j]))), z2));
        const float2 dg = __fadd2_rn(dgb2, make_float2(-(float)k, -(float)k));
        const float2 qq = __fmul2_rn(dg, dg);
        const float2 in2 = __ffma2_rn(mu2, __half22float2(P2), cb2);
        const float2 v = __ffma2_rn(a2, qq, in2);
        float w0 = ex2_ftz(v.x), w1 = ex2_ftz(v.y);
        if (c * kChunk + k >= m.L)
            w0 = 0.0f;
        if (c * kChunk + k + 1 >= m.L)
            w1 = 0.0f;
        S = __fadd_rn(S, w0);
        p[k] = S;
        S = __fadd_rn(S, w1);
        p[k + 1] = S;
    }
}


}  // namespace tcm
}  // namespace pcad
