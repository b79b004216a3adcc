// The small-label draw (3 <= L <= 16, Section 5.2, Eq.
// posterior_pca_transition_matrix): prior sums of all labels from a table of
// neighbour pairs, weights two labels per packed FP32x2 instruction, inverse
// CDF over chunks of 4 labels with the per-site certified margin.  Shared by
// the small-label sweep (small.cu) and the TMA-tiled k-sweep kernel (tb.cu).
#pragma once

#include "pcad_internal.h"

namespace pcad {
namespace sld {

constexpr int kCodes = 17;                       // labels 0..15 and "missing"
constexpr int kPtabWords = kCodes * kCodes * 4;  // 16 bytes per pair
constexpr int kPrefixStride = 20;                // floats per thread row (conflict-free)
constexpr int kAqStride = 20;                    // floats per row of the data-term table

// Row g of the data-term table: fl(alpha (g - s)^2) for s = 0..15 (observations
// g < 16; every chain checks g < L at creation).
__device__ __forceinline__ void fill_aq(const DevModel &m, float *aq, int tid, int nthreads)
{
    for (int i = tid; i < 16 * 16; i += nthreads) {
        const int g = i >> 4, sl = i & 15;
        aq[g * kAqStride + sl] = __fmul_rn(m.alpha, (float)((g - sl) * (g - sl)));
    }
}

// The draw of one site from its neighbour codes nc[] and observation g.
// Returns the label; `certain` is false when the uniform lies within the
// certified margin of the chosen label's CDF interval (the caller re-draws
// it in FP64).  pt: the pair table in shared memory; pre: this thread's row
// of shared memory (kPrefixStride floats), which receives the weights.  AQ:
// the data term from the table aq (fill_aq; g < 16), the exponent
// fl(gam P + fl(alpha q)) in one FFMA per label; otherwise
// fl(alpha q + fl(gam P)).  Both terms are non-positive, so either form is
// within 3u |v| of the exact exponent, the per-site margin's bound.
template <int LMAX, int NB, bool MASK, bool AQ = false>
__device__ __forceinline__ int draw_small(const DevModel &m, const uint32_t *pt, const int (&nc)[NB],
                                          int g, int xi, uint32_t ub, float *pre, bool &certain,
                                          const float *aq = nullptr)
{
    constexpr int NW = LMAX / 4;      // table words used per pair = chunks of 4 labels
    uint32_t P[NW];
    {
        const int e0 = (nc[0] * kCodes + nc[1]) * 4;
        const int e1 = (nc[2] * kCodes + nc[3]) * 4;
        if constexpr (NW == 4) {
            uint4 a = *reinterpret_cast<const uint4 *>(pt + e0);
            const uint4 b = *reinterpret_cast<const uint4 *>(pt + e1);
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
            if constexpr (NB == 8) {
                const uint4 c = *reinterpret_cast<const uint4 *>(pt + (nc[4] * kCodes + nc[5]) * 4);
                const uint4 d = *reinterpret_cast<const uint4 *>(pt + (nc[6] * kCodes + nc[7]) * 4);
                a.x += c.x + d.x;
                a.y += c.y + d.y;
                a.z += c.z + d.z;
                a.w += c.w + d.w;
            }
            P[0] = a.x;
            P[1] = a.y;
            P[2] = a.z;
            P[3] = a.w;
        } else {
            uint2 a = *reinterpret_cast<const uint2 *>(pt + e0);
            const uint2 b = *reinterpret_cast<const uint2 *>(pt + e1);
            a.x += b.x;
            a.y += b.y;
            if constexpr (NB == 8) {
                const uint2 c = *reinterpret_cast<const uint2 *>(pt + (nc[4] * kCodes + nc[5]) * 4);
                const uint2 d = *reinterpret_cast<const uint2 *>(pt + (nc[6] * kCodes + nc[7]) * 4);
                a.x += c.x + d.x;
                a.y += c.y + d.y;
            }
            P[0] = a.x;
            P[1] = a.y;
        }
    }
    const float gf = (float)g;
    const float2 a2 = make_float2(m.alpha, m.alpha), g2 = make_float2(m.gam, m.gam);
    const float2 off2 = make_float2(-8388608.0f, -8388608.0f);
    const float2 gg = make_float2(gf, gf);
    float w[LMAX];
    float4 aq4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int s = 0; s < LMAX; s += 2) {
        const uint32_t p = P[s >> 2];
        const float2 pm = make_float2(
            __uint_as_float(__byte_perm(p, 0x4B000000u, 0x7440u | (uint32_t)(s & 3))),
            __uint_as_float(__byte_perm(p, 0x4B000000u, 0x7440u | (uint32_t)((s + 1) & 3))));
        const float2 Pf = __fadd2_rn(pm, off2);
        float2 v;
        if constexpr (AQ) {
            if ((s & 3) == 0)
                aq4 = *reinterpret_cast<const float4 *>(aq + g * kAqStride + s);
            v = __ffma2_rn(g2, Pf, (s & 3) == 0 ? make_float2(aq4.x, aq4.y)
                                                : make_float2(aq4.z, aq4.w));
        } else {
            const float2 dg = __fadd2_rn(gg, make_float2(-(float)s, -(float)(s + 1)));
            v = __ffma2_rn(a2, __fmul2_rn(dg, dg), __fmul2_rn(g2, Pf));
        }
        w[s] = ex2_ftz(v.x);
        w[s + 1] = ex2_ftz(v.y);
        if (MASK) {
            w[s] = s < m.L ? w[s] : 0.0f;
            w[s + 1] = s + 1 < m.L ? w[s + 1] : 0.0f;
        }
    }
    // the weights (to shared memory) and the chunk prefix G over the in-chunk
    // sums ((w0 + w1) + w2) + w3
    float G[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        const float p3 = __fadd_rn(__fadd_rn(__fadd_rn(w[4 * c], w[4 * c + 1]), w[4 * c + 2]),
                                   w[4 * c + 3]);
        reinterpret_cast<float4 *>(pre)[c] =
            make_float4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
        G[c] = c == 0 ? p3 : __fadd_rn(G[c - 1], p3);
    }
    // inertia correction from w(x_i) as evaluated above
    const float delta = m.em1 != 0.0f ? __fmul_rn(pre[xi], m.em1) : 0.0f;
    const float G0 = G[NW - 1];
    const float Z = __fadd_rn(G0, delta);
    const float t = __fmul_rn((float)ub * (1.0f / 16777216.0f), Z);
    const float margin = __fmul_rn(site_margin(m, G0, delta), Z);
    // chunk: the number of chunk ends <= t, compared with t - delta where
    // delta is added (at and above x_i); Gp: the chunk prefix before it.  Any
    // rounding here only selects which label's interval is certified below:
    // a chunk chosen off by one leaves t within a few u Z of that interval's
    // end, inside the margin, and goes to FP64.
    const float tmd = __fsub_rn(t, delta);
    int cs = 0;
    float Gp = 0.0f;
#pragma unroll
    for (int c = 0; c + 1 < NW; ++c) {
        const bool below = G[c] <= ((4 * c + 3 >= xi) ? tmd : t);
        cs += below ? 1 : 0;
        Gp = below ? G[c] : Gp;
    }
    // the chosen chunk's in-chunk prefix sums, as summed for G; C_k joins
    // them to Gp or to Gp + delta (two roundings either way)
    const float4 wc = reinterpret_cast<const float4 *>(pre)[cs];
    const float p1 = __fadd_rn(wc.x, wc.y), p2 = __fadd_rn(p1, wc.z), p3 = __fadd_rn(p2, wc.w);
    const int base = 4 * cs;
    const float Gpd = __fadd_rn(Gp, delta);
    const float C0 = __fadd_rn((base >= xi) ? Gpd : Gp, wc.x);
    const float C1 = __fadd_rn((base + 1 >= xi) ? Gpd : Gp, p1);
    const float C2 = __fadd_rn((base + 2 >= xi) ? Gpd : Gp, p2);
    const float C3 = __fadd_rn((base + 3 >= xi) ? Gpd : Gp, p3);
    const bool b0 = C0 <= t, b1 = C1 <= t, b2 = C2 <= t;
    const int k = (int)b0 + (int)b1 + (int)b2;
    const float hiC = b2 ? C3 : (b1 ? C2 : (b0 ? C1 : C0));
    const float Cm = (base - 1 >= xi) ? Gpd : Gp;   // before the chunk
    const float loC = b2 ? C2 : (b1 ? C1 : (b0 ? C0 : Cm));
    const int s = base + k;
    certain = (t < hiC) & (s < m.L) & ((s == m.L - 1) | (__fsub_rn(hiC, t) > margin)) &
              ((s == 0) | (__fsub_rn(t, loC) > margin));
    return min(s, m.L - 1);
}

}  // namespace sld
}  // namespace pcad
