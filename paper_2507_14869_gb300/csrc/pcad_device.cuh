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
#include <cuda_fp16.h>
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
    float gam;         // prior exponent coefficient, -c log2(e)
    float alpha;       // data exponent coefficient: -log2(e)/(2 sigma^2) (Gaussian) or
                       // -log2(e) ln((1-p)/p) (flip, with Q = (g-s)^2 in {0,1})
    float Tf;          // (float)T
    float em1;         // e^lambda - 1 (0: no inertia)
    float eta;         // FP32 error bound of the normalised CDF
    float cb;          // tensor-core sweep: common exponent offset (-mu nbhd T, mu > 0)
    float hb, kb0, kb1, kbr;   // its per-site margin kb1 (hb - log2 Z) + kb0 + kbr delta / Z
    int norm;          // inertia price: 0 L0 (via em1 / el64), 1 or 2 Lp (via kappa / in64)
    float kappa;       // Lp price exponent coefficient, -lambda log2(e) / (L - 1)^p
    const double *ta64;  // [511] data factor exp(-(U(g, g-d) - U(g,g))) at d + 255, FP64
    const double *pr64;  // [pmax + 1] exp(-c P), FP64
    const double *in64;  // [256] Lp price factor exp(-lambda (d / (L - 1))^p), FP64
    double el64;         // e^lambda, FP64
    const uint32_t *ptab;  // small-L sweep: pair prior table (nullptr: not built)
    const uint4 *btab;     // two-label draw thresholds per site configuration (nullptr: not built)
};

// ------------------------------------------------------------ bounded waits
// Every device-side wait of the library (a wavefront dependency, a TMA tile
// load, an MMA completion) is bounded by elapsed time, read from the
// nanosecond %globaltimer, and gives up at once when the launch's error
// flag is already set.  One lost dependency therefore ends the whole
// launch within about one limit: the first wait that runs out sets the
// flag, every other wait and every later item sees it and stops.
constexpr long long kWaitLimitNs = 1000000000ll;   // default limit: 1 s

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The error flag, read past L1 (another SM may have set it).
__device__ __forceinline__ int ld_flag(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The limit a launch uses: its own (nanoseconds, > 0) or the default.
__device__ __forceinline__ long long wait_limit(long long ns)
{
    return ns > 0 ? ns : kWaitLimitNs;
}

// Wait until *d >= k (acquire loads); `seen` is an earlier observation of
// *d.  Returns false if the wait ran out of time or *err was set meanwhile.
__device__ __forceinline__ bool wait_ge(const unsigned int *d, unsigned int k, unsigned int seen,
                                        const int *err, long long limit_ns)
{
    if (seen >= k)
        return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned int i = 1;; ++i) {
        __nanosleep(64);
        if (ld_acquire_u32(d) >= k)
            return true;
        if ((i & 15u) == 0u &&
            (ld_flag(err) != 0 || (long long)(globaltimer_ns() - t0) > limit_ns))
            return false;
    }
}

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

__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_ftz(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Certified CDF margin of one site's draw from its own total Z = G + delta
// (the weights' exponents must be sums of non-positive terms, each label's
// exponent error within 3u |v|: the tensor-core weights, and the CUDA-core
// weights when gam <= 0):
// eta = kb1 (log2(L + 1) + slack - log2 Z) + kb0 + kbr delta / Z.
__device__ __forceinline__ float site_margin(const DevModel &m, float G, float delta)
{
    const float Z = __fadd_rn(G, delta);
    return __fmaf_rn(m.kb1, __fsub_rn(m.hb, lg2_ftz(Z)), m.kb0) + m.kbr * __fdividef(delta, Z);
}

// Weight 2^v of one label: v = alpha (g - s)^2 + gam P(s).  dg = g - s and
// P are exact small integers; (g - s)^2 <= 65025 is exact in FP32.
__device__ __forceinline__ float label_w(const DevModel &m, float P, float dg)
{
    const float q = __fmul_rn(dg, dg);
    const float v = __fmaf_rn(m.alpha, q, __fmul_rn(m.gam, P));
    return ex2_ftz(v);
}

// Prior sums P(s), s = sb + kk and sb + kk + 1, for two labels at once in
// half precision (all operands are integers <= 2048, so exact): each
// neighbour contributes min(|x_j - s|, T).
template <int NB>
__device__ __forceinline__ float2 prior_pair(const __half2 (&xr)[NB], __half2 k2, __half2 T2)
{
    __half2 P2 = __hmin2(__habs2(__hsub2(xr[0], k2)), T2);
#pragma unroll
    for (int j = 1; j < NB; ++j)
        P2 = __hadd2(P2, __hmin2(__habs2(__hsub2(xr[j], k2)), T2));
    return __half22float2(P2);
}

// Weights of labels [8c, 8c + 8); returns their sequential sum and, when
// PREFIX, the inclusive running sums p[k].  Labels >= L weigh 0 when MASK.
template <int NB, bool MASK, bool PREFIX>
__device__ __forceinline__ float chunk_weights(const DevModel &m, const __half2 (&xh)[NB],
                                               __half2 T2, float gf, int c,
                                               float (&p)[kChunk])
{
    const float sbf = (float)(c * kChunk);
    const __half2 sb2 = __float2half2_rn(sbf);
    __half2 xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = __hsub2(xh[j], sb2);
    const float dgb = gf - sbf;
    float S = 0.0f;
#pragma unroll
    for (int kk = 0; kk < kChunk; kk += 2) {
        const float2 P = prior_pair<NB>(xr, __floats2half2_rn((float)kk, (float)(kk + 1)), T2);
        float e0 = label_w(m, P.x, dgb - (float)kk);
        float e1 = label_w(m, P.y, dgb - (float)(kk + 1));
        if (MASK) {
            if (c * kChunk + kk >= m.L) e0 = 0.0f;
            if (c * kChunk + kk + 1 >= m.L) e1 = 0.0f;
        }
        S = __fadd_rn(S, e0);
        if (PREFIX) p[kk] = S;
        S = __fadd_rn(S, e1);
        if (PREFIX) p[kk + 1] = S;
    }
    return S;
}

// Chunks whose labels see a linear prior.  P(s+1) - P(s) changes only at
// s = x_j - T, x_j, x_j + T (the kinks of min(|s - x_j|, T)); a chunk
// [8c, 8c+7] is linear unless such a kink lies in [8c+1, 8c+6].  Returns a
// bit per chunk that holds a kink ("dirty").  Neighbours outside the image
// (label 1024) contribute a constant and no kink.
template <int NB>
__device__ __forceinline__ uint32_t dirty_chunks(const int (&xni)[NB], int T)
{
    uint32_t mask = 0u;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (xni[j] >= kMissingLabelI)
            continue;
#pragma unroll
        for (int o = -1; o <= 1; ++o) {
            const int e = xni[j] + o * T;
            const int r = e & 7;
            if (e > 0 && e < 256 && r != 0 && r != 7)
                mask |= 1u << (e >> 3);
        }
    }
    return mask;
}

// Chunk sum when P is linear on the chunk: P(8c + k) = P0 + k (P1 - P0),
// exact; every weight is then bit-identical to chunk_weights's.
template <int NB, bool MASK>
__device__ __forceinline__ float chunk_weights_linear(const DevModel &m, const __half2 (&xh)[NB],
                                                      __half2 T2, float gf, int c)
{
    const float sbf = (float)(c * kChunk);
    const __half2 sb2 = __float2half2_rn(sbf);
    __half2 xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = __hsub2(xh[j], sb2);
    const float2 P01 = prior_pair<NB>(xr, __floats2half2_rn(0.0f, 1.0f), T2);
    const float slope = __fsub_rn(P01.y, P01.x);
    const float dgb = gf - sbf;
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        const float P = k == 0 ? P01.x : (k == 1 ? P01.y : __fmaf_rn(slope, (float)k, P01.x));
        float e = label_w(m, P, dgb - (float)k);
        if (MASK && c * kChunk + k >= m.L)
            e = 0.0f;
        S = __fadd_rn(S, e);
    }
    return S;
}

// Weight of a single label s (used for the inertia correction).
template <int NB>
__device__ __forceinline__ float single_w(const DevModel &m, const float (&xn)[NB], float gf, int s)
{
    const float sf = (float)s;
    float P = fminf(fabsf(xn[0] - sf), m.Tf);
#pragma unroll
    for (int j = 1; j < NB; ++j)
        P = __fadd_rn(P, fminf(fabsf(xn[j] - sf), m.Tf));
    return label_w(m, P, gf - sf);
}

// Per-site inputs of a draw.
template <int NB>
struct SiteIn {
    int g, xi;
    int xni[NB];     // neighbour labels (missing: 1024)
    uint32_t ub;     // 24-bit uniform numerator
};

// Two-label draw (L = 2): the same weights and the same certified test as
// the chunked path, without the chunk machinery.  Label 0 iff u Z < w0.
template <int NB>
__device__ __forceinline__ int draw_binary(const DevModel &m, const SiteIn<NB> &in, bool &certain)
{
    float P0 = 0.0f, P1 = 0.0f;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const float xj = (float)in.xni[j];
        P0 = __fadd_rn(P0, fminf(fabsf(xj), m.Tf));
        P1 = __fadd_rn(P1, fminf(fabsf(xj - 1.0f), m.Tf));
    }
    const float gf = (float)in.g;
    float w0 = label_w(m, P0, gf);
    float w1 = label_w(m, P1, gf - 1.0f);
    float delta = 0.0f;
    if (m.em1 != 0.0f)
        delta = __fmul_rn(in.xi == 0 ? w0 : w1, m.em1);
    const float C0 = in.xi == 0 ? __fadd_rn(w0, delta) : w0;
    const float Z = __fadd_rn(__fadd_rn(w0, w1), delta);
    const float t = __fmul_rn((float)in.ub * (1.0f / 16777216.0f), Z);
    const float margin = __fmul_rn(m.eta, Z);
    const int s = t < C0 ? 0 : 1;
    certain = s == 0 ? (__fsub_rn(C0, t) > margin) : (__fsub_rn(t, C0) > margin);
    return s;
}

// Chunk step of the inverse CDF: the smallest chunk c (of nc) whose
// inclusive, inertia-corrected prefix Gc(c) (+ delta when label xi lies at
// or below the chunk's end) exceeds t.
template <typename ChunkG>
__device__ __forceinline__ int cdf_find_chunk(ChunkG Gc, int nc, float t, float delta, int xi)
{
    int lo = 0, hi = nc - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float gm = __fadd_rn(Gc(mid), (xi <= mid * kChunk + kChunk - 1) ? delta : 0.0f);
        if (t < gm)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Label step of the inverse CDF inside chunk cs, whose predecessors sum to
// Gprev, with the certification: chunk_prefix(c, p) must return the
// inclusive prefix sums p[0..7] of chunk c's weights, bit-identical to the
// weights behind the chunk sums.  Returns the label; `certain` is false when
// t = u Z lies within eta Z of an end of the chosen label's CDF interval.
template <typename ChunkPrefix>
__device__ __forceinline__ int cdf_finish(const DevModel &m, float eta, int cs, float Gprev,
                                          float Z, float t, float delta, int xi, bool &certain,
                                          ChunkPrefix chunk_prefix)
{
    const int base = cs * kChunk;
    const int kmax = min(kChunk - 1, m.L - 1 - base);
    if (kmax < 0) {  // only reachable through rounding: leave it to FP64
        certain = false;
        return m.L - 1;
    }
    float p[kChunk];
    chunk_prefix(cs, p);
    int k = kmax;
    float hiC = 0.0f;
    bool found = false;
#pragma unroll
    for (int kk = kChunk - 1; kk >= 0; --kk) {
        const float Ck = __fadd_rn(__fadd_rn(Gprev, p[kk]), (base + kk >= xi) ? delta : 0.0f);
        if (kk <= kmax && t < Ck) {
            k = kk;
            hiC = Ck;
            found = true;
        }
    }
    if (!found)
        hiC = __fadd_rn(__fadd_rn(Gprev, p[kmax]), (base + kmax >= xi) ? delta : 0.0f);
    float loC;
    if (k > 0)
        loC = __fadd_rn(__fadd_rn(Gprev, p[k - 1]), (base + k - 1 >= xi) ? delta : 0.0f);
    else
        loC = __fadd_rn(Gprev, (base - 1 >= xi) ? delta : 0.0f);
    const int s = max(0, base + k);
    const float margin = __fmul_rn(eta, Z);
    const bool ok_hi = (s == m.L - 1) || (__fsub_rn(hiC, t) > margin);
    const bool ok_lo = (s == 0) || (__fsub_rn(t, loC) > margin);
    certain = found && ok_hi && ok_lo;
    return min(s, m.L - 1);
}

// Inverse-CDF selection shared by the FP32 draws.  Gc(c) returns the
// inclusive prefix sum of the inertia-free weights up to chunk c (of nc), G
// their total; delta is the inertia correction added at and above label xi;
// ub the 24-bit uniform numerator.
template <typename ChunkG, typename ChunkPrefix>
__device__ __forceinline__ int cdf_select(const DevModel &m, float eta, ChunkG Gc, int nc,
                                          float G, float delta, int xi, uint32_t ub,
                                          bool &certain, ChunkPrefix chunk_prefix)
{
    const float Z = __fadd_rn(G, delta);
    const float t = __fmul_rn((float)ub * (1.0f / 16777216.0f), Z);
    const int cs = cdf_find_chunk(Gc, nc, t, delta, xi);
    const float Gprev = cs > 0 ? Gc(cs - 1) : 0.0f;
    return cdf_finish(m, eta, cs, Gprev, Z, t, delta, xi, certain, chunk_prefix);
}

// FP32 inverse-CDF draw.  Gcol points at this thread's column of a shared
// scratch array (stride gstride floats) holding the chunk prefix sums.
// Returns the label; `certain` is false when the uniform lies within the
// error bound of a boundary of the chosen label's CDF interval.
template <int NC, int NB>
__device__ __forceinline__ int draw_fp32(const DevModel &m, float *Gcol, int gstride,
                                         const SiteIn<NB> &in, uint32_t dirty, bool &certain)
{
    if (NC == 1 && m.L == 2)
        return draw_binary<NB>(m, in, certain);
    float xn[NB];
    __half2 xh[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        xn[j] = (float)in.xni[j];
        xh[j] = __float2half2_rn(xn[j]);
    }
    const __half2 T2 = __float2half2_rn(m.Tf);
    const float gf = (float)in.g;
    const int xi = in.xi;
    float pdummy[kChunk];
    // pass 1: chunk prefix sums of the inertia-free weights (Kahan-compensated)
    float G = 0.0f, comp = 0.0f;
    const int nfull = m.L / kChunk;  // chunks with no label >= L
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        float S;
        if ((dirty >> c) & 1u)   // warp-uniform branch
            S = (c < nfull) ? chunk_weights<NB, false, false>(m, xh, T2, gf, c, pdummy)
                            : chunk_weights<NB, true, false>(m, xh, T2, gf, c, pdummy);
        else
            S = (c < nfull) ? chunk_weights_linear<NB, false>(m, xh, T2, gf, c)
                            : chunk_weights_linear<NB, true>(m, xh, T2, gf, c);
        const float y = __fsub_rn(S, comp);
        const float tt = __fadd_rn(G, y);
        comp = __fsub_rn(__fsub_rn(tt, G), y);
        G = tt;
        Gcol[c * gstride] = G;
    }
    float delta = 0.0f;
    if (m.em1 != 0.0f)
        delta = __fmul_rn(single_w<NB>(m, xn, gf, xi), m.em1);
    // gam <= 0: both exponent terms are non-positive, the per-site margin holds
    const float eta = m.gam <= 0.0f ? site_margin(m, G, delta) : m.eta;
    return cdf_select(m, eta, [&](int c) { return Gcol[c * gstride]; }, NC, G, delta, xi,
                      in.ub, certain, [&](int cs, float (&p)[kChunk]) {
                          chunk_weights<NB, true, true>(m, xh, T2, gf, cs, p);
                      });
}

// ------------------------------------------------- Lp inertia price (p = 1, 2)
// Exponent v' = alpha (g - s)^2 + gam P(s) + kappa R(s) + c with R = |s - x_i|^p
// (exact integers) and the per-site shift c = |kappa| |g - x_i|^p, evaluated
// as one FFMA chain: kappa R + c, + gam P, + alpha Q.

__device__ __forceinline__ float label_wn(const DevModel &m, float P, float dg, float R, float c)
{
    const float q = __fmul_rn(dg, dg);
    const float t1 = __fmaf_rn(m.kappa, R, c);
    const float t2 = __fmaf_rn(m.gam, P, t1);
    return ex2_ftz(__fmaf_rn(m.alpha, q, t2));
}

// Weights of labels [8c, 8c + 8) with the Lp price; as chunk_weights.
template <int NB, bool MASK, bool PREFIX, int NORM>
__device__ __forceinline__ float chunk_weights_n(const DevModel &m, const __half2 (&xh)[NB],
                                                 __half2 T2, float gf, float xif, float csite,
                                                 int c, float (&p)[kChunk])
{
    const float sbf = (float)(c * kChunk);
    const __half2 sb2 = __float2half2_rn(sbf);
    __half2 xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xr[j] = __hsub2(xh[j], sb2);
    const float dgb = gf - sbf;
    const float dxb = sbf - xif;
    float S = 0.0f;
#pragma unroll
    for (int kk = 0; kk < kChunk; kk += 2) {
        const float2 P = prior_pair<NB>(xr, __floats2half2_rn((float)kk, (float)(kk + 1)), T2);
        const float d0 = dxb + (float)kk, d1 = dxb + (float)(kk + 1);
        const float R0 = NORM == 1 ? fabsf(d0) : __fmul_rn(d0, d0);
        const float R1 = NORM == 1 ? fabsf(d1) : __fmul_rn(d1, d1);
        float e0 = label_wn(m, P.x, dgb - (float)kk, R0, csite);
        float e1 = label_wn(m, P.y, dgb - (float)(kk + 1), R1, csite);
        if (MASK) {
            if (c * kChunk + kk >= m.L) e0 = 0.0f;
            if (c * kChunk + kk + 1 >= m.L) e1 = 0.0f;
        }
        S = __fadd_rn(S, e0);
        if (PREFIX) p[kk] = S;
        S = __fadd_rn(S, e1);
        if (PREFIX) p[kk + 1] = S;
    }
    return S;
}

// FP32 inverse-CDF draw with the Lp price (no single-label correction: the
// price is part of every weight); as draw_fp32.
template <int NC, int NB, int NORM>
__device__ __forceinline__ int draw_fp32_norm(const DevModel &m, float *Gcol, int gstride,
                                              const SiteIn<NB> &in, bool &certain)
{
    __half2 xh[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xh[j] = __float2half2_rn((float)in.xni[j]);
    const __half2 T2 = __float2half2_rn(m.Tf);
    const float gf = (float)in.g;
    const float xif = (float)in.xi;
    const float D = fabsf(gf - xif);
    const float csite = __fmul_rn(-m.kappa, NORM == 1 ? D : __fmul_rn(D, D));
    float pdummy[kChunk];
    float G = 0.0f, comp = 0.0f;
    const int nfull = m.L / kChunk;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        const float S = (c < nfull)
                            ? chunk_weights_n<NB, false, false, NORM>(m, xh, T2, gf, xif, csite, c,
                                                                      pdummy)
                            : chunk_weights_n<NB, true, false, NORM>(m, xh, T2, gf, xif, csite, c,
                                                                     pdummy);
        const float y = __fsub_rn(S, comp);
        const float tt = __fadd_rn(G, y);
        comp = __fsub_rn(__fsub_rn(tt, G), y);
        G = tt;
        Gcol[c * gstride] = G;
    }
    return cdf_select(m, m.eta, [&](int cc) { return Gcol[cc * gstride]; }, NC, G, 0.0f, in.xi,
                      in.ub, certain, [&](int cs, float (&pp)[kChunk]) {
                          chunk_weights_n<NB, true, true, NORM>(m, xh, T2, gf, xif, csite, cs, pp);
                      });
}

// ------------------------------------------------------------ FP64 re-draw

template <int NB, int NORM = 0>
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
    if constexpr (NORM != 0)
        w = __dmul_rn(w, m.in64[abs(s - xi)]);
    else if (m.em1 != 0.0f && s == xi)
        w = __dmul_rn(w, m.el64);
    return w;
}

// Warp-cooperative FP64 evaluation of the draws of the lanes with `need`
// set: for each such lane in turn, the 32 lanes compute 8 labels' FP64
// weights each, an FP64 warp scan gives the CDF, and the lane holding u*Z
// finds the label.  All 32 lanes of the warp must call this together.
template <int NB, int NORM = 0>
__device__ __forceinline__ int warp_redraw_fp64(const DevModel &m, bool need, const SiteIn<NB> &in,
                                                int s, unsigned long long *counter)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    unsigned todo = __ballot_sync(kFull, need);
    if (todo == 0u)
        return s;
    const int lane = (int)(threadIdx.x & 31u);
    if (lane == 0)
        atomicAdd(counter, (unsigned long long)__popc(todo));
    while (todo) {
        const int leader = __ffs((int)todo) - 1;
        todo &= todo - 1u;
        const int lg = __shfl_sync(kFull, in.g, leader);
        const int lxi = __shfl_sync(kFull, in.xi, leader);
        int lx[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j)
            lx[j] = __shfl_sync(kFull, in.xni[j], leader);
        const uint32_t lub = __shfl_sync(kFull, in.ub, leader);
        double w[kChunk];
        double part = 0.0;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            const int sl = lane * kChunk + k;
            w[k] = sl < m.L ? weight64<NB, NORM>(m, lg, lxi, lx, sl) : 0.0;
            part = __dadd_rn(part, w[k]);
        }
        double incl = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o)
                incl = __dadd_rn(incl, v);
        }
        const double Z = __shfl_sync(kFull, incl, 31);
        const double t = __dmul_rn((double)lub * (1.0 / 16777216.0), Z);
        double excl = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0)
            excl = 0.0;
        const unsigned hit = __ballot_sync(kFull, t < incl);
        const int hl = hit ? __ffs((int)hit) - 1 : 31;
        int res = 0;
        if (lane == hl) {
            double C = excl;
            res = min(lane * kChunk + kChunk - 1, m.L - 1);
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                C = __dadd_rn(C, w[k]);
                if (t < C && lane * kChunk + k < m.L) {
                    res = lane * kChunk + k;
                    break;
                }
            }
        }
        res = __shfl_sync(kFull, res, hl);
        if (lane == leader)
            s = res;
    }
    return s;
}

}  // namespace pcad
