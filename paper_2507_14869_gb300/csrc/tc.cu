// Lazy-PCA sweep with the prior sums on the tensor cores (Section 5.2, Eq.
// posterior_pca_transition_matrix), for models with many labels.
//
// For label s the truncated-linear prior sum is
//   P(s) = sum_j min(|x_j - s|, T) = n T - Pb(s),  Pb(s) = sum_j max(T - |x_j - s|, 0),
// n the number of neighbours inside the image.  n T is the same for every
// label of the site and cancels in the normalisation, so the weights are
// built from Pb: w(s) = 2^(alpha (g - s)^2 + mu Pb(s)), mu = c log2(e).
// Pb is the product of the site's neighbour-label histogram h (a row with at
// most NB nonzero counts) and the banded Toeplitz matrix
// K(t, s) = max(T - |t - s|, 0): a contraction whose operands are small
// integers, exact with FP16 inputs and FP32 accumulation.
//
// 128 sites (4 image rows x 32 columns) form the M dimension of one
// tcgen05.mma, one TMEM lane per site.  Labels form N in tiles of 64.  K is
// banded, so a label tile [s0, s0 + 64) only needs histogram columns
// (s0 - T, s0 + 64 + T); with the histogram padded by o >= T - 1 columns on
// both sides, the window [s0 - o, s0 + 64 + o) of every label tile meets
// the same 64 x (64 + 2o) block of K, so one small B operand serves all
// tiles.  For L = 256, T = 30: 32 MMAs of 128 x 64 x 16 per 128 sites.
//
// One persistent CTA per SM runs a four-stage warp-specialised pipeline over
// its tiles (128-site tiles strided over the grid), double-buffered in the
// histogram operand A (shared memory), the accumulators (TMEM) and the
// chunk sums G, with a ring of four slots of staged site inputs:
//   * loader warps (4, one thread per site): read the site's labels,
//     observation and uniform into the stage ring, write its histogram row
//     of A[i & 1] (clearing the row's entries of tile i - 2) once the MMAs
//     of tile i - 2 completed, arrive on barA and barS;
//   * MMA warp (one elected thread): once A is written (barA) and pass 1 of
//     tile i - 2 has read TMEM buffer i & 1 (barP), issue tile i's 32 MMAs
//     into that buffer and commit them to barM;
//   * pass-1 warps (16, four threads per site, one per quarter of the label
//     groups): wait barM, read their part of the site's accumulator row
//     (tcgen05.ld, 32 labels per load), evaluate exponent, exp2 and the
//     Kahan chunk prefix sums into G[i & 1], arrive on barP;
//   * selector warps (4, one thread per site): wait barS and barP, join the
//     parts' prefix sums, add the inertia correction, select chunk and label
//     (certified, pass 2 on the CUDA cores), arrive on barG (G free),
//     re-draw uncertain draws in FP64 by the warp, write the label and the
//     accumulator, arrive on barF (stage slot free).
// Each buffer is released by the stage that last reads it, so no cycle of
// the dependency graph runs through all four stages.  The tensor core, the
// exp2/CDF work and the selection of consecutive tiles overlap.  Every wait
// is bounded: on timeout a warp records an error flag and leaves its loop
// (the others then time out in turn), the MMA warp waits (bounded) for the
// MMAs it issued, and TMEM is freed before return.
//
// The draw is the certified FP32 inverse CDF of the CUDA-core kernel (same
// uniforms, same selection) with the error bound of this formulation; the
// four parts' prefix sums are joined by three more roundings (24u of
// summation).
#include <cuda_fp16.h>

#include "async_ptx.cuh"
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kSites = 128;                   // tile: 4 rows x 32 columns = MMA M
constexpr int kTileRows = 4;
// Warp roles: loader warps 0-3, pass-1 warps 4 .. 4 + 4 kP1Parts - 1,
// selector warps (4), MMA warp.  Pass-1 warp 4 + 4h + q handles label part
// h of the sites in TMEM lanes 32 q .. 32 q + 31 (a warp reaches the lane
// quarter given by its index mod 4).
constexpr int kLoadWarp0 = 0;
constexpr int kP1Warp0 = 4;
#ifndef PCAD_TC_PARTS
#define PCAD_TC_PARTS 2
#endif
constexpr int kP1Parts = PCAD_TC_PARTS;
constexpr int kSelWarp0 = kP1Warp0 + 4 * kP1Parts;
constexpr int kMmaWarp = kSelWarp0 + 4;
constexpr int kLoadThreads = kSites;
constexpr int kSelThreads = kSites;
constexpr int kTcThreads = (kMmaWarp + 1) * 32;
constexpr int kLabelTile = 64;                // MMA N
constexpr int kASlab = kSites * 128;          // bytes of a 64-column slab of A (128 rows)
constexpr int kBSlab = kLabelTile * 128;      // bytes of a 64-column slab of B (64 rows)
constexpr long long kTcSpinLimit = 20000000;  // ~1 s of polling
constexpr uint32_t kIdesc = idesc_f16_f32(kSites, kLabelTile);
constexpr int kSmemPerSM = 233472;            // shared memory of one SM (228 KB)
constexpr int kSmemReserved = 1024;           // reserved per resident CTA
constexpr int kSmemMax = kSmemPerSM - kSmemReserved;
constexpr int kTmemCols = 512;

// Shape of one model's operands (host-computed).
struct TcLayout {
    int o;           // histogram padding: multiple of 16, >= T - 1
    int kw;          // K window of one label tile: 64 + 2o
    int nt;          // label tiles
    int a_slabs;     // 64-column slabs of one A buffer (nt * 64 + 2o columns)
    int b_slabs;     // 64-column slabs of B (kw columns)
    int tmem_cols;   // accumulator columns of one buffer (power of two >= nt * 64)
    int nc;          // 8-label chunks, ceil(L / 8)
    int ng;          // 32-label groups, ceil(L / 32); part h takes [h ng / 4, (h + 1) ng / 4)
    int smem;        // dynamic shared memory bytes
};

// Ring of staged site inputs.
constexpr int kRing = 4;
constexpr int kStageBytes = 2048;   // per slot: see TcSmem

TcLayout tc_layout(int L, int T)
{
    TcLayout t{};
    t.o = (T - 1 + 15) / 16 * 16;
    t.kw = kLabelTile + 2 * t.o;
    t.nt = (L + kLabelTile - 1) / kLabelTile;
    t.a_slabs = (t.nt * kLabelTile + 2 * t.o + 63) / 64;
    t.b_slabs = (t.kw + 63) / 64;
    t.tmem_cols = 32;
    while (t.tmem_cols < t.nt * kLabelTile)
        t.tmem_cols *= 2;
    t.nc = (L + kChunk - 1) / kChunk;
    t.ng = (L + 31) / 32;
    t.smem = 2 * t.a_slabs * kASlab + t.b_slabs * kBSlab + 2 * t.nc * kSites * 4 +
             kRing * kStageBytes + 8 * (6 + 4 * kP1Parts + 2 * kRing) + 64;
    // no more resident CTAs than TMEM can hold (two buffers each): pad the
    // shared memory request
    const int max_ctas = kTmemCols / (2 * t.tmem_cols);
    const int min_smem = kSmemPerSM / (max_ctas + 1) - kSmemReserved + 1;
    if (t.smem < min_smem)
        t.smem = (min_smem + 15) / 16 * 16;
    return t;
}

// Byte offset of element (row, k) of a K-major, 128-byte-swizzled operand
// stored as 64-column slabs of `slab` bytes (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k, int slab)
{
    return (uint32_t)((k >> 6) * slab + (row >> 3) * 1024 + (row & 7) * 128 +
                      ((((k & 63) >> 3) ^ (row & 7)) << 4) + ((k & 7) << 1));
}

// Weight of one label from the banded prior sum Pb (an exact integer):
// 2^(alpha dg^2 + mu Pb).
__device__ __forceinline__ float label_wb(float alpha, float mu, float Pb, float dg)
{
    const float q = __fmul_rn(dg, dg);
    const float v = __fmaf_rn(alpha, q, __fmul_rn(mu, Pb));
    return ex2_ftz(v);
}

// Inclusive prefix sums of chunk c's weights on the CUDA cores, bit-identical
// to the tensor-core pass: Pb = NB T - P with P from the half-precision prior
// (missing neighbours give T - T = 0 in both).
template <int NB>
__device__ __forceinline__ void chunk_prefix_b(const DevModel &m, float mu, float nbT,
                                               const __half2 (&xh)[NB], __half2 T2, float gf,
                                               int c, float (&p)[kChunk])
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
        float e0 = label_wb(m.alpha, mu, __fsub_rn(nbT, P.x), dgb - (float)kk);
        float e1 = label_wb(m.alpha, mu, __fsub_rn(nbT, P.y), dgb - (float)(kk + 1));
        if (c * kChunk + kk >= m.L)
            e0 = 0.0f;
        if (c * kChunk + kk + 1 >= m.L)
            e1 = 0.0f;
        S = __fadd_rn(S, e0);
        p[kk] = S;
        S = __fadd_rn(S, e1);
        p[kk + 1] = S;
    }
}

// Weight of the single label s (inertia correction), same formula.
template <int NB>
__device__ __forceinline__ float single_wb(const DevModel &m, float mu, float nbT,
                                           const float (&xn)[NB], float gf, int s)
{
    const float sf = (float)s;
    float P = fminf(fabsf(xn[0] - sf), m.Tf);
#pragma unroll
    for (int j = 1; j < NB; ++j)
        P = __fadd_rn(P, fminf(fabsf(xn[j] - sf), m.Tf));
    return label_wb(m.alpha, mu, __fsub_rn(nbT, P), gf - sf);
}

// Pass 1 over one group of 32 labels [32 grp, 32 grp + 32) whose banded
// prior sums are in pb: four chunk sums, Kahan-accumulated into G and stored
// as chunk prefix sums (stride kSites).  MASK zeroes labels >= L.
template <bool MASK>
__device__ __forceinline__ void group_pass(const DevModel &m, float mu, float gf, int grp,
                                           const uint32_t (&pb)[32], int nc, float *Gcol,
                                           float &G, float &comp)
{
    const float dgb = gf - (float)(grp * 32);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float S = 0.0f;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            const int kk = i * kChunk + k;
            float e = label_wb(m.alpha, mu, __uint_as_float(pb[kk]), dgb - (float)kk);
            if (MASK && grp * 32 + kk >= m.L)
                e = 0.0f;
            S = __fadd_rn(S, e);
        }
        const float y = __fsub_rn(S, comp);
        const float tt = __fadd_rn(G, y);
        comp = __fsub_rn(__fsub_rn(tt, G), y);
        G = tt;
        const int c = grp * 4 + i;
        if (c < nc)
            Gcol[c * kSites] = G;
    }
}

// Shared-memory carve-up of one CTA:
//   A[2]      histogram operands (buffer b at A0 + b * a_bytes)
//   B         band block of K
//   G[2]      chunk prefix sums [chunk][site] (buffer b at G0 + b * g_elems),
//             each label part's chunks prefix-summed from its own start
//   stage[4]  site inputs: uniform u32[128], neighbour labels u8[8][128],
//             missing-neighbour bits u8[128], label u8[128], observation u8[128]
//   barriers  barA[2] (A written, count kLoadThreads), barM[2][4] (MMAs of
//             label tile / part h done, by commit), barP[2][4] (part h read
//             its TMEM columns and wrote its chunk sums, kSites),
//             barG[2] (selection done with G, kSelThreads), barS[4] (stage
//             written, kLoadThreads), barF[4] (selection done with the stage,
//             kSelThreads)
struct TcSmem {
    uint8_t *A0;
    int a_bytes;
    uint8_t *B;
    float *G0;
    int g_elems;
    uint8_t *S0;
    uint64_t *barA, *barM, *barP, *barG, *barS, *barF;
    uint32_t *tmem_slot;
};

constexpr int kStageXn = 4 * kSites;
constexpr int kStageMiss = kStageXn + 8 * kSites;
constexpr int kStageXi = kStageMiss + kSites;
constexpr int kStageG = kStageXi + kSites;
static_assert(kStageG + kSites <= kStageBytes, "stage slot");

__device__ __forceinline__ TcSmem carve(uint8_t *base, const TcLayout &lay)
{
    TcSmem s;
    s.a_bytes = lay.a_slabs * kASlab;
    s.A0 = base;
    s.B = base + 2 * s.a_bytes;
    s.G0 = reinterpret_cast<float *>(s.B + lay.b_slabs * kBSlab);
    s.g_elems = lay.nc * kSites;
    s.S0 = reinterpret_cast<uint8_t *>(s.G0 + 2 * s.g_elems);
    uint64_t *bars = reinterpret_cast<uint64_t *>(s.S0 + kRing * kStageBytes);
    s.barA = bars;                        // [b]
    s.barM = bars + 2;                    // [b * kP1Parts + h]
    s.barP = s.barM + 2 * kP1Parts;       // [b * kP1Parts + h]
    s.barG = s.barP + 2 * kP1Parts;       // [b]
    s.barS = s.barG + 2;                  // [slot]
    s.barF = s.barS + kRing;              // [slot]
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.barF + kRing);
    return s;
}

// Label groups [g_lo, g_hi) of pass-1 part h.
__host__ __device__ __forceinline__ int part_lo(int ng, int h)
{
    return h * ng / kP1Parts;
}

__device__ __forceinline__ void tile_site(const SweepArgs &a, int tiles_x, int i, int site, int &r,
                                          int &c)
{
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    r = (tile / tiles_x) * kTileRows + (site >> 5);
    c = (tile % tiles_x) * 32 + (site & 31);
}

// Waits for phase `use` of a barrier that completes once per use (use 0, 1, ...).
__device__ __forceinline__ bool wait_use(uint64_t *bar, int use)
{
    return mbar_wait_bounded(bar, (uint32_t)use & 1u, kTcSpinLimit);
}

// Site inputs of one site from a stage slot.
template <int NB>
__device__ __forceinline__ void stage_get(const uint8_t *S, int site, SiteIn<NB> &in)
{
    in.ub = reinterpret_cast<const uint32_t *>(S)[site];
    const uint32_t miss = S[kStageMiss + site];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        in.xni[j] = ((miss >> j) & 1u) ? kMissingLabelI : (int)S[kStageXn + j * kSites + site];
    in.xi = S[kStageXi + site];
    in.g = S[kStageG + site];
}

// Loader warps: inputs into the stage ring, histogram rows into A.
template <int NB>
__device__ __forceinline__ bool load_role(const SweepArgs &a, const TcLayout &lay,
                                          const TcSmem &sm, int n_my, int tiles_x)
{
    const int site = (int)threadIdx.x - kLoadWarp0 * 32;
    const uint32_t t = sweep_index(a);
    // A entries this row set for the tiles two back (this iteration's
    // buffer) and one back (~0u: none)
    uint32_t off2[NB], off1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        off2[j] = off1[j] = ~0u;
    for (int i = 0; i < n_my; ++i) {
        const int b = i & 1;
        const int q = i & (kRing - 1);
        int r, c;
        tile_site(a, tiles_x, i, site, r, c);
        const bool valid = r < a.H && c < a.W;
        SiteIn<NB> in{};
        if (valid)
            load_site<NB>(a, a.xin, r, c, kTagPCA, t, in);
        if (i >= 2 && !wait_use(&sm.barM[b * kP1Parts + kP1Parts - 1], (i - 2) >> 1))  // A[b] read
            return false;
        if (i >= kRing && !wait_use(&sm.barF[q], (i - kRing) >> 2))  // stage slot free
            return false;
        uint8_t *S = sm.S0 + q * kStageBytes;
        reinterpret_cast<uint32_t *>(S)[site] = in.ub;
        uint32_t miss = 0;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const bool m = in.xni[j] >= kMissingLabelI;
            miss |= (m ? 1u : 0u) << j;
            S[kStageXn + j * kSites + site] = m ? 0 : (uint8_t)in.xni[j];
        }
        S[kStageMiss + site] = (uint8_t)miss;
        S[kStageXi + site] = (uint8_t)in.xi;
        S[kStageG + site] = (uint8_t)in.g;
        uint8_t *A = sm.A0 + b * sm.a_bytes;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (off2[j] != ~0u)
                *reinterpret_cast<__half *>(A + off2[j]) = __ushort_as_half((unsigned short)0);
        // one store per distinct neighbour label, of its multiplicity
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            off2[j] = off1[j];
            off1[j] = ~0u;
            bool first = valid && in.xni[j] < kMissingLabelI;
            int cnt = 1;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (k < j && in.xni[k] == in.xni[j])
                    first = false;
                if (k > j && in.xni[k] == in.xni[j])
                    ++cnt;
            }
            if (first) {
                const uint32_t off = sw128_offset(site, in.xni[j] + lay.o, kASlab);
                *reinterpret_cast<__half *>(A + off) = __int2half_rn(cnt);
                off1[j] = off;
            }
        }
        fence_async_smem();
        mbar_arrive(&sm.barA[b]);
        mbar_arrive(&sm.barS[q]);
    }
    return true;
}

// Byte offsets (in 16-byte units, the descriptors' address unit) of the
// K step at histogram column kp of A and window column kb of B.
__host__ __device__ constexpr uint32_t a_step16(int kp)
{
    return (uint32_t)(((kp >> 6) * kASlab + (kp & 63) * 2) >> 4);
}
__host__ __device__ constexpr uint32_t b_step16(int kb)
{
    return (uint32_t)(((kb >> 6) * kBSlab + (kb & 63) * 2) >> 4);
}

// MMAs of label tile lt of one tile: its K window in ksteps steps into TMEM
// columns [d0 + 64 lt, d0 + 64 lt + 64).  The start-address field of a
// descriptor is its low 14 bits and every address stays below 256 KB, so
// adding an offset to the descriptor moves its start.
template <int KS>
__device__ __forceinline__ void issue_label_tile(uint64_t adesc, uint64_t bdesc, uint32_t d0,
                                                 int lt, int ksteps)
{
    if constexpr (KS > 0) {
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
            umma_f16_ss(d0 + (uint32_t)(lt * kLabelTile),
                        adesc + a_step16(lt * kLabelTile + ks * 16), bdesc + b_step16(ks * 16),
                        kIdesc, ks > 0 ? 1u : 0u);
    } else {
        for (int ks = 0; ks < ksteps; ++ks)
            umma_f16_ss(d0 + (uint32_t)(lt * kLabelTile),
                        adesc + a_step16(lt * kLabelTile + ks * 16), bdesc + b_step16(ks * 16),
                        kIdesc, ks > 0 ? 1u : 0u);
    }
}

// MMA warp: one elected thread issues each tile's MMAs once A is written
// (barA) and TMEM buffer i & 1 has been read by pass 1 of tile i - 2
// (barP).  With the fixed shape (NT = 4 label tiles = the 4 pass-1 parts,
// KS K steps) label tile h waits only for part h and is committed on its
// own (barM[b][h]), so pass 1 and the MMAs overlap inside a tile; other
// shapes wait for all parts and commit once to every part.  Before
// returning the thread waits (bounded) for the MMAs it issued, so TMEM can
// be freed.
template <int NT, int KS>
__device__ __forceinline__ bool mma_role(const TcLayout &lay, const TcSmem &sm, uint32_t tmem,
                                         int n_my)
{
    static_assert(NT % kP1Parts == 0, "fixed shape: whole label tiles per pass-1 part");
    constexpr int kTpp = NT / kP1Parts;   // label tiles per part (fixed shape)
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0) {
        const uint64_t bdesc = sw128_kmajor_desc(smem_u32(sm.B));
        const uint64_t adesc0 = sw128_kmajor_desc(smem_u32(sm.A0));
        const uint64_t adesc1 = sw128_kmajor_desc(smem_u32(sm.A0 + sm.a_bytes));
        const int ksteps = lay.kw / 16;
        int issued = 0;
        for (int i = 0; i < n_my && ok; ++i) {
            const int b = i & 1;
            const uint64_t adesc = b ? adesc1 : adesc0;
            const uint32_t d0 = tmem + (uint32_t)(b * lay.tmem_cols);
            if (!wait_use(&sm.barA[b], i >> 1)) {
                ok = 0;
                break;
            }
            if constexpr (NT > 0) {
#pragma unroll
                for (int h = 0; h < kP1Parts; ++h) {
                    if (i >= 2 && !wait_use(&sm.barP[b * kP1Parts + h], (i - 2) >> 1)) {
                        ok = 0;
                        break;
                    }
                    tc_fence_after_sync();
#pragma unroll
                    for (int lt = h * kTpp; lt < (h + 1) * kTpp; ++lt)
                        issue_label_tile<KS>(adesc, bdesc, d0, lt, ksteps);
                    umma_commit(&sm.barM[b * kP1Parts + h]);
                }
            } else {
                for (int h = 0; h < kP1Parts && ok; ++h)
                    if (i >= 2 && !wait_use(&sm.barP[b * kP1Parts + h], (i - 2) >> 1))
                        ok = 0;
                if (!ok)
                    break;
                tc_fence_after_sync();
                for (int lt = 0; lt < lay.nt; ++lt)
                    issue_label_tile<0>(adesc, bdesc, d0, lt, ksteps);
                for (int h = 0; h < kP1Parts; ++h)
                    umma_commit(&sm.barM[b * kP1Parts + h]);
            }
            if (ok)
                ++issued;
        }
        // every commit of the last tiles (a partly issued one included) has
        // completed once the last label tile's barrier of each buffer has
        for (int k = issued - 2; k < issued + (ok ? 0 : 1); ++k)
            if (k >= 0 && k < n_my)
                mbar_wait_bounded(&sm.barM[(k & 1) * kP1Parts + kP1Parts - 1],
                                  (uint32_t)(k >> 1) & 1u, kTcSpinLimit);
    }
    __syncwarp();
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// Pass-1 warps: exponent, exp2 and chunk prefix sums of one label part of
// each site from the accumulators into G.
__device__ __forceinline__ bool pass1_role(const SweepArgs &a, const TcLayout &lay,
                                           const TcSmem &sm, uint32_t tmem, int n_my,
                                           int tiles_x)
{
    const int idx = (int)(threadIdx.x >> 5) - kP1Warp0;   // 0..15
    const int q = idx & 3;                                // lane quarter = warp index mod 4
    const int part = idx >> 2;
    const int site = q * 32 + (int)(threadIdx.x & 31);
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const int g_lo = part_lo(lay.ng, part);
    const int g_hi = part_lo(lay.ng, part + 1);
    const float mu = -a.m.gam;
    for (int i = 0; i < n_my; ++i) {
        const int b = i & 1;
        int r, c;
        tile_site(a, tiles_x, i, site, r, c);
        const float gf = (r < a.H && c < a.W) ? (float)a.g[(size_t)r * a.pitch + c] : 0.0f;
        bool ok = wait_use(&sm.barM[b * kP1Parts + part], i >> 1);
        if (ok && i >= 2)   // the selection of tile i - 2 has read G[b]
            ok = wait_use(&sm.barG[b], (i - 2) >> 1);
        if (__any_sync(0xFFFFFFFFu, !ok))   // tcgen05.ld below is warp-collective
            return false;
        tc_fence_after_sync();
        float *Gcol = sm.G0 + b * sm.g_elems + site;
        float G = 0.0f, comp = 0.0f;
        const uint32_t tb = trow + (uint32_t)(b * lay.tmem_cols);
#pragma unroll 1
        for (int grp = g_lo; grp < g_hi; ++grp) {
            uint32_t pb[32];
            tmem_ld32(tb + (uint32_t)(grp * 32), pb);
            tmem_wait_ld(pb);
            if ((grp + 1) * 32 > a.m.L)
                group_pass<true>(a.m, mu, gf, grp, pb, lay.nc, Gcol, G, comp);
            else
                group_pass<false>(a.m, mu, gf, grp, pb, lay.nc, Gcol, G, comp);
        }
        tc_fence_before_sync();
        mbar_arrive(&sm.barP[b * kP1Parts + part]);   // TMEM columns read, chunk sums written
    }
    return true;
}

// Selector warps: inertia, joining of the label parts' prefix sums, the
// certified chunk and label selection (pass 2 on the CUDA cores), FP64
// re-draws, writes.
template <int NB>
__device__ __forceinline__ bool select_role(const SweepArgs &a, const TcLayout &lay,
                                            const TcSmem &sm, int n_my, int tiles_x)
{
    const int site = (int)threadIdx.x - kSelWarp0 * 32;   // 0..127
    const uint32_t t = sweep_index(a);
    const float mu = -a.m.gam;
    const float nbT = (float)(NB * a.m.T);
    const int nc = lay.nc;
    // first group of every part and the last chunk of every part (-1: empty)
    int gstart[kP1Parts];
    int last[kP1Parts];
#pragma unroll
    for (int h = 0; h < kP1Parts; ++h) {
        const int lo = part_lo(lay.ng, h), hi = part_lo(lay.ng, h + 1);
        gstart[h] = lo;
        last[h] = hi > lo ? min(4 * hi, nc) - 1 : -1;
    }
    for (int i = 0; i < n_my; ++i) {
        const int b = i & 1;
        const int rq = i & (kRing - 1);
        int r, c;
        tile_site(a, tiles_x, i, site, r, c);
        const bool valid = r < a.H && c < a.W;
        bool ok = wait_use(&sm.barS[rq], i >> 2);
#pragma unroll
        for (int h = 0; h < kP1Parts; ++h)
            ok = ok && wait_use(&sm.barP[b * kP1Parts + h], i >> 1);
        if (__any_sync(0xFFFFFFFFu, !ok))   // the re-draw below is warp-collective
            return false;
        SiteIn<NB> in;
        stage_get<NB>(sm.S0 + rq * kStageBytes, site, in);
        const float *Gcol = sm.G0 + b * sm.g_elems + site;
        int s = 0;
        bool certain = true;
        float xn[NB];
        __half2 xh[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            xn[j] = (float)in.xni[j];
            xh[j] = __float2half2_rn(xn[j]);
        }
        const float gf = (float)in.g;
        float delta = 0.0f, Z = 0.0f, tu = 0.0f, Gprev = 0.0f;
        int cs = 0;
        if (valid) {
            // offsets of the parts: sums of the preceding parts' totals
            float O[kP1Parts + 1];
            O[0] = 0.0f;
#pragma unroll
            for (int h = 0; h < kP1Parts; ++h)
                O[h + 1] = last[h] >= 0 ? __fadd_rn(O[h], Gcol[last[h] * kSites]) : O[h];
            const auto Gc = [&](int cc) {
                const int g = cc >> 2;
                float off = O[0];
#pragma unroll
                for (int h = 1; h < kP1Parts; ++h)
                    off = g >= gstart[h] ? O[h] : off;
                return __fadd_rn(off, Gcol[cc * kSites]);
            };
            if (a.m.em1 != 0.0f)
                delta = __fmul_rn(single_wb<NB>(a.m, mu, nbT, xn, gf, in.xi), a.m.em1);
            // the steps of cdf_select, with G released after the chunk search
            Z = __fadd_rn(O[kP1Parts], delta);
            tu = __fmul_rn((float)in.ub * (1.0f / 16777216.0f), Z);
            cs = cdf_find_chunk(Gc, nc, tu, delta, in.xi);
            Gprev = cs > 0 ? Gc(cs - 1) : 0.0f;
        }
        mbar_arrive(&sm.barG[b]);   // G[b] may be overwritten
        if (valid) {
            const __half2 T2 = __float2half2_rn(a.m.Tf);
            s = cdf_finish(a.m, a.m.eta_b, cs, Gprev, Z, tu, delta, in.xi, certain,
                           [&](int cc, float (&pp)[kChunk]) {
                               chunk_prefix_b<NB>(a.m, mu, nbT, xh, T2, gf, cc, pp);
                           });
        }
        s = warp_redraw_fp64<NB>(a.m, valid && !certain, in, s, a.fp64_draws);
        if (valid) {
            a.xout[(size_t)r * a.pitch + c] = (uint8_t)s;
            if (accumulate_after(a, t))
                a.acc[(size_t)r * a.W + c] += (float)s;
        }
        mbar_arrive(&sm.barF[rq]);
    }
    return true;
}

template <int NB, int NT, int KS>
__global__ void __launch_bounds__(kTcThreads, 1) pca_tc_kernel(const SweepArgs a,
                                                               const TcLayout lay, int *err)
{
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (smem_u32(tc_smem) & 1023u) {  // the swizzled operands need 1024-byte alignment
        if (tid == 0)
            atomicExch(err, 2);
        return;
    }
    const TcSmem sm = carve(tc_smem, lay);

    // A and B start zero; B holds K(t, s) for window column kk <-> t = s0 - o + kk
    // and row n <-> s = s0 + n.
    {
        uint4 *z = reinterpret_cast<uint4 *>(tc_smem);
        const int n16 = (2 * sm.a_bytes + lay.b_slabs * kBSlab) / 16;
        for (int i = tid; i < n16; i += kTcThreads)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (int i = tid; i < kLabelTile * lay.kw; i += kTcThreads) {
        const int n = i / lay.kw;
        const int kk = i - n * lay.kw;
        const int v = max(a.m.T - abs(kk - lay.o - n), 0);
        *reinterpret_cast<__half *>(sm.B + sw128_offset(n, kk, kBSlab)) = __int2half_rn(v);
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.barA[b], kLoadThreads);
            mbar_init(&sm.barG[b], kSelThreads);
            for (int h = 0; h < kP1Parts; ++h) {
                mbar_init(&sm.barM[b * kP1Parts + h], 1);
                mbar_init(&sm.barP[b * kP1Parts + h], kSites);
            }
        }
        for (int k = 0; k < kRing; ++k) {
            mbar_init(&sm.barS[k], kLoadThreads);
            mbar_init(&sm.barF[k], kSelThreads);
        }
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(sm.tmem_slot, (uint32_t)(2 * lay.tmem_cols));
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *sm.tmem_slot;

    const int tiles_x = (a.W + 31) >> 5;
    const int ntiles = tiles_x * ((a.H + kTileRows - 1) / kTileRows);
    const int n_my = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                                              : 0;
    bool ok;
    if (warp < kP1Warp0)
        ok = load_role<NB>(a, lay, sm, n_my, tiles_x);
    else if (warp < kSelWarp0)
        ok = pass1_role(a, lay, sm, tmem, n_my, tiles_x);
    else if (warp < kMmaWarp)
        ok = select_role<NB>(a, lay, sm, n_my, tiles_x);
    else
        ok = mma_role<NT, KS>(lay, sm, tmem, n_my);
    if (!ok && (tid & 31) == 0)
        atomicExch(err, 1);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, (uint32_t)(2 * lay.tmem_cols));
    }
}

// Per-(model shape, device) launch configuration.
struct TcConfig {
    int L = -1, T = -1, nbhd = -1, device = -1;
    TcLayout lay{};
    int grid = 0;
};

// The issue loop is unrolled for the shape of L in (192, 256] with T <= 33
// (4 label tiles, K window 128); other shapes use the runtime loop.
bool fixed_shape(const TcLayout &lay)
{
    return lay.nt == 4 && lay.kw == 128;
}

template <int NB, int NT, int KS>
cudaError_t launch_tc_t(const SweepArgs &a, const TcLayout &lay, int grid, int *err,
                        cudaStream_t st)
{
    pca_tc_kernel<NB, NT, KS><<<grid, kTcThreads, lay.smem, st>>>(a, lay, err);
    return cudaGetLastError();
}

template <int NB>
cudaError_t launch_tc(const SweepArgs &a, const TcLayout &lay, int grid, int *err,
                      cudaStream_t st)
{
    return fixed_shape(lay) ? launch_tc_t<NB, 4, 8>(a, lay, grid, err, st)
                            : launch_tc_t<NB, 0, 0>(a, lay, grid, err, st);
}

template <int NB, int NT, int KS>
cudaError_t set_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(pca_tc_kernel<NB, NT, KS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pca_tc_kernel<NB, NT, KS>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int NB>
cudaError_t configure(TcConfig &cfg)
{
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 64 && !attr_set[dev]) {
        e = set_attributes<NB, 4, 8>();
        if (e == cudaSuccess)
            e = set_attributes<NB, 0, 0>();
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    int per_sm = 0;
    e = fixed_shape(cfg.lay)
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pca_tc_kernel<NB, 4, 8>,
                                                            kTcThreads, cfg.lay.smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pca_tc_kernel<NB, 0, 0>,
                                                            kTcThreads, cfg.lay.smem);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1 || per_sm * 2 * cfg.lay.tmem_cols > kTmemCols)
        return cudaErrorInvalidConfiguration;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    cfg.grid = sms * per_sm;
    cfg.device = dev;
    return cudaSuccess;
}

}  // namespace

bool pca_tc_eligible(const DevModel &m)
{
    if (m.L < kTcMinLabels || m.L > 256 || m.T > kTcMaxT || m.norm != 0)
        return false;
    return tc_layout(m.L, m.T).smem <= kSmemMax;
}

cudaError_t launch_pca_tc(const SweepArgs &a, int *err, cudaStream_t st)
{
    if (!pca_tc_eligible(a.m))
        return cudaErrorInvalidValue;
    thread_local TcConfig cfg;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (cfg.L != a.m.L || cfg.T != a.m.T || cfg.nbhd != a.m.nbhd || cfg.device != dev) {
        cfg.L = a.m.L;
        cfg.T = a.m.T;
        cfg.nbhd = a.m.nbhd;
        cfg.lay = tc_layout(a.m.L, a.m.T);
        e = a.m.nbhd == 8 ? configure<8>(cfg) : configure<4>(cfg);
        if (e != cudaSuccess) {
            cfg.L = -1;
            return e;
        }
    }
    const int tiles = ((a.W + 31) / 32) * ((a.H + kTileRows - 1) / kTileRows);
    const int grid = tiles < cfg.grid ? tiles : cfg.grid;
    if (grid <= 0)
        return cudaSuccess;
    return a.m.nbhd == 8 ? launch_tc<8>(a, cfg.lay, grid, err, st)
                         : launch_tc<4>(a, cfg.lay, grid, err, st);
}

}  // namespace pcad
