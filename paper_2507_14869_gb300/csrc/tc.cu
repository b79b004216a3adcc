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
// Per tile of 128 sites: each thread (site) writes its histogram row into
// the A operand (shared memory, K-major, 128-byte swizzle) -- clearing the
// previous tile's entries first --, one thread issues the MMAs and commits
// them to an mbarrier, then each thread reads its own row of the accumulator
// (tcgen05.ld, 32 labels per load) and runs exponent, exp2 and the chunked
// CDF on the CUDA cores.  The kernel is persistent (grid = SMs x resident
// CTAs, tiles strided over the grid); two CTAs per SM overlap one's MMAs
// with the other's CDF work.  The draw is the certified FP32 inverse CDF of
// the CUDA-core kernel (same uniforms, same selection) with the error bound
// of this formulation; uncertain draws are re-evaluated in FP64 by the warp.
// Every mbarrier wait is bounded: on timeout the kernel records an error
// flag, waits once more (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_fp16.h>

#include "async_ptx.cuh"
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kTcRows = 4;                    // tile rows; 32 columns per row
constexpr int kTcThreads = 32 * kTcRows;      // = MMA M: one site per thread and TMEM lane
constexpr int kLabelTile = 64;                // MMA N
constexpr int kASlab = kTcThreads * 128;      // bytes of a 64-column slab of A (128 rows)
constexpr int kBSlab = kLabelTile * 128;      // bytes of a 64-column slab of B (64 rows)
constexpr long long kTcSpinLimit = 20000000;  // ~1 s of polling
constexpr uint32_t kIdesc = idesc_f16_f32(kTcThreads, kLabelTile);
constexpr int kSmemPerSM = 233472;            // shared memory of one SM (228 KB)
constexpr int kSmemReserved = 1024;           // reserved per resident CTA
constexpr int kTmemCols = 512;

// Shape of one model's operands (host-computed).
struct TcLayout {
    int o;           // histogram padding: multiple of 16, >= T - 1
    int kw;          // K window of one label tile: 64 + 2o
    int nt;          // label tiles
    int a_slabs;     // 64-column slabs of A (nt * 64 + 2o columns)
    int b_slabs;     // 64-column slabs of B (kw columns)
    int tmem_cols;   // accumulator columns (power of two >= nt * 64)
    int nc;          // 8-label chunks, ceil(L / 8)
    int ng;          // 32-label groups, ceil(L / 32)
    int smem;        // dynamic shared memory bytes
};

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
    t.smem = t.a_slabs * kASlab + t.b_slabs * kBSlab + t.nc * kTcThreads * 4 + 16;
    // no more resident CTAs than TMEM can hold: pad the shared memory request
    const int max_ctas = kTmemCols / t.tmem_cols;
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
// as the chunk prefix sums.  MASK zeroes labels >= L.
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
            Gcol[c * kTcThreads] = G;
    }
}

template <int NB>
__global__ void __launch_bounds__(kTcThreads) pca_tc_kernel(const SweepArgs a, const TcLayout lay,
                                                            int *err)
{
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t *A = tc_smem;
    uint8_t *B = A + lay.a_slabs * kASlab;
    float *Gs = reinterpret_cast<float *>(B + lay.b_slabs * kBSlab);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Gs + lay.nc * kTcThreads);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    if (smem_u32(tc_smem) & 1023u) {  // the swizzled operands need 1024-byte alignment
        if (tid == 0)
            atomicExch(err, 2);
        return;
    }

    // A and B start zero; B holds K(t, s) for window column kk <-> t = s0 - o + kk
    // and row n <-> s = s0 + n.
    {
        uint4 *z = reinterpret_cast<uint4 *>(A);
        const int n16 = (lay.a_slabs * kASlab + lay.b_slabs * kBSlab) / 16;
        for (int i = tid; i < n16; i += kTcThreads)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (int i = tid; i < kLabelTile * lay.kw; i += kTcThreads) {
        const int n = i / lay.kw;
        const int kk = i - n * lay.kw;
        const int v = max(a.m.T - abs(kk - lay.o - n), 0);
        *reinterpret_cast<__half *>(B + sw128_offset(n, kk, kBSlab)) = __int2half_rn(v);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, (uint32_t)lay.tmem_cols);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int tiles_x = (a.W + 31) >> 5;
    const int ntiles = tiles_x * ((a.H + kTcRows - 1) / kTcRows);
    const uint32_t t = sweep_index(a);
    const float mu = -a.m.gam;
    const float nbT = (float)(NB * a.m.T);
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float *Gcol = Gs + tid;
    uint32_t prev[NB];  // A offsets this thread set for the previous tile (~0u: none)
#pragma unroll
    for (int j = 0; j < NB; ++j)
        prev[j] = ~0u;
    uint32_t phase = 0;
    bool failed = false;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r = (tile / tiles_x) * kTcRows + warp;
        const int c = (tile % tiles_x) * 32 + lane;
        const bool valid = r < a.H && c < a.W;
        SiteIn<NB> in{};
        if (valid)
            load_site<NB>(a, a.xin, r, c, kTagPCA, t, in);

        // this site's histogram row of A
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (prev[j] != ~0u)
                *reinterpret_cast<__half *>(A + prev[j]) = __ushort_as_half((unsigned short)0);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            prev[j] = ~0u;
            if (valid && in.xni[j] < kMissingLabelI) {
                const uint32_t off = sw128_offset(tid, in.xni[j] + lay.o, kASlab);
                __half *h = reinterpret_cast<__half *>(A + off);
                *h = __hadd(*h, __ushort_as_half((unsigned short)0x3C00));  // + 1
                prev[j] = off;
            }
        }
        fence_async_smem();
        __syncthreads();

        if (tid == 0) {
            tc_fence_after_sync();
            const uint32_t a0 = smem_u32(A);
            const uint32_t b0 = smem_u32(B);
            const int ksteps = lay.kw / 16;
            for (int lt = 0; lt < lay.nt; ++lt)
                for (int ks = 0; ks < ksteps; ++ks) {
                    const int kp = lt * kLabelTile + ks * 16;
                    const int kb = ks * 16;
                    umma_f16_ss(tmem + (uint32_t)(lt * kLabelTile),
                                sw128_kmajor_desc(a0 + (kp >> 6) * kASlab + (kp & 63) * 2),
                                sw128_kmajor_desc(b0 + (kb >> 6) * kBSlab + (kb & 63) * 2),
                                kIdesc, ks > 0 ? 1u : 0u);
                }
            umma_commit(bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase, kTcSpinLimit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after_sync();

        // pass 1: chunk prefix sums of the inertia-free weights
        const float gf = (float)in.g;
        float G = 0.0f, comp = 0.0f;
#pragma unroll 1
        for (int grp = 0; grp < lay.ng; ++grp) {
            uint32_t pb[32];
            tmem_ld32(trow + (uint32_t)(grp * 32), pb);
            tmem_wait_ld(pb);
            if ((grp + 1) * 32 > a.m.L)
                group_pass<true>(a.m, mu, gf, grp, pb, lay.nc, Gcol, G, comp);
            else
                group_pass<false>(a.m, mu, gf, grp, pb, lay.nc, Gcol, G, comp);
        }
        tc_fence_before_sync();

        // inertia, selection, pass 2 on the CUDA cores
        int s = 0;
        bool certain = true;
        if (valid) {
            float xn[NB];
            __half2 xh[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                xn[j] = (float)in.xni[j];
                xh[j] = __float2half2_rn(xn[j]);
            }
            const __half2 T2 = __float2half2_rn(a.m.Tf);
            float delta = 0.0f;
            if (a.m.em1 != 0.0f)
                delta = __fmul_rn(single_wb<NB>(a.m, mu, nbT, xn, gf, in.xi), a.m.em1);
            s = cdf_select(a.m, a.m.eta_b, Gcol, kTcThreads, lay.nc, G, delta, in.xi, in.ub,
                           certain, [&](int cs, float (&p)[kChunk]) {
                               chunk_prefix_b<NB>(a.m, mu, nbT, xh, T2, gf, cs, p);
                           });
        }
        s = warp_redraw_fp64<NB>(a.m, valid && !certain, in, s, a.fp64_draws);
        if (valid) {
            a.xout[(size_t)r * a.pitch + c] = (uint8_t)s;
            if (accumulate_after(a, t))
                a.acc[(size_t)r * a.W + c] += (float)s;
        }
    }

    if (failed) {
        if (tid == 0)
            atomicExch(err, 1);
        mbar_wait_bounded(bar, phase, kTcSpinLimit);  // let the MMAs in flight finish
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, (uint32_t)lay.tmem_cols);
    }
}

// Per-(model shape) launch configuration.
struct TcConfig {
    int L = -1, T = -1, nbhd = -1, device = -1;
    TcLayout lay{};
    int grid = 0;
};

template <int NB>
cudaError_t launch_tc(const SweepArgs &a, const TcLayout &lay, int grid, int *err,
                      cudaStream_t st)
{
    pca_tc_kernel<NB><<<grid, kTcThreads, lay.smem, st>>>(a, lay, err);
    return cudaGetLastError();
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
        e = cudaFuncSetAttribute(pca_tc_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemPerSM - kSmemReserved);
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pca_tc_kernel<NB>, kTcThreads,
                                                      cfg.lay.smem);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1 || per_sm * cfg.lay.tmem_cols > kTmemCols)
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
    if (m.L < kTcMinLabels || m.T > kTcMaxT)
        return false;
    const TcLayout lay = tc_layout(m.L, m.T);
    return lay.smem <= kSmemPerSM - kSmemReserved;
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
    const int tiles = ((a.W + 31) / 32) * ((a.H + kTcRows - 1) / kTcRows);
    const int grid = tiles < cfg.grid ? tiles : cfg.grid;
    if (grid <= 0)
        return cudaSuccess;
    return a.m.nbhd == 8 ? launch_tc<8>(a, cfg.lay, grid, err, st)
                         : launch_tc<4>(a, cfg.lay, grid, err, st);
}

}  // namespace pcad
