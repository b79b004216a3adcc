// Temporally blocked lazy-PCA sweeps: k sweeps per HBM round trip.
//
// A block owns an output tile of 64 columns x (48 - 2k) rows.  One thread
// issues two TMA loads (cp.async.bulk.tensor.2d) of a 96 x 48 box of the
// current labels and of the observation -- columns [x0 - 16, x0 + 80), rows
// [y0 - k, y0 + 48 - k), so the column start stays 16-byte aligned and the
// halo holds k sites on every side -- completing on an mbarrier.  The block
// then runs k sweeps in shared memory (ping-pong planes); sweep j recomputes
// the region shrunk by j + 1 sites per side, so after k sweeps the output
// tile is exact.  A site's draw uses the uniform keyed by its global (row,
// col, sweep), so the redundant halo work of neighbouring tiles gives
// identical labels.  Each thread accumulates its own output sites in
// registers after every post-burn-in sweep; labels and the accumulator go
// back to global memory once per k sweeps.  Every mbarrier wait is bounded:
// on timeout the kernel records an error flag and returns.  Models the
// small-label kernel accepts (3 <= L <= 16) draw with its pair table and
// chunked CDF (small_draw.cuh).
#include <cuda.h>

#include "async_ptx.cuh"
#include "small_draw.cuh"

namespace pcad {

namespace {

constexpr int kTbThreads = 256;
constexpr int kBoxW = 96;          // loaded columns
constexpr int kBoxH = 48;          // loaded rows
constexpr int kOutW = 64;          // output columns
constexpr int kColOff = 16;        // output column offset inside the box
constexpr int kPlane = kBoxW * kBoxH;

// Inputs of site (lr, lc) of the box from the shared planes; neighbours
// outside the image are "missing" (label 1024).
template <int NB>
__device__ __forceinline__ void site_from_box(const uint8_t *xp, const uint8_t *gp, int lr, int lc,
                                              int gr, int gc, int H, int W, SiteIn<NB> &in)
{
    constexpr int dr[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
    constexpr int dc[8] = {0, 0, -1, 1, -1, 1, -1, 1};
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int rr = gr + dr[j], cc = gc + dc[j];
        const bool inside = rr >= 0 && rr < H && cc >= 0 && cc < W;
        in.xni[j] = inside ? (int)xp[(lr + dr[j]) * kBoxW + lc + dc[j]] : kMissingLabelI;
    }
    in.xi = xp[lr * kBoxW + lc];
    in.g = gp[lr * kBoxW + lc];
}

// Pair-table codes of site (lr, lc)'s neighbours for the small-label draw:
// the label, or 16 outside the image.
template <int NB>
__device__ __forceinline__ void codes_from_box(const uint8_t *xp, int lr, int lc, int gr, int gc,
                                               int H, int W, int (&nc)[NB])
{
    constexpr int dr[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
    constexpr int dc[8] = {0, 0, -1, 1, -1, 1, -1, 1};
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int rr = gr + dr[j], cc = gc + dc[j];
        const bool inside = rr >= 0 && rr < H && cc >= 0 && cc < W;
        nc[j] = inside ? (int)xp[(lr + dr[j]) * kBoxW + lc + dc[j]] : 16;
    }
}

template <int NC, int NB>
__device__ __forceinline__ int tb_draw(const DevModel &m, bool valid, const SiteIn<NB> &in,
                                       float *Gcol, unsigned long long *fp64)
{
    int s = 0;
    bool certain = true;
    uint32_t dirty = 0xFFFFFFFFu;
    if (NC >= 8)
        dirty = __reduce_or_sync(0xFFFFFFFFu, valid ? dirty_chunks<NB>(in.xni, m.T) : 0u);
    if (valid)
        s = draw_fp32<NC, NB>(m, Gcol, kTbThreads, in, dirty, certain);
    return warp_redraw_fp64<NB>(m, valid && !certain, in, s, fp64);
}

constexpr int kOwnMax = (kOutW * (kBoxH - 2) + kTbThreads - 1) / kTbThreads;   // 12

// SL = 0: the general CUDA-core draw over NC chunks of 8 labels; SL = 8 or
// 16: the small-label draw (labels < SL, MASK when L < SL) with the pair
// table and a weight row per thread in shared memory.
template <int NC, int NB, int SL, bool MASK>
__global__ void __launch_bounds__(kTbThreads)
    pca_tb_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap gmap,
                  const SweepArgs a, int k, int *err)
{
    __shared__ __align__(128) uint8_t xs[2][kPlane];
    __shared__ __align__(128) uint8_t gs[kPlane];
    __shared__ float G_s[SL > 0 ? 1 : NC * kTbThreads];
    __shared__ __align__(16) uint32_t pt[SL > 0 ? sld::kPtabWords : 4];
    __shared__ __align__(16) float pre_s[SL > 0 ? kTbThreads * sld::kPrefixStride : 4];
    __shared__ __align__(16) float aq_s[SL > 0 ? 16 * sld::kAqStride : 4];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    if constexpr (SL > 0) {   // ordered before use by the barrier after the loads
        for (int i = tid; i < sld::kPtabWords / 4; i += kTbThreads)
            reinterpret_cast<uint4 *>(pt)[i] =
                __ldg(reinterpret_cast<const uint4 *>(a.m.ptab) + i);
        sld::fill_aq(a.m, aq_s, tid, kTbThreads);   // chains hold observations g < L <= 16
    }
    const int TH = kBoxH - 2 * k;
    const int x0 = blockIdx.x * kOutW, y0 = blockIdx.y * TH;
    const int bx = x0 - kColOff, by = y0 - k;       // global origin of the box
    const uint32_t t0 = *a.sweep_base + a.sweep_off;

    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bar, 2u * kPlane);
        tma_load_2d(xs[0], &xmap, bx, by, &bar);
        tma_load_2d(gs, &gmap, bx, by, &bar);
    }
    const long long limit = wait_limit(a.wait_ns);
    const bool ok = mbar_wait_timed(&bar, 0u, limit);
    if (!__syncthreads_and(ok)) {
        // the copies may still land: wait for them (bounded again) before the
        // block's shared memory is released
        if (tid == 0)
            atomicExch(err, 1);
        mbar_wait_timed(&bar, 0u, limit);
        return;
    }

    uint32_t accp[(kOwnMax + 1) / 2];   // two 16-bit label sums per register (<= 8 x 255)
#pragma unroll
    for (int q = 0; q < (kOwnMax + 1) / 2; ++q)
        accp[q] = 0u;
    bool any_acc = false;
    const uint32_t key0 = (uint32_t)(a.seed & 0xFFFFFFFFull), key1 = (uint32_t)(a.seed >> 32);
    const uint32_t c3 = (kTagPCA << 24) | (a.chain & 0xFFFFFFu);
    int cur = 0;
    for (int j = 0; j < k; ++j) {
        const uint32_t t = t0 + (uint32_t)j;
        const int r_lo = j + 1, r_hi = kBoxH - j - 1;
        const int c_lo = kColOff - k + j + 1, c_hi = kColOff + kOutW + k - j - 1;
        const int g_lo = c_lo & ~3;
        const int ngroups = (c_hi - g_lo + 3) >> 2;
        const int npairs = (r_hi - r_lo) * ngroups;
        const int iters = (npairs + kTbThreads - 1) / kTbThreads;
        const uint8_t *xp = xs[cur];
        uint8_t *xo = xs[cur ^ 1];
        for (int it = 0; it < iters; ++it) {
            const int pidx = it * kTbThreads + tid;
            const bool pvalid = pidx < npairs;
            const int lr = r_lo + (pvalid ? pidx / ngroups : 0);
            const int lcg = g_lo + 4 * (pvalid ? pidx % ngroups : 0);
            const int gr = by + lr, gc0 = bx + lcg;
            uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
            if (pvalid && gr >= 0 && gr < a.H && gc0 + 3 >= 0 && gc0 < a.W)
                philox4x32_10((uint32_t)gc0 >> 2, (uint32_t)(gr + a.row_off), t, c3, key0, key1,
                              w0, w1, w2, w3);
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int lc = lcg + q, gc = gc0 + q;
                const bool valid = pvalid && lc >= c_lo && lc < c_hi && gr >= 0 && gr < a.H &&
                                   gc >= 0 && gc < a.W;
                const uint32_t w = q == 0 ? w0 : (q == 1 ? w1 : (q == 2 ? w2 : w3));
                int s = 0;
                if constexpr (SL > 0) {
                    int nc[NB];
                    int xi = 0, gv = 0;
                    bool certain = true;
                    if (valid) {
                        codes_from_box<NB>(xp, lr, lc, gr, gc, a.H, a.W, nc);
                        xi = xp[lr * kBoxW + lc];
                        gv = gs[lr * kBoxW + lc];
                        s = sld::draw_small<SL, NB, MASK, true>(
                            a.m, pt, nc, gv, xi, w >> 8, pre_s + tid * sld::kPrefixStride,
                            certain, aq_s);
                    }
                    const bool need = valid && !certain;
                    if (__any_sync(0xFFFFFFFFu, need)) {
                        SiteIn<NB> in{};
                        if (valid) {
                            site_from_box<NB>(xp, gs, lr, lc, gr, gc, a.H, a.W, in);
                            in.ub = w >> 8;
                        }
                        s = warp_redraw_fp64<NB>(a.m, need, in, s, a.fp64_draws);
                    }
                } else {
                    SiteIn<NB> in{};
                    if (valid) {
                        site_from_box<NB>(xp, gs, lr, lc, gr, gc, a.H, a.W, in);
                        in.ub = w >> 8;
                    }
                    s = tb_draw<NC, NB>(a.m, valid, in, G_s + tid, a.fp64_draws);
                }
                if (valid)
                    xo[lr * kBoxW + lc] = (uint8_t)s;
            }
        }
        __syncthreads();
        cur ^= 1;
        if (accumulate_after(a, t)) {
            any_acc = true;
#pragma unroll
            for (int q = 0; q < kOwnMax; ++q) {
                const int o = tid + q * kTbThreads;
                if (o < kOutW * TH)
                    accp[q >> 1] += (uint32_t)xs[cur][(k + o / kOutW) * kBoxW + kColOff + o % kOutW] << (16 * (q & 1));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kOwnMax; ++q) {
        const int o = tid + q * kTbThreads;
        const int gr = y0 + o / kOutW, gc = x0 + o % kOutW;
        if (o < kOutW * TH && gr < a.H && gc < a.W) {
            a.xout[(size_t)gr * a.pitch + gc] = xs[cur][(k + o / kOutW) * kBoxW + kColOff + o % kOutW];
            if (any_acc)
                a.acc[(size_t)gr * a.W + gc] += (float)((accp[q >> 1] >> (16 * (q & 1))) & 0xFFFFu);
        }
    }
}

template <int NB>
cudaError_t dispatch_tb(const CUtensorMap &xm, const CUtensorMap &gm, const SweepArgs &a, int k,
                        int *err, cudaStream_t s)
{
    const dim3 grid((a.W + kOutW - 1) / kOutW, (a.H + (kBoxH - 2 * k) - 1) / (kBoxH - 2 * k));
    if (pca_small_eligible(a.m)) {   // the small-label draw, as the unblocked default
        if (a.m.L <= 8) {
            if (a.m.L == 8)
                pca_tb_kernel<1, NB, 8, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err);
            else
                pca_tb_kernel<1, NB, 8, true><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err);
        } else if (a.m.L == 16) {
            pca_tb_kernel<1, NB, 16, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err);
        } else {
            pca_tb_kernel<1, NB, 16, true><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err);
        }
        return cudaGetLastError();
    }
    switch (chunk_class(a.m.L)) {
    case 1: pca_tb_kernel<1, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 2: pca_tb_kernel<2, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 3: pca_tb_kernel<3, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 4: pca_tb_kernel<4, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 5: pca_tb_kernel<5, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 8: pca_tb_kernel<8, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    case 16: pca_tb_kernel<16, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    default: pca_tb_kernel<32, NB, 0, false><<<grid, kTbThreads, 0, s>>>(xm, gm, a, k, err); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pca_tb(const CUtensorMap &xmap, const CUtensorMap &gmap, const SweepArgs &a,
                          int k, int *err, cudaStream_t s)
{
    if (k < 1 || k > 8)
        return cudaErrorInvalidValue;
    return a.m.nbhd == 8 ? dispatch_tb<8>(xmap, gmap, a, k, err, s)
                         : dispatch_tb<4>(xmap, gmap, a, k, err, s);
}

// Tensor map of one uint8 label plane: H rows of W labels, row stride
// `pitch` bytes (a multiple of 16), box 96 x 48.
bool encode_plane_map(CUtensorMap *map, void *base, int H, int W, int pitch)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = (Encode)p;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace pcad
