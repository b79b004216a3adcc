// Lazy-PCA sweep for small label counts (3 <= L <= 16) on the CUDA cores
// (Section 5.2, Eq. posterior_pca_transition_matrix).
//
// With few labels the per-label work of the general kernel (4 neighbour
// terms per label, chunked two-pass CDF) is dominated by fixed costs.  Here:
//
//   * Prior sums from a pair table.  P(s) = sum_j min(|s - x_j|, T) splits
//     into pairs of neighbours (up + down, left + right, and the two
//     diagonal pairs for the 8-neighbourhood).  For every pair of labels
//     (a, b), a, b in [0, 16] with 16 standing for a neighbour outside the
//     image, the table holds min(|s - a|, T) + min(|s - b|, T) for s = 0..15
//     as 16 bytes (a missing neighbour contributes 0: its term is the same
//     for every s and cancels in the normalisation).  One 16-byte shared-
//     memory read per pair and four integer adds give the exact P(s) of all
//     16 labels, four per 32-bit word (every byte <= 120, no carries).
//   * Weights by the formula of the general kernel, w(s) =
//     2^fl(alpha q + fl(gam P)), q = (g - s)^2 and P exact integers, two
//     labels per packed FP32x2 instruction (every lane rounds as the scalar
//     operation).  A byte of P becomes an exact float by placing it in the
//     mantissa of 2^23 and subtracting 2^23.  Chains (whose observations are
//     checked against L at creation) take fl(alpha q) from a 16 x 16 table in
//     shared memory instead: one FFMA per label, fl(gam P + fl(alpha q)),
//     within the same 3u |v| exponent bound; batches and the server keep the
//     arithmetic form.  (Products of two table
//     factors per label measured slower: the per-lane table reads conflict
//     in shared memory, while the exponential unit has room.)
//   * Inverse CDF over chunks of 4 labels: in-chunk prefix sums (3
//     roundings), chunk prefix (3 more), the inertia correction delta =
//     w(x_i)(e^lambda - 1) (w(x_i) read back from the weights in shared
//     memory) joined once to the chunk prefix, one join per probed label:
//     every C_k within 8u and Z within 7u of exact, inside the 22u summation
//     budget of the per-site certified margin (valid because gam <= 0 and
//     alpha <= 0 keep both exponent terms non-positive).  The chunk, then the
//     label in it, are found by comparisons; draws within the margin of a CDF
//     boundary are re-drawn by the warp in FP64.
//
// Persistent blocks of 128 threads take tiles of 16 x 32 sites in a
// grid-stride loop; a thread updates the 4 sites of its column in rows
// w, w + 4, w + 8, w + 12 of the tile (w its warp).  Each block copies the
// pair table (4.6 KB) into shared memory once.  Per tile, the block stages
// the tile's labels with a one-site halo as table codes (aligned 32-bit
// loads, one barrier), and each warp computes the uniforms of its own 4 rows
// (one Philox call per 4 sites, one per lane).  Images of 2^23 sites and
// more take the same draw on TMA-loaded tiles instead (pca_small_tma_kernel
// below: no per-thread staging, the next tile's copy in flight).
#include "async_ptx.cuh"
#include "small_draw.cuh"

namespace pcad {

namespace {

using namespace sld;

constexpr int kBX = 32;
constexpr int kWarps = 4;
constexpr int kThreads = kBX * kWarps;
constexpr int kSPT = 4;                          // sites per thread (rows w + 4 i)
constexpr int kTileR = kWarps * kSPT;            // 16 rows per tile
constexpr int kCodeCols = kBX + 8;               // columns c0 - 4 .. c0 + 35
constexpr int kCodeRows = kTileR + 2;            // rows r0 - 1 .. r0 + 16
constexpr int kCodeWords = kCodeRows * kCodeCols / 4;

__global__ void ptab_kernel(int T, uint32_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPtabWords)
        return;
    const int e = i >> 2, w = i & 3;
    const int a = e / kCodes, b = e - (e / kCodes) * kCodes;
    uint32_t word = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int s = 4 * w + k;
        const int da = a == 16 ? 0 : min(abs(s - a), T);
        const int db = b == 16 ? 0 : min(abs(s - b), T);
        word |= (uint32_t)(da + db) << (8 * k);
    }
    out[i] = word;
}

// planes: a.xin -> a.xout, or (par_from_t) x0 / x1 holding the states of
// even / odd sweep indices; budget (optional): sweeps with index >= *budget
// are skipped (a chain of a batch or of the server).
template <int LMAX, int NB, bool MASK, bool AQ>
__global__ void __launch_bounds__(kThreads) pca_small_kernel(const SweepArgs a, int tiles_x,
                                                             int ntiles, uint8_t *x0, uint8_t *x1,
                                                             int par_from_t,
                                                             const uint32_t *budget)
{
    __shared__ __align__(16) uint32_t pt[kPtabWords];
    __shared__ __align__(16) uint32_t U_s[kWarps * kSPT * kBX];
    __shared__ __align__(16) uint32_t codes[kCodeWords];
    __shared__ __align__(16) float pre_s[kThreads * kPrefixStride];
    __shared__ __align__(16) float aq_s[AQ ? 16 * kAqStride : 4];
    const int lane = (int)threadIdx.x, wp = (int)threadIdx.y;
    const int tid = wp * kBX + lane;
    for (int i = tid; i < kPtabWords / 4; i += kThreads)
        reinterpret_cast<uint4 *>(pt)[i] = __ldg(reinterpret_cast<const uint4 *>(a.m.ptab) + i);
    if (AQ)   // ordered before use by the tile loop's first barrier
        fill_aq(a.m, aq_s, tid, kThreads);
    const uint32_t t = sweep_index(a);
    if (budget && t >= *budget)
        return;   // the whole launch: before any barrier
    const uint8_t *xin = par_from_t ? ((t & 1u) ? x1 : x0) : a.xin;
    uint8_t *xout = par_from_t ? ((t & 1u) ? x0 : x1) : a.xout;
    const bool acc_on = accumulate_after(a, t);
    const uint8_t *cb = reinterpret_cast<const uint8_t *>(codes);
    float *pre = pre_s + tid * kPrefixStride;
    uint32_t *Uw = U_s + wp * kSPT * kBX;
    const uint32_t key0 = (uint32_t)(a.seed & 0xFFFFFFFFull), key1 = (uint32_t)(a.seed >> 32);
    const uint32_t ctr3 = (kTagPCA << 24) | (a.chain & 0xFFFFFFu);
    // tiles in a grid-stride loop, walked as (row, column) without division
    const int step_y = (int)gridDim.x / tiles_x, step_x = (int)gridDim.x - step_y * tiles_x;
    int ty = (int)blockIdx.x / tiles_x, tx = (int)blockIdx.x - ty * tiles_x;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = ty * kTileR, c0 = tx * kBX;
        const int c = c0 + lane;
        // this thread's observations and accumulators, issued early
        int g[kSPT];
        float acc_old[kSPT];
#pragma unroll
        for (int i = 0; i < kSPT; ++i) {
            const int r = r0 + wp + kWarps * i;
            g[i] = 0;
            acc_old[i] = 0.0f;
            if (r < a.H && c < a.W) {
                g[i] = a.g[(size_t)r * a.pitch + c];
                if (acc_on)
                    acc_old[i] = a.acc[(size_t)r * a.W + c];
            }
        }
        __syncthreads();   // tables in place; the previous tile's codes are read
        // the tile's label codes, one aligned word per thread and round
        for (int i = tid; i < kCodeWords; i += kThreads) {
            const int wr = i / (kCodeCols / 4), wc = i - wr * (kCodeCols / 4);
            const int gr = r0 - 1 + wr, gc = c0 - 4 + 4 * wc;
            uint32_t word = 0x10101010u;
            if (gr >= 0 && gr < a.H && gc >= 0 && gc < a.W) {
                word = *reinterpret_cast<const uint32_t *>(xin + (size_t)gr * a.pitch + gc);
                if (gc + 3 >= a.W) {   // the image's right edge inside this word
                    const uint32_t mask = (1u << (8 * (a.W - gc))) - 1u;
                    word = (word & mask) | (0x10101010u & ~mask);
                }
            }
            codes[i] = word;
        }
        // this warp's uniforms: rows wp + 4 i, one Philox call per lane
        {
            const int i = lane >> 3, q = lane & 7;
            uint32_t o0, o1, o2, o3;
            philox4x32_10((uint32_t)((c0 >> 2) + q), (uint32_t)(r0 + wp + kWarps * i + a.row_off),
                          t, ctr3, key0, key1, o0, o1, o2, o3);
            reinterpret_cast<uint4 *>(Uw)[lane] = make_uint4(o0 >> 8, o1 >> 8, o2 >> 8, o3 >> 8);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kSPT; ++i) {
            const int lr = wp + kWarps * i;
            const int r = r0 + lr;
            const bool valid = r < a.H && c < a.W;
            const uint8_t *me = cb + (1 + lr) * kCodeCols + 4 + lane;
            int nc[NB];
            nc[0] = me[-kCodeCols];
            nc[1] = me[kCodeCols];
            nc[2] = me[-1];
            nc[3] = me[1];
            if constexpr (NB == 8) {
                nc[4] = me[-kCodeCols - 1];
                nc[5] = me[-kCodeCols + 1];
                nc[6] = me[kCodeCols - 1];
                nc[7] = me[kCodeCols + 1];
            }
            const int xi = me[0];
            const uint32_t ub = Uw[i * kBX + lane];
            int s = 0;
            bool certain = true;
            if (valid)
                s = draw_small<LMAX, NB, MASK, AQ>(a.m, pt, nc, g[i], xi, ub, pre, certain, aq_s);
            const bool need = valid && !certain;
            if (__any_sync(0xFFFFFFFFu, need)) {
                SiteIn<NB> in{};
                in.g = g[i];
                in.xi = xi;
                in.ub = ub;
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    in.xni[j] = nc[j] == 16 ? kMissingLabelI : nc[j];
                s = warp_redraw_fp64<NB>(a.m, need, in, s, a.fp64_draws);
            }
            if (valid) {
                xout[(size_t)r * a.pitch + c] = (uint8_t)s;
                if (acc_on)
                    a.acc[(size_t)r * a.W + c] = acc_old[i] + (float)s;
            }
        }
        tx += step_x;
        ty += step_y;
        if (tx >= tiles_x) {
            tx -= tiles_x;
            ++ty;
        }
    }
}

// ---------------------------------------------------------------- tile form
// Large images: persistent blocks of 256 threads over output tiles of
// 64 x 46 sites, each loaded by TMA as the 96 x 48 box of the plane maps
// (labels and observation, columns x0 - 16 .. x0 + 79, rows y0 - 1 ..
// y0 + 46: a one-site halo, the column start 16-byte aligned).  Two box
// buffers: while the block draws one tile, the next tile's copies are in
// flight (one mbarrier per buffer, bounded waits, one block barrier per
// tile); the tables are loaded once per block.  A thread takes groups of 4
// sites of a row (one Philox call each): neighbour codes from the box (no
// bounds tests for tiles whose halo lies inside the image), the 4 labels
// stored as one 32-bit word and the accumulator read-modify-written as one
// float4, loaded before the draws.  The data term comes from the table
// (chains: g < L checked).
constexpr int kTmThreads = 256;
constexpr int kTmBoxW = 96, kTmBoxH = 48;   // the box of encode_plane_map
constexpr int kTmOutW = 64, kTmOutH = kTmBoxH - 2;
constexpr int kTmColOff = 16;
constexpr int kTmPlane = kTmBoxW * kTmBoxH;
constexpr int kTmQuadsPerRow = kTmOutW / 4;
constexpr int kTmQuads = kTmQuadsPerRow * kTmOutH;
constexpr int kTmRounds = (kTmQuads + kTmThreads - 1) / kTmThreads;

// One tile from box buffers xb, gb: INTERIOR when the tile and its halo lie
// inside the image.
template <int LMAX, int NB, bool MASK, bool INTERIOR>
__device__ __forceinline__ void small_tma_tile(const SweepArgs &a, const uint8_t *xb,
                                               const uint8_t *gb, const uint32_t *pt,
                                               const float *aq, float *pre, int x0, int y0,
                                               uint32_t t, bool acc_on, bool acc_vec, int tid)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    constexpr int dr[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
    constexpr int dc[8] = {0, 0, -1, 1, -1, 1, -1, 1};
    const uint32_t key0 = (uint32_t)(a.seed & 0xFFFFFFFFull), key1 = (uint32_t)(a.seed >> 32);
    const uint32_t ctr3 = (kTagPCA << 24) | (a.chain & 0xFFFFFFu);
    const int H = a.H, W = a.W;
#pragma unroll 1
    for (int rd = 0; rd < kTmRounds; ++rd) {
        const int qd = rd * kTmThreads + tid;
        const bool qv = qd < kTmQuads;
        const int qr = qv ? qd / kTmQuadsPerRow : 0;
        const int qc = qv ? qd - qr * kTmQuadsPerRow : 0;
        const int lr = 1 + qr, lc0 = kTmColOff + 4 * qc;   // box coordinates
        const int gr = y0 + qr, gc0 = x0 + 4 * qc;         // image coordinates
        const bool rowv = qv && (INTERIOR || gr < H);
        const bool full = rowv && (INTERIOR || gc0 + 3 < W);
        const size_t oa = (size_t)gr * W + gc0;
        float4 acc4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (acc_on && full && acc_vec)
            acc4 = *reinterpret_cast<const float4 *>(a.acc + oa);
        uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        if (rowv && gc0 < W)
            philox4x32_10((uint32_t)gc0 >> 2, (uint32_t)(gr + a.row_off), t, ctr3, key0, key1, w0,
                          w1, w2, w3);
        uint32_t packed = 0u;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int lc = lc0 + q, gc = gc0 + q;
            const bool valid = rowv && (INTERIOR || gc < W);
            const uint32_t ub = (q == 0 ? w0 : (q == 1 ? w1 : (q == 2 ? w2 : w3))) >> 8;
            const uint8_t *me = xb + lr * kTmBoxW + lc;
            int nc[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const bool inside = INTERIOR || ((unsigned)(gr + dr[j]) < (unsigned)H &&
                                                 (unsigned)(gc + dc[j]) < (unsigned)W);
                nc[j] = inside ? (int)me[dr[j] * kTmBoxW + dc[j]] : 16;
            }
            const int xi = me[0];
            const int gv = gb[lr * kTmBoxW + lc];
            int sl = 0;
            bool certain = true;
            if (valid)
                sl = draw_small<LMAX, NB, MASK, true>(a.m, pt, nc, gv, xi, ub, pre, certain, aq);
            const bool need = valid && !certain;
            if (__any_sync(kFull, need)) {
                SiteIn<NB> in{};
                in.g = gv;
                in.xi = xi;
                in.ub = ub;
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    in.xni[j] = nc[j] == 16 ? kMissingLabelI : nc[j];
                sl = warp_redraw_fp64<NB>(a.m, need, in, sl, a.fp64_draws);
            }
            packed |= (uint32_t)sl << (8 * q);
        }
        if (full) {
            *reinterpret_cast<uint32_t *>(a.xout + (size_t)gr * a.pitch + gc0) = packed;
            if (acc_on) {
                const float l0 = (float)(packed & 0xFFu), l1 = (float)((packed >> 8) & 0xFFu),
                            l2 = (float)((packed >> 16) & 0xFFu), l3 = (float)(packed >> 24);
                if (acc_vec) {
                    *reinterpret_cast<float4 *>(a.acc + oa) =
                        make_float4(acc4.x + l0, acc4.y + l1, acc4.z + l2, acc4.w + l3);
                } else {
                    a.acc[oa] += l0;
                    a.acc[oa + 1] += l1;
                    a.acc[oa + 2] += l2;
                    a.acc[oa + 3] += l3;
                }
            }
        } else if (rowv) {
            for (int q = 0; q < 4 && gc0 + q < W; ++q) {
                const uint32_t sl = (packed >> (8 * q)) & 0xFFu;
                a.xout[(size_t)gr * a.pitch + gc0 + q] = (uint8_t)sl;
                if (acc_on)
                    a.acc[oa + q] += (float)sl;
            }
        }
    }
}

template <int LMAX, int NB, bool MASK>
__global__ void __launch_bounds__(kTmThreads)
    pca_small_tma_kernel(const __grid_constant__ CUtensorMap xmap,
                         const __grid_constant__ CUtensorMap gmap, const SweepArgs a, int tiles_x,
                         int ntiles, int acc_vec, int *err)
{
    __shared__ __align__(128) uint8_t xs[2][kTmPlane];
    __shared__ __align__(128) uint8_t gs[2][kTmPlane];
    __shared__ __align__(16) uint32_t pt[kPtabWords];
    __shared__ __align__(16) float pre_s[kTmThreads * kPrefixStride];
    __shared__ __align__(16) float aq_s[16 * kAqStride];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = (int)threadIdx.x;
    for (int i = tid; i < kPtabWords / 4; i += kTmThreads)
        reinterpret_cast<uint4 *>(pt)[i] = __ldg(reinterpret_cast<const uint4 *>(a.m.ptab) + i);
    fill_aq(a.m, aq_s, tid, kTmThreads);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    const uint32_t t = sweep_index(a);
    const bool acc_on = accumulate_after(a, t);
    const long long limit = wait_limit(a.wait_ns);
    auto issue = [&](int tile, int b) {
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        mbar_expect_tx(&bar[b], 2u * kTmPlane);
        tma_load_2d(xs[b], &xmap, tx * kTmOutW - kTmColOff, ty * kTmOutH - 1, &bar[b]);
        tma_load_2d(gs[b], &gmap, tx * kTmOutW - kTmColOff, ty * kTmOutH - 1, &bar[b]);
    };
    int tile = (int)blockIdx.x;
    if (tid == 0 && tile < ntiles)
        issue(tile, 0);
    uint32_t phase0 = 0u, phase1 = 0u;
    float *pre = pre_s + tid * kPrefixStride;
    for (int it = 0; tile < ntiles; ++it, tile += (int)gridDim.x) {
        const int b = it & 1;
        const int next = tile + (int)gridDim.x;
        // buffer b ^ 1 was released by the barrier that ended the last tile
        if (tid == 0 && next < ntiles) {
            fence_async_smem();   // order those reads before the copy's writes
            issue(next, b ^ 1);
        }
        const uint32_t ph = b ? phase1 : phase0;
        const bool ok = mbar_wait_timed(&bar[b], ph, limit);
        if (!__syncthreads_and(ok)) {
            // record, then wait (bounded) for the copies still in flight
            // before the block's shared memory is released
            if (tid == 0)
                atomicExch(err, 1);
            mbar_wait_timed(&bar[b], ph, limit);
            if (next < ntiles)
                mbar_wait_timed(&bar[b ^ 1], b ? phase0 : phase1, limit);
            return;
        }
        if (b)
            phase1 ^= 1u;
        else
            phase0 ^= 1u;
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int x0 = tx * kTmOutW, y0 = ty * kTmOutH;
        const bool interior = x0 >= 1 && y0 >= 1 && x0 + kTmOutW < a.W && y0 + kTmOutH < a.H;
        if (interior)
            small_tma_tile<LMAX, NB, MASK, true>(a, xs[b], gs[b], pt, aq_s, pre, x0, y0, t,
                                                 acc_on, acc_vec != 0, tid);
        else
            small_tma_tile<LMAX, NB, MASK, false>(a, xs[b], gs[b], pt, aq_s, pre, x0, y0, t,
                                                  acc_on, acc_vec != 0, tid);
        __syncthreads();   // buffer b is read: the load after next may overwrite it
    }
}

template <int LMAX, int NB, bool MASK>
cudaError_t launch_small_tma_t(const CUtensorMap &xmap, const CUtensorMap &gmap,
                               const SweepArgs &a, int *err, cudaStream_t st)
{
    static int per_sm[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64)
        return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, pca_small_tma_kernel<LMAX, NB, MASK>, kTmThreads, 0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = n > 0 ? n : 1;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (a.W + kTmOutW - 1) / kTmOutW;
    const long long ntiles = (long long)tiles_x * ((a.H + kTmOutH - 1) / kTmOutH);
    if (ntiles <= 0)
        return cudaSuccess;
    if (ntiles >= (1ll << 31))
        return cudaErrorInvalidValue;
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    const int acc_vec = (a.W % 4 == 0 && (reinterpret_cast<uintptr_t>(a.acc) & 15u) == 0) ? 1 : 0;
    pca_small_tma_kernel<LMAX, NB, MASK><<<grid, kTmThreads, 0, st>>>(xmap, gmap, a, tiles_x,
                                                                      (int)ntiles, acc_vec, err);
    return cudaGetLastError();
}

template <int LMAX, int NB, bool MASK, bool AQ>
cudaError_t launch_small_t(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int par_from_t,
                           const uint32_t *budget, cudaStream_t st)
{
    static int per_sm[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64)
        return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pca_small_kernel<LMAX, NB, MASK, AQ>,
                                                          kThreads, 0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = n > 0 ? n : 1;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (a.W + kBX - 1) / kBX;
    const long long ntiles = (long long)tiles_x * ((a.H + kTileR - 1) / kTileR);
    if (ntiles <= 0)
        return cudaSuccess;
    if (ntiles >= (1ll << 31))
        return cudaErrorInvalidValue;
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    pca_small_kernel<LMAX, NB, MASK, AQ><<<grid, dim3(kBX, kWarps), 0, st>>>(
        a, tiles_x, (int)ntiles, x0, x1, par_from_t, budget);
    return cudaGetLastError();
}

template <int NB, bool AQ>
cudaError_t dispatch_small(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int par_from_t,
                           const uint32_t *budget, cudaStream_t st)
{
    if (a.m.L <= 8)
        return a.m.L == 8 ? launch_small_t<8, NB, false, AQ>(a, x0, x1, par_from_t, budget, st)
                          : launch_small_t<8, NB, true, AQ>(a, x0, x1, par_from_t, budget, st);
    return a.m.L == 16 ? launch_small_t<16, NB, false, AQ>(a, x0, x1, par_from_t, budget, st)
                       : launch_small_t<16, NB, true, AQ>(a, x0, x1, par_from_t, budget, st);
}

}  // namespace

int ptab_words()
{
    return kPtabWords;
}

cudaError_t launch_ptab(int T, uint32_t *out, cudaStream_t st)
{
    ptab_kernel<<<(kPtabWords + 255) / 256, 256, 0, st>>>(T, out);
    return cudaGetLastError();
}

cudaError_t launch_pca_small_tma(const CUtensorMap &xmap, const CUtensorMap &gmap,
                                 const SweepArgs &a, int *err, cudaStream_t st)
{
    if (!pca_small_eligible(a.m))
        return cudaErrorInvalidValue;
    if ((a.pitch & 3) != 0 || (reinterpret_cast<uintptr_t>(a.xout) & 3u) != 0)
        return cudaErrorMisalignedAddress;
    if (a.m.nbhd == 8) {
        if (a.m.L <= 8)
            return a.m.L == 8 ? launch_small_tma_t<8, 8, false>(xmap, gmap, a, err, st)
                              : launch_small_tma_t<8, 8, true>(xmap, gmap, a, err, st);
        return a.m.L == 16 ? launch_small_tma_t<16, 8, false>(xmap, gmap, a, err, st)
                           : launch_small_tma_t<16, 8, true>(xmap, gmap, a, err, st);
    }
    if (a.m.L <= 8)
        return a.m.L == 8 ? launch_small_tma_t<8, 4, false>(xmap, gmap, a, err, st)
                          : launch_small_tma_t<8, 4, true>(xmap, gmap, a, err, st);
    return a.m.L == 16 ? launch_small_tma_t<16, 4, false>(xmap, gmap, a, err, st)
                       : launch_small_tma_t<16, 4, true>(xmap, gmap, a, err, st);
}

bool pca_small_eligible(const DevModel &m)
{
    return m.ptab != nullptr && m.ta64 != nullptr && m.pr64 != nullptr &&
           m.L >= kSmallMinLabels && m.L <= kSmallMaxLabels && m.norm == 0 && m.gam <= 0.0f &&
           m.alpha <= 0.0f && (m.nbhd == 4 || m.nbhd == 8);
}

cudaError_t launch_pca_small(const SweepArgs &a, cudaStream_t st, uint8_t *x0, uint8_t *x1,
                             const uint32_t *budget, bool aq)
{
    if (!pca_small_eligible(a.m))
        return cudaErrorInvalidValue;
    const int par = x0 != nullptr ? 1 : 0;
    // the label tile is staged with aligned 32-bit loads
    const uintptr_t align = par ? (reinterpret_cast<uintptr_t>(x0) | reinterpret_cast<uintptr_t>(x1))
                                : reinterpret_cast<uintptr_t>(a.xin);
    if ((a.pitch & 3) != 0 || (align & 3u) != 0)
        return cudaErrorMisalignedAddress;
    if (aq)
        return a.m.nbhd == 8 ? dispatch_small<8, true>(a, x0, x1, par, budget, st)
                             : dispatch_small<4, true>(a, x0, x1, par, budget, st);
    return a.m.nbhd == 8 ? dispatch_small<8, false>(a, x0, x1, par, budget, st)
                         : dispatch_small<4, false>(a, x0, x1, par, budget, st);
}

}  // namespace pcad
