// Lazy-PCA sweep with the prior sums on the tensor cores (Section 5.2, Eq.
// posterior_pca_transition_matrix), for truncated-linear priors with many
// labels.
//
// For label s the truncated-linear prior sum is
//   P(s) = sum_j min(|x_j - s|, T) = n T - Pb(s),  Pb(s) = sum_j max(T - |x_j - s|, 0),
// n the number of neighbours inside the image.  n T is the same for every
// label of the site and cancels in the normalisation, so the weights are
// built from Pb: w(s) = 2^(alpha (g - s)^2 + mu Pb(s) + cb), mu = c log2(e),
// with one offset cb = -mu nbhd T for every label (mu > 0) that keeps both
// exponent terms non-positive and the per-site certified margin small.
// Every tent max(T - |x_j - s|, 0) is zero farther than T - 1 from x_j, so
// Pb lives in a window of labels around the neighbours' labels:
//
//   * window: each site takes its own base b = 8 m + T - 1 with
//     m = floor((x_min - T + 1) / 8), x_min the smallest neighbour label, so
//     b <= x_min < b + 8.  Neighbour labels x_j - b in [0, 64) go into a
//     64-bin histogram h (at most NB nonzero counts); the window's labels
//     are s = 8 m + c, c in [0, 128), and
//       Pb(8 m + c) = sum_k h(k) K(k, c),  K(k, c) = max(T - |c - (T - 1) - k|, 0),
//     which covers the whole support of the histogram's tents for T <= 33.
//     One tcgen05.mma chain (M = 128 sites, N = 128 window labels, K = 64
//     bins: four 128 x 128 x 16 steps) computes it; the operands are small
//     integers, exact with FP16 inputs and FP32 accumulation.  K is the same
//     matrix for every site and stays in shared memory.
//   * outliers: neighbours with x_j - b >= 64 (wide neighbourhoods, image
//     edges) add their tents on the CUDA cores in both label ranges.
//   * outside the window Pb is the outliers' part only (zero for most
//     sites): w(s) = 2^(alpha (g - s)^2 + cb), no prior arithmetic; the
//     chunk sums come from a table of (observation, chunk).
//
// The window is chunk-aligned (8 | 8 m), so every label chunk of the draw is
// either a window chunk or an outside chunk of the site.  Pass 1 writes the
// chunk sums in label order into shared memory; they are prefix-summed
// (Kahan) and the certified inverse-CDF selection of the CUDA-core kernel
// runs on them (same uniforms), with pass 2 recomputing the chosen chunk's
// weights from exact prior sums on the CUDA cores (bit-identical: Pb is the
// same integer either way and the weight formula is the same).
//
// CTA: 4 warpgroups (512 threads), one per SM; each group owns one 4 x 32
// tile at a time, its histogram operand (16 KB) and 128 TMEM columns, so
// four tiles are in flight.  A group: loads its sites, writes their
// histogram rows, one thread issues the 4 MMAs and commits them to the
// group's mbarrier; while the tensor core runs, the group reads the
// outside chunks from the table; then it reads the window from TMEM (up
// to 4 x tcgen05.ld of 32 columns; two labels per packed FP32x2
// instruction), selects, re-draws uncertain draws in FP64 with the whole
// group and writes.
//
// The same kernel runs the 4-neighbourhood checkerboard Gibbs sweep (GIBBS):
// items are colour phases over 8 x 32 tiles, updated in place.
//
// Work items (sweep k, tile) are taken in increasing order, sweep-major,
// from an atomic counter; item (k, tile) waits until the 3 x 3 tiles around
// it finished sweep k - 1 (done[] counts finished sweeps per tile; acquire
// loads observe them, a release store publishes), so one
// launch runs many sweeps with no sweep-wide barrier (as the wavefront
// CUDA-core kernel).  Every item waited on was taken earlier by a resident
// group, so the waits end; each wait is bounded anyway (error flag), and
// TMEM is freed before return.
#include <cuda_fp16.h>

#include "async_ptx.cuh"
#include "pcad_internal.h"
#include "tc_math.cuh"

namespace pcad {

namespace {

using namespace tcm;

constexpr int kSites = 128;                 // tile: 4 rows x 32 columns = MMA M = TMEM lanes
constexpr int kTileRows = 4;
constexpr int kGibbsRows = 8;    // Gibbs tiles: 8 x 32 sites, 128 of each colour
constexpr int kGroups = 4;                  // warpgroups per CTA, one tile each
constexpr int kThr = kGroups * kSites;      // 512 threads
constexpr int kWin = 128;                   // window labels = MMA N = TMEM columns per group
constexpr int kBins = 64;                   // histogram bins = MMA K (4 steps of 16)
constexpr int kWinChunks = kWin / kChunk;   // 16
constexpr int kOpBytes = kSites * kBins * 2;   // 16 KB: one operand (128 rows x 128 bytes)
constexpr int kTmemCols = kGroups * kWin;   // 512
constexpr uint32_t kIdesc = idesc_f16_f32(kSites, kWin);
constexpr float kNoLabel = -4096.0f;        // unused outlier slot: its tent is zero everywhere

// Shared memory: B (16 KB), A[4] (64 KB), G [chunk][thread] floats, the
// outside-chunk sums [chunk][observation], then mbarriers, the groups' work
// items and the TMEM base.
constexpr int kOffB = 0;
constexpr int kOffA = kOpBytes;
constexpr int kOffG = kOffA + kGroups * kOpBytes;

// After G (and the one-chain table): mbarriers, work items and the TMEM
// base (64 bytes), then for batched chains the staged items of each group.
constexpr int kTcCtlBytes = 64;
// Per group: the sites' inputs for the group's FP64 re-draws (g, xi, ub,
// the neighbour labels), the warps' need masks, partial sums and result.
constexpr int kRedrawInts = 3 + 8;
constexpr int kRedrawBytes = kGroups * (kSites * kRedrawInts * 4 + 4 * 4 + 4 * 8 + 16);
constexpr int kTcStageBytes = 2 * kGroups * ((int)sizeof(SweepArgs) + 4 + 4);

// One chain keeps the outside sums as a [chunk][observation] table (row
// stride 257 against bank conflicts), rounded to an even float count.
constexpr int kTabRow = 257;
__host__ __device__ constexpr int tab2_floats(int nc)
{
    return (nc * kTabRow + 1) & ~1;
}

// G, then the tables (one chain: the 2-D table; batched chains: two 1-D
// tables per group), control, stage.
__host__ __device__ constexpr int tc_smem_bytes(int nc, bool batch)
{
    return kOffG + nc * kThr * 4 + (batch ? 2 * kGroups * kTabF : tab2_floats(nc)) * 4 +
           kTcCtlBytes + (batch ? kTcStageBytes : 0) + kRedrawBytes;
}

// Byte offset of element (row, k), k < 64, of a K-major operand in the
// 128-byte swizzled layout (8-row groups 1024 bytes apart, the 16-byte
// chunks of row r stored at chunk ^ (r mod 8)).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7))) << 4) +
                      ((k & 7) << 1));
}

// Tile counters: published with a release store by one thread after a
// group barrier, observed with acquire loads (the first one early, while the
// group still works on its current item).
__device__ __forceinline__ void st_release_gpu(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Per-site state of one item.
template <int NB>
struct TcSite {
    SiteIn<NB> in;
    float xn[NB];       // neighbour labels (missing: 1024)
    float xo[NB];       // outlier labels (unused: kNoLabel)
    int n_out;          // outliers of this site
    int m;              // window = chunks [m, m + 16)
    int wlast;          // last window chunk (relative) an in-window tent reaches, -1: none
    float gf;
};

// Window and histogram entries of one site: per neighbour the A byte offset
// it sets (~0u: none) and the count stored there (one store per distinct
// in-window label, of its multiplicity).
template <int NB>
__device__ __forceinline__ void site_window(TcSite<NB> &st, int T, int row, bool valid,
                                            uint32_t (&off)[NB], int (&cnt)[NB])
{
    int xmin = kMissingLabelI;
#pragma unroll
    for (int j = 0; j < NB; ++j)
        xmin = min(xmin, st.in.xni[j]);
    // no neighbour inside the image: every tent sum is zero, any window works
    st.m = xmin < kMissingLabelI ? (xmin - T + 1) >> 3 : 0;
    const int b = 8 * st.m + T - 1;
    st.n_out = 0;
    int xmax_in = -1;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        st.xo[j] = kNoLabel;
        off[j] = ~0u;
        cnt[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int x = st.in.xni[j];
        const bool inside = valid && x < kMissingLabelI;
        const int kb = x - b;
        if (inside && kb >= kBins) {
            // outlier: kept for the CUDA-core tents (slots filled in order)
#pragma unroll
            for (int o = 0; o < NB; ++o)
                if (o == st.n_out)
                    st.xo[o] = (float)x;
            ++st.n_out;
        } else if (inside) {
            xmax_in = max(xmax_in, x);
            bool first = true;
            int c = 1;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (k < j && st.in.xni[k] == x)
                    first = false;
                if (k > j && st.in.xni[k] == x)
                    ++c;
            }
            if (first) {
                off[j] = sw128_offset(row, kb);
                cnt[j] = c;
            }
        }
    }
    // tents of in-window labels end at x + T - 1 <= 8 m + 127 (T <= 33)
    st.wlast = xmax_in >= 0 ? (xmax_in + T - 1 - 8 * st.m) >> 3 : -1;
}

// Chunks (bit c) that an outlier's tent reaches: labels within T - 1 of it.
template <int NB>
__device__ __forceinline__ uint32_t outlier_chunks(const TcSite<NB> &st, int T, int nc)
{
    uint32_t mask = 0u;
#pragma unroll
    for (int o = 0; o < NB; ++o) {
        if (o < st.n_out) {
            const int x = (int)st.xo[o];
            const int c0 = max(x - T + 1, 0) >> 3;
            const int c1 = min((x + T - 1) >> 3, nc - 1);
            if (c1 >= c0)
                mask |= (c1 - c0 >= 31 ? 0xFFFFFFFFu : ((2u << (c1 - c0)) - 1u)) << c0;
        }
    }
    return mask;
}

// Counter of the tile that lane `lane` (0-8) of warp 0 watches for item
// (k, tile j): one of the 3 x 3 tiles around j, or nullptr (none: outside
// the grid, k = 0, or lanes 9-31).
__device__ __forceinline__ const unsigned int *dep_counter(const unsigned int *done, int k, int j,
                                                           int tiles_x, int tiles_y, int lane)
{
    if (k == 0 || lane >= 9)
        return nullptr;
    const int ty = j / tiles_x;
    const int tx = j - ty * tiles_x;
    const int yy = ty + lane / 3 - 1;
    const int xx = tx + lane % 3 - 1;
    if (yy < 0 || yy >= tiles_y || xx < 0 || xx >= tiles_x)
        return nullptr;
    return done + (size_t)yy * tiles_x + xx;
}

// Wait (bounded) until *d >= k; `seen` is an earlier acquire load of *d.
// Every observation is an acquire load, so the labels read after the
// group's next barrier are those the tile published (the publisher's
// release store) without a fence on this path.  Returns false if the wait
// ran out of time or another wait of the launch already gave up.
__device__ __forceinline__ bool wait_counter(const unsigned int *d, unsigned int k,
                                             unsigned int seen, const int *err, long long limit)
{
    return d == nullptr || wait_ge(d, k, seen, err, limit);
}

// Launch parameters.  One chain (BATCH false): a, the planes and the tile
// grid.  Batched chains (BATCH true): slot descriptors with their tile grids
// (4-row tiles, counters done[base + tile]) and the tiles of one sweep; the
// sweep index of slot s is *tdev + k and a slot stops at its budget.
struct TcParams {
    SweepArgs a;
    uint8_t *x0, *x1;    // planes of sweep 0 and 1 of the launch, or (par_from_t) of even and odd t
    const uint32_t *budget;   // one chain: sweeps t >= *budget are skipped (nullptr: none)
    int par_from_t;
    int tiles_x, tiles_y;
    const SlotDesc *slots;
    const uint32_t *t_arr, *budget_arr;   // slot s: sweep counter t_arr[s], budget budget_arr[s]
    const WaveGeom *geom;
    const WaveItem *items;
    int n_items;
    int nsweeps;
    int T;               // truncation shared by every chain of the launch (B operand)
    int nc_max;          // largest chunk count of the launch's chains
    unsigned int *done, *grab;
    int *err;
    long long wait_ns;   // limit of each bounded wait (0: kWaitLimitNs)
};

// One work item: sweep k of `tile` (of a tiles_x x tiles_y grid whose
// counters start at done + base) of chain `slot`.
struct TcItem {
    int k, tile, tx, ty, tiles_x, tiles_y, base, slot;
};

template <bool BATCH>
__device__ __forceinline__ TcItem tc_decode(const TcParams &p, unsigned int item)
{
    TcItem it;
    if constexpr (BATCH) {
        it.k = (int)(item / (unsigned int)p.n_items);
        const WaveItem w = p.items[item - (unsigned int)it.k * (unsigned int)p.n_items];
        const WaveGeom g = p.geom[w.slot];
        it.slot = w.slot;
        it.tile = w.tile;
        it.tiles_x = g.tiles_x;
        it.tiles_y = g.tiles_y;
        it.base = g.base;
    } else {
        const unsigned int ntiles = (unsigned int)(p.tiles_x * p.tiles_y);
        it.k = (int)(item / ntiles);
        it.tile = (int)(item - (unsigned int)it.k * ntiles);
        it.slot = 0;
        it.tiles_x = p.tiles_x;
        it.tiles_y = p.tiles_y;
        it.base = 0;
    }
    it.ty = it.tile / it.tiles_x;
    it.tx = it.tile - it.ty * it.tiles_x;
    return it;
}

// Batched chains, warp 0 of a group: stage item ii (lane 0: its arguments,
// sweep and run flag; every lane: its chain's outside-chunk table into
// `tab`).  Returns whether the chain runs that sweep (active and within its
// budget).
__device__ __forceinline__ bool tc_stage_warp(const TcParams &p, const TcItem &ii, int lane,
                                              SweepArgs *sa, uint32_t *tt, int *go, float *tab)
{
    int run = 0;
    unsigned long long src = 0ull;
    if (lane == 0) {
        const SlotDesc &d = p.slots[ii.slot];
        const uint32_t t = p.t_arr[ii.slot] + (uint32_t)ii.k;
        if (d.active && t < p.budget_arr[ii.slot]) {
            slot_args(d, t, *sa);
            *tt = t;
            run = 1;
            src = reinterpret_cast<unsigned long long>(d.tctab);
        }
        *go = run;
    }
    run = __shfl_sync(0xFFFFFFFFu, run, 0);
    if (run) {
        src = __shfl_sync(0xFFFFFFFFu, src, 0);
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(tab);
        for (int i = lane; i < kTabF / 4; i += 32)
            d4[i] = __ldg(s4 + i);
    }
    return run != 0;
}

// Warp 0 of a group, lanes 0-8: wait for the 3 x 3 tiles around item ii to
// finish sweep k - 1 (pre_d, pre: an earlier look at a counter).
template <bool BATCH>
__device__ __forceinline__ void tc_wait_item(const TcParams &p, const TcItem &ii, int lane,
                                             const unsigned int *pre_d, unsigned int pre)
{
    const unsigned int *d =
        dep_counter(p.done + ii.base, ii.k, ii.tile, ii.tiles_x, ii.tiles_y, lane);
    const unsigned int seen = (d && d == pre_d) ? pre : (d ? ld_acquire_gpu(d) : 0u);
    if (!wait_counter(d, (unsigned int)ii.k, seen, p.err, wait_limit(p.wait_ns)))
        atomicExch(p.err, 1);
}

// Shared memory of one group's FP64 re-draws.
struct GroupRedraw {
    int *site;          // [kSites][kRedrawInts]: g, xi, ub, neighbour labels
    unsigned int *need; // [4] the warps' masks of sites to re-draw
    double *wsum;       // [4] the warps' sums of the site's weights
    int *res;           // the re-drawn label
};

// FP64 re-draw of the group's uncertain draws by all 128 threads: per site
// in turn, thread lt evaluates labels 2 lt and 2 lt + 1 (weight64, the FP64
// tables), a warp scan and the warps' prefix give the CDF, and the thread
// holding u Z finds the label (as warp_redraw_fp64, over 128 threads, so
// the FP64 work of a re-draw spreads over the four schedulers of the
// group's warps).  Every thread of the group calls it; returns s or the
// re-drawn label.  Its first step is a group barrier (any: whether any
// draw of the group is re-drawn), which also orders the memory writes made
// before the call.
template <int NB>
__device__ __forceinline__ int group_redraw_fp64(const DevModel &m, bool need,
                                                 const SiteIn<NB> &in, int s,
                                                 unsigned long long *counter, const GroupRedraw &gr,
                                                 int lt, int bar_id, bool &any)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const int lane = lt & 31, q = lt >> 5;
    const unsigned mask = __ballot_sync(kFull, need);
    if (need) {
        int *row = gr.site + lt * kRedrawInts;
        row[0] = in.g;
        row[1] = in.xi;
        row[2] = (int)in.ub;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            row[3 + j] = in.xni[j];
    }
    if (lane == 0) {
        gr.need[q] = mask;
        if (mask)
            atomicAdd(counter, (unsigned long long)__popc(mask));
    }
    any = named_bar_or(bar_id, kSites, need);   // the masks and inputs are visible after it
    if (!any)
        return s;
    unsigned masks[4];
#pragma unroll
    for (int w = 0; w < 4; ++w)
        masks[w] = gr.need[w];
#pragma unroll 1
    for (int w = 0; w < 4; ++w) {
#pragma unroll 1
        while (masks[w]) {
            const int ol = __ffs((int)masks[w]) - 1;
            masks[w] &= masks[w] - 1u;
            const int owner = w * 32 + ol;
            const int *row = gr.site + owner * kRedrawInts;
            const int lg = row[0], lxi = row[1];
            const uint32_t lub = (uint32_t)row[2];
            int lx[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j)
                lx[j] = row[3 + j];
            const int s0 = 2 * lt, s1 = 2 * lt + 1;
            const double w0 = s0 < m.L ? weight64<NB>(m, lg, lxi, lx, s0) : 0.0;
            const double w1 = s1 < m.L ? weight64<NB>(m, lg, lxi, lx, s1) : 0.0;
            const double part = __dadd_rn(w0, w1);
            double incl = part;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl = __dadd_rn(incl, v);
            }
            double excl = __shfl_up_sync(kFull, incl, 1);
            if (lane == 31)
                gr.wsum[q] = incl;
            named_bar_sync(bar_id, kSites);
            double pre = 0.0, Z = 0.0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double ws = gr.wsum[v];
                if (v < q)
                    pre = __dadd_rn(pre, ws);
                Z = __dadd_rn(Z, ws);
            }
            incl = __dadd_rn(pre, incl);
            excl = lane == 0 ? pre : __dadd_rn(pre, excl);
            const double t = __dmul_rn((double)lub * (1.0 / 16777216.0), Z);
            if (lt == 0)
                *gr.res = m.L - 1;   // no label below t: the last one
            named_bar_sync(bar_id, kSites);
            if (excl <= t && t < incl) {
                const double c0 = __dadd_rn(excl, w0);
                *gr.res = (t < c0 && s0 < m.L) ? s0 : min(s1, m.L - 1);
            }
            named_bar_sync(bar_id, kSites);
            const int r = *gr.res;
            if (lt == owner)
                s = r;
            named_bar_sync(bar_id, kSites);   // wsum and res are free again
        }
    }
    return s;
}

// The arguments of the current item: the launch's (one chain, read from
// the kernel parameters) or the staged ones (batched chains).
template <bool BATCH>
__device__ __forceinline__ const SweepArgs &item_args(const TcParams &p, const SweepArgs *staged)
{
    if constexpr (BATCH)
        return *staged;
    else
        return p.a;
}

// BUDGET (one chain): sweeps with index >= *p.budget are skipped.  GIBBS
// (one chain, 4-neighbourhood): the checkerboard Gibbs sweep in place on
// p.x0; item k is colour phase k & 1 of sweep k >> 1 over 8 x 32 tiles,
// whose 128 sites of that colour are the group's sites.
template <int NB, bool LMASK, bool BATCH, bool BUDGET, bool GIBBS = false>
__global__ void __launch_bounds__(kThr, 1) pca_tcw_kernel(const TcParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = (int)threadIdx.x;
    const int grp = tid >> 7;          // warpgroup = tile slot
    const int lt = tid & 127;          // site of the tile = TMEM lane
    const int q = lt >> 5;             // warp of the group = lane quarter = tile row
    const int lane = tid & 31;
    if (smem_u32(smem) & 1023u) {      // the swizzled operands need 1024-byte alignment
        if (tid == 0)
            atomicExch(p.err, 2);
        return;
    }
    const int ncm = p.nc_max;
    uint8_t *B = smem + kOffB;
    uint8_t *A = smem + kOffA + grp * kOpBytes;
    float *Gcol = reinterpret_cast<float *>(smem + kOffG) + tid;
    // outside-chunk tables: the chain's, or two per group (staged items)
    float *tabs = reinterpret_cast<float *>(smem + kOffG + ncm * kThr * 4);
    uint64_t *mbar =
        reinterpret_cast<uint64_t *>(tabs + (BATCH ? 2 * kGroups * kTabF : tab2_floats(ncm)));
    unsigned int *s_item = reinterpret_cast<unsigned int *>(mbar + kGroups);
    uint32_t *tmem_slot = s_item + kGroups;
    // batched chains: per group, two staged items (arguments, sweep, run flag)
    SweepArgs *s_args = reinterpret_cast<SweepArgs *>(
        reinterpret_cast<uint8_t *>(mbar) + kTcCtlBytes);
    uint32_t *s_t = reinterpret_cast<uint32_t *>(s_args + 2 * kGroups);
    int *s_go = reinterpret_cast<int *>(s_t + 2 * kGroups);
    float *gtabs = tabs + grp * 2 * kTabF;   // batched chains: this group's two tables
    GroupRedraw gr;
    {
        uint8_t *rb = reinterpret_cast<uint8_t *>(mbar) + kTcCtlBytes + (BATCH ? kTcStageBytes : 0) +
                      grp * (kSites * kRedrawInts * 4 + 4 * 4 + 4 * 8 + 16);
        gr.wsum = reinterpret_cast<double *>(rb);
        gr.need = reinterpret_cast<unsigned int *>(rb + 4 * 8);
        gr.res = reinterpret_cast<int *>(rb + 4 * 8 + 4 * 4);
        gr.site = reinterpret_cast<int *>(rb + 4 * 8 + 4 * 4 + 16);
    }

    // A starts zero; B holds K(k, c) at row c (window label), column k (bin)
    for (int i = tid; i < (kOpBytes * (1 + kGroups)) / 16; i += kThr)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int i = tid; i < kWin * kBins; i += kThr) {
        const int c = i / kBins, k = i - (i / kBins) * kBins;
        const int v = max(p.T - abs(c - (p.T - 1) - k), 0);
        *reinterpret_cast<__half *>(B + sw128_offset(c, k)) = __int2half_rn(v);
    }
    if constexpr (!BATCH) {
        // outside-chunk sums: chunk c of observation g (the same function,
        // hence the same values, as computing them per site)
        for (int i = tid; i < ncm * 256; i += kThr) {
            const int c = i >> 8, gobs = i & 255;
            tabs[c * kTabRow + gobs] = outside_chunk<LMASK>(p.a.m, (float)gobs, c);
        }
    }
    if (tid == 0) {
        for (int g = 0; g < kGroups; ++g)
            mbar_init(&mbar[g], 1);
        mbar_init_fence();
    }
    if (tid < 32) {
        tmem_alloc(tmem_slot, (uint32_t)kTmemCols);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tcol = tmem + (uint32_t)(grp * kWin);          // the group's columns
    const uint32_t trow = tcol + ((uint32_t)(q * 32) << 16);      // this warp's lanes
    const int bar_id = 1 + grp;
    const unsigned int total =
        (unsigned int)(BATCH ? p.n_items : p.tiles_x * p.tiles_y) * (unsigned int)p.nsweeps;
    const uint32_t t0 = BATCH ? 0u : sweep_index(p.a);
    const uint32_t tlim = BUDGET ? *p.budget : 0xFFFFFFFFu;   // one chain
    const long long limit = wait_limit(p.wait_ns);

    uint32_t prev_off[NB];   // A entries this thread set for its previous item
#pragma unroll
    for (int j = 0; j < NB; ++j)
        prev_off[j] = ~0u;
    int uses = 0;            // completed phases of the group's mbarrier
    bool ok = true;
    unsigned int seq = 0;    // items this group took (parity: staging buffer)

    // first item (warp 0 waits for its neighbourhood; thread 0 stages it)
    if (q == 0) {
        unsigned int it = 0;
        if (lane == 0)
            it = atomicAdd(p.grab, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it < total) {
            const TcItem ii = tc_decode<BATCH>(p, it);
            bool run = !BUDGET || t0 + (uint32_t)ii.k < tlim;
            if constexpr (BATCH)
                run = tc_stage_warp(p, ii, lane, s_args + grp * 2, s_t + grp * 2, s_go + grp * 2,
                                    gtabs);
            if (run)
                tc_wait_item<BATCH>(p, ii, lane, nullptr, 0u);
        }
        if (lane == 0)
            s_item[grp] = it;
    }
    named_bar_sync(bar_id, kSites);
    unsigned int item = s_item[grp];
    unsigned int next = 0;   // warp 0, lane 0: the item taken for after this one

    while (item < total) {
        const unsigned int par = seq & 1u;
        const TcItem ii = tc_decode<BATCH>(p, item);
        const int k = ii.k;
        // Gibbs: thread lt takes tile row lt / 16 and, in column pair lt % 16,
        // the site of the phase's colour ((r + c) mod 2 = colour)
        const int colour = GIBBS ? (k & 1) : 0;
        const int r = GIBBS ? ii.ty * kGibbsRows + (lt >> 4) : ii.ty * kTileRows + q;
        const int c = GIBBS ? ii.tx * 32 + 2 * (lt & 15) + ((r + colour) & 1) : ii.tx * 32 + lane;
        bool go = true;
        const SweepArgs *bp = nullptr;   // batched chains: the staged arguments
        const float *tab;        // outside-chunk sums (shared memory)
        const uint8_t *xin;      // planes of this sweep
        uint8_t *xout;
        uint32_t t;
        if constexpr (BATCH) {
            go = s_go[grp * 2 + par] != 0;
            bp = &s_args[grp * 2 + par];
            tab = gtabs + par * kTabF;
            t = s_t[grp * 2 + par];
            xin = bp->xin;
            xout = bp->xout;
        } else if constexpr (GIBBS) {
            t = t0 + (uint32_t)(k >> 1);
            xin = p.x0;   // in place: a phase reads the other colour only
            xout = p.x0;
            tab = tabs;
        } else {
            t = t0 + (uint32_t)k;
            const uint32_t ph = p.par_from_t ? (t & 1u) : (uint32_t)(k & 1);
            xin = ph ? p.x1 : p.x0;
            xout = ph ? p.x0 : p.x1;
            tab = tabs;
            if constexpr (BUDGET)
                go = t < tlim;
        }
        const unsigned int *dnext = nullptr;   // warp 0: an early look at the next item
        unsigned int seen = 0u;
        int knext = -1;                        // its sweep (-1: no look taken)

        if (go) {
            const SweepArgs &b = item_args<BATCH>(p, bp);
            const DevModel &m = b.m;
            const float mu = -m.gam;
            const int nc = (m.L + kChunk - 1) / kChunk;
            const bool valid = r < b.H && c < b.W;

            // site inputs, window, histogram row
            TcSite<NB> st;
            st.in = SiteIn<NB>{};
            if (valid)
                load_site<NB, true>(b, xin, r, c, GIBBS ? kTagGibbs : kTagPCA, t, st.in);
            float *accp = b.acc + (size_t)r * b.W + c;
            // Gibbs accumulates after the last phase: this site and its pair's
            // colour-0 site, final since phase 0 of this sweep
            const bool acc_on = valid && (!GIBBS || colour == 1) && accumulate_after(b, t);
            const float acc_old = acc_on ? __ldcg(accp) : 0.0f;   // prefetched
            if constexpr (GIBBS) {
                const int cp = c ^ 1;
                if (colour == 1 && r < b.H && cp < b.W && accumulate_after(b, t)) {
                    float *ap = b.acc + (size_t)r * b.W + cp;
                    *ap = __ldcg(ap) + (float)__ldcg(xin + (size_t)r * b.pitch + cp);
                }
            }
#pragma unroll
            for (int jn = 0; jn < NB; ++jn)
                st.xn[jn] = (float)st.in.xni[jn];
            st.gf = (float)st.in.g;
            uint32_t off[NB];
            int cnt[NB];
            site_window<NB>(st, m.T, lt, valid, off, cnt);
#pragma unroll
            for (int jn = 0; jn < NB; ++jn)
                if (prev_off[jn] != ~0u)
                    *reinterpret_cast<__half *>(A + prev_off[jn]) =
                        __ushort_as_half((unsigned short)0);
#pragma unroll
            for (int jn = 0; jn < NB; ++jn) {
                if (off[jn] != ~0u)
                    *reinterpret_cast<__half *>(A + off[jn]) = __int2half_rn(cnt[jn]);
                prev_off[jn] = off[jn];
            }
            fence_async_smem();
            tc_fence_before_sync();
            named_bar_sync(bar_id, kSites);   // rows written, the previous item's TMEM reads done
            if (lt == 0) {
                tc_fence_after_sync();
                const uint64_t adesc = sw128_kmajor_desc(smem_u32(A));
                const uint64_t bdesc = sw128_kmajor_desc(smem_u32(B));
#pragma unroll
                for (int ks = 0; ks < kBins / 16; ++ks)   // 32-byte K steps inside the row
                    umma_f16_ss(tcol, adesc + (uint64_t)(2 * ks), bdesc + (uint64_t)(2 * ks),
                                kIdesc, ks > 0 ? 1u : 0u);
                umma_commit(&mbar[grp]);
                next = atomicAdd(p.grab, 1u);   // used at the end of this item
            }
            if constexpr (BATCH) {
                // stage the next item now, off the group's critical path
                if (q == 0) {
                    const unsigned int nx = __shfl_sync(0xFFFFFFFFu, next, 0);
                    if (nx < total)
                        tc_stage_warp(p, tc_decode<BATCH>(p, nx), lane, s_args + grp * 2 + (par ^ 1u),
                                      s_t + grp * 2 + (par ^ 1u), s_go + grp * 2 + (par ^ 1u),
                                      gtabs + (par ^ 1u) * kTabF);
                }
            }

            // outside chunks, while the tensor core runs
            const int lo = max(st.m, 0);
            const int hi = min(st.m + kWinChunks, nc);
            const int n_oc = lo + nc - hi;
            const int n_oc_w = __reduce_max_sync(0xFFFFFFFFu, n_oc);
            // outside sum of chunk cc: the chain's 2-D table or the staged 1-D one
            const auto outside = [&](int cc) {
                if constexpr (BATCH)
                    return tab_sum<LMASK>(tab, st.in.g, cc, nc);
                else
                    return tab[cc * kTabRow + st.in.g];
            };
#pragma unroll 4
            for (int jj = 0; jj < n_oc_w; ++jj) {
                const int cc = jj < lo ? jj : hi + (jj - lo);
                if (jj < n_oc)
                    Gcol[cc * kThr] = outside(cc);
            }

            // an early look at the next item's neighbourhood (warp 0)
            if (q == 0) {
                const unsigned int nx = __shfl_sync(0xFFFFFFFFu, next, 0);
                if (nx < total) {
                    const TcItem in2 = tc_decode<BATCH>(p, nx);
                    knext = in2.k;
                    dnext = dep_counter(p.done + in2.base, in2.k, in2.tile, in2.tiles_x,
                                        in2.tiles_y, lane);
                    if (dnext)
                        seen = ld_acquire_gpu(dnext);
                }
            }

            // window chunks from TMEM
            if (!mbar_wait_timed(&mbar[grp], (uint32_t)(uses & 1), limit)) {
                atomicExch(p.err, 1);
                ok = false;
            }
            ++uses;
            tc_fence_after_sync();
            // 32-column groups up to the warp's last chunk with a tent; the
            // window chunks after it hold zero tent sums: outside sums
            const int ngrp = (__reduce_max_sync(0xFFFFFFFFu, st.wlast) >> 2) + 1;
#pragma unroll 1
            for (int h = 0; h < ngrp; ++h) {
                uint32_t pb[32];
                tmem_ld32(trow + (uint32_t)(32 * h), pb);
                tmem_wait_ld(pb);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int cc = st.m + 4 * h + i;
                    const float S = window_chunk<LMASK>(m, mu, st.gf, pb + 8 * i, cc);
                    if (cc >= 0 && cc < nc)
                        Gcol[cc * kThr] = S;
                }
            }
#pragma unroll 1
            for (int i = 4 * ngrp; i < kWinChunks; ++i) {
                const int cc = st.m + i;
                if (cc >= 0 && cc < nc)
                    Gcol[cc * kThr] = outside(cc);
            }
            tc_fence_before_sync();

            // chunks an outlier's tent reaches are recomputed from exact tent
            // sums; the (site, chunk) tasks of the warp are dealt out to all
            // 32 lanes (a lane takes task lane + 32 r and writes the owner's
            // column)
            const uint32_t omask = outlier_chunks<NB>(st, m.T, nc);
            if (__any_sync(0xFFFFFFFFu, omask != 0u)) {
                const int cntb = __popc(omask);
                int incl = cntb;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o)
                        incl += v;
                }
                const int ntask = __shfl_sync(0xFFFFFFFFu, incl, 31);
#pragma unroll 1
                for (int base = 0; base < ntask; base += 32) {
                    const int tsk = base + lane;
                    int owner = 0;   // lanes whose inclusive count is <= tsk
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(0xFFFFFFFFu, incl, owner + step - 1);
                        if (v <= tsk)
                            owner += step;
                    }
                    owner = min(owner, 31);
                    const int o_excl = __shfl_sync(0xFFFFFFFFu, incl - cntb, owner);
                    const uint32_t o_mask = __shfl_sync(0xFFFFFFFFu, omask, owner);
                    const float o_gf = __shfl_sync(0xFFFFFFFFu, st.gf, owner);
                    float o_xn[NB];
#pragma unroll
                    for (int jn = 0; jn < NB; ++jn)
                        o_xn[jn] = __shfl_sync(0xFFFFFFFFu, st.xn[jn], owner);
                    const bool mine = tsk < ntask;
                    const int cc = mine ? (int)__fns(o_mask, 0u, tsk - o_excl + 1) : 0;
                    float pp[kChunk];
                    chunk_prefix_exact<NB>(m, mu, o_xn, o_gf, cc, pp);
                    if (mine)
                        Gcol[cc * kThr + owner - lane] = pp[kChunk - 1];
                }
                __syncwarp();   // the owners read their columns below
            }

            // chunk prefix sums in label order (Kahan), certified selection
            float G = 0.0f, comp = 0.0f;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) {
                if (cc < nc) {
                    const float y = __fsub_rn(Gcol[cc * kThr], comp);
                    const float tt = __fadd_rn(G, y);
                    comp = __fsub_rn(__fsub_rn(tt, G), y);
                    G = tt;
                    Gcol[cc * kThr] = G;
                }
            }
            int s = 0;
            bool certain = true;
            if (valid) {
                float delta = 0.0f;
                if (m.em1 != 0.0f) {
                    const float xif = (float)st.in.xi;
                    delta = __fmul_rn(label_wb(m, mu, tent_sum<NB>(st.xn, m.Tf, xif),
                                               __fsub_rn(st.gf, xif)),
                                      m.em1);
                }
                // the site's certified margin from its own total (entropy bound)
                s = cdf_select(m, site_margin(m, G, delta), [&](int cc) { return Gcol[cc * kThr]; },
                               nc, G, delta,
                               st.in.xi, st.in.ub, certain, [&](int cs, float (&pp)[kChunk]) {
                                   chunk_prefix_exact<NB>(m, mu, st.xn, st.gf, cs, pp);
                               });
            }
            // certain draws are written now; the re-draw's first barrier
            // orders them before the tile is published; re-drawn ones
            // follow with one more barrier
            const bool need = valid && !certain;
            const auto write_site = [&]() {
                xout[(size_t)r * b.pitch + c] = (uint8_t)s;
                if (acc_on)
                    *accp = acc_old + (float)s;
            };
            if (valid && !need)
                write_site();
            bool any = false;
            s = group_redraw_fp64<NB>(m, need, st.in, s, b.fp64_draws, gr, lt, bar_id, any);
            if (any) {
                if (need)
                    write_site();
                named_bar_sync(bar_id, kSites);
            }
        } else {
            if (lt == 0)
                next = atomicAdd(p.grab, 1u);   // a skipped item: take the next one here
            named_bar_sync(bar_id, kSites);
        }

        // publish the tile's sweep (every output written), take the next item
        // warp 1 publishes (its release store waits for the tile's writes to
        // drain) while warp 0 takes the next item
        if (q == 1 && lane == 0 && go &&   // after every output of the tile
            (BATCH || ii.tile != p.a.stall_tile - 1))
            st_release_gpu(p.done + ii.base + ii.tile, (unsigned int)(k + 1));
        if (q == 0) {
            if (lane == 0)   // no further item once a wait of the launch gave up
                s_item[grp] = ld_flag(p.err) ? total : next;
            const unsigned int nx = __shfl_sync(0xFFFFFFFFu, next, 0);
            if (nx < total) {
                if constexpr (BATCH) {
                    const TcItem in2 = tc_decode<BATCH>(p, nx);
                    const unsigned int pn = par ^ 1u;
                    bool run;
                    if (go)   // staged when this item issued its MMA
                        run = __shfl_sync(0xFFFFFFFFu, s_go[grp * 2 + pn], 0) != 0;
                    else
                        run = tc_stage_warp(p, in2, lane, s_args + grp * 2 + pn, s_t + grp * 2 + pn,
                                            s_go + grp * 2 + pn, gtabs + pn * kTabF);
                    if (run)
                        tc_wait_item<BATCH>(p, in2, lane, dnext, seen);
                } else if (knext >= 0) {   // looked at during this item
                    if (!BUDGET || t0 + (uint32_t)knext < tlim)
                        if (!wait_counter(dnext, (unsigned int)knext, seen, p.err, limit))
                            atomicExch(p.err, 1);
                } else {
                    const TcItem in2 = tc_decode<BATCH>(p, nx);
                    if (!BUDGET || t0 + (uint32_t)in2.k < tlim)
                        tc_wait_item<BATCH>(p, in2, lane, nullptr, 0u);
                }
            }
        }
        named_bar_sync(bar_id, kSites);
        item = s_item[grp];
        ++seq;
    }

    // a timed-out wait may leave an MMA in flight: wait for it (bounded)
    // before TMEM is freed
    if (!ok && lt == 0 && uses > 0)
        mbar_wait_timed(&mbar[grp], (uint32_t)((uses - 1) & 1), limit);
    tc_fence_before_sync();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, (uint32_t)kTmemCols);
    }
}

template <int NB, bool LMASK, bool BATCH, bool BUDGET, bool GIBBS = false>
cudaError_t launch_tcw_t(const TcParams &p, long long items, cudaStream_t st)
{
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64)
        return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(pca_tcw_kernel<NB, LMASK, BATCH, BUDGET, GIBBS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem_bytes(32, BATCH));
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    if (items <= 0)
        return cudaSuccess;
    if (items >= (1ll << 32))
        return cudaErrorInvalidValue;
    // one CTA per SM (TMEM: all 512 columns); no more CTAs than 4-item groups
    const long long need = (items + kGroups - 1) / kGroups;
    const int grid = (int)(need < sms ? need : sms);
    pca_tcw_kernel<NB, LMASK, BATCH, BUDGET, GIBBS><<<grid, kThr, tc_smem_bytes(p.nc_max, BATCH), st>>>(
        p);
    return cudaGetLastError();
}

template <bool BATCH, bool BUDGET>
cudaError_t launch_tcw(const TcParams &p, int nbhd, bool lmask, long long items, cudaStream_t st)
{
    if (nbhd == 8)
        return lmask ? launch_tcw_t<8, true, BATCH, BUDGET>(p, items, st)
                     : launch_tcw_t<8, false, BATCH, BUDGET>(p, items, st);
    return lmask ? launch_tcw_t<4, true, BATCH, BUDGET>(p, items, st)
                 : launch_tcw_t<4, false, BATCH, BUDGET>(p, items, st);
}

template <bool LMASK>
__global__ void tc_table_kernel(const DevModel m, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kTabF)
        out[i] = tab_entry<LMASK>(m, i);
}

}  // namespace

bool pca_tc_eligible(const DevModel &m)
{
    return m.L >= kTcMinLabels && m.L <= 256 && m.T >= 1 && m.T <= kTcMaxT && m.norm == 0 &&
           (m.nbhd == 4 || m.nbhd == 8);
}

bool pca_tc_auto(const DevModel &m)
{
    return pca_tc_eligible(m) && m.L >= kTcAutoLabels;
}

int tc_table_floats(int)
{
    return kTabF;
}

cudaError_t launch_tc_table(const DevModel &m, float *out, cudaStream_t st)
{
    if (m.L % kChunk)
        tc_table_kernel<true><<<(kTabF + 255) / 256, 256, 0, st>>>(m, out);
    else
        tc_table_kernel<false><<<(kTabF + 255) / 256, 256, 0, st>>>(m, out);
    return cudaGetLastError();
}

cudaError_t launch_pca_tc(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int nsweeps,
                          unsigned int *done, unsigned int *grab, int *err, cudaStream_t st,
                          const uint32_t *budget, bool par_from_t)
{
    if (!pca_tc_eligible(a.m))
        return cudaErrorInvalidValue;
    TcParams p{};
    p.a = a;
    p.x0 = x0;
    p.x1 = x1;
    p.budget = budget;
    p.par_from_t = par_from_t ? 1 : 0;
    p.tiles_x = (a.W + 31) / 32;
    p.tiles_y = (a.H + kTileRows - 1) / kTileRows;
    p.nsweeps = nsweeps;
    p.T = a.m.T;
    p.nc_max = (a.m.L + kChunk - 1) / kChunk;
    p.done = done;
    p.grab = grab;
    p.err = err;
    p.wait_ns = a.wait_ns;
    const long long items = (long long)p.tiles_x * p.tiles_y * nsweeps;
    if (budget)
        return launch_tcw<false, true>(p, a.m.nbhd, (a.m.L % kChunk) != 0, items, st);
    return launch_tcw<false, false>(p, a.m.nbhd, (a.m.L % kChunk) != 0,
                             (long long)p.tiles_x * p.tiles_y * nsweeps, st);
}

cudaError_t launch_gibbs_tc(const SweepArgs &a, uint8_t *x, int nsweeps, unsigned int *done,
                            unsigned int *grab, int *err, cudaStream_t st)
{
    if (!pca_tc_eligible(a.m) || a.m.nbhd != 4)
        return cudaErrorInvalidValue;
    TcParams p{};
    p.a = a;
    p.x0 = x;
    p.x1 = x;
    p.tiles_x = (a.W + 31) / 32;
    p.tiles_y = (a.H + kGibbsRows - 1) / kGibbsRows;
    p.nsweeps = 2 * nsweeps;   // colour phases
    p.T = a.m.T;
    p.nc_max = (a.m.L + kChunk - 1) / kChunk;
    p.done = done;
    p.grab = grab;
    p.err = err;
    p.wait_ns = a.wait_ns;
    const long long items = (long long)p.tiles_x * p.tiles_y * p.nsweeps;
    return (a.m.L % kChunk) != 0 ? launch_tcw_t<4, true, false, false, true>(p, items, st)
                                 : launch_tcw_t<4, false, false, false, true>(p, items, st);
}

cudaError_t launch_batch_tc(const SlotDesc *slots, const uint32_t *t_arr,
                            const uint32_t *budget_arr, const WaveGeom *geom,
                            const WaveItem *items, int n_items, int nsweeps, int T, int nbhd,
                            bool lmask, int nc_max, unsigned int *done, unsigned int *grab,
                            int *err, cudaStream_t st)
{
    if (T < 1 || T > kTcMaxT || (nbhd != 4 && nbhd != 8) || nc_max < 1 || nc_max > 32)
        return cudaErrorInvalidValue;
    TcParams p{};
    p.slots = slots;
    p.t_arr = t_arr;
    p.budget_arr = budget_arr;
    p.geom = geom;
    p.items = items;
    p.n_items = n_items;
    p.nsweeps = nsweeps;
    p.T = T;
    p.nc_max = nc_max;
    p.done = done;
    p.grab = grab;
    p.err = err;
    return launch_tcw<true, false>(p, nbhd, lmask, (long long)n_items * nsweeps, st);
}

}  // namespace pcad
