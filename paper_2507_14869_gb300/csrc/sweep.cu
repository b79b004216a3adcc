// Sweep kernels: lazy PCA (Section 5.2) and checkerboard Gibbs (Section 5.1).
//
// One thread per site.  The site's label, its neighbours' labels and its
// observation are read straight from global memory (each byte is reused by
// up to 9 threads through L1); the per-label work (energy, exponential, CDF)
// dominates for L >= 16.  The per-thread chunk prefix sums of the two-pass
// CDF live in shared memory.
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 4;
constexpr int kThreads = kBX * kBY;

// Draw the new label of every valid site of the warp; uncertain FP32 draws
// are re-evaluated in FP64 by the whole warp.  Every lane must call this.
// NORM: the inertia price (0: L0 via the single-label correction; 1, 2: Lp).
template <int NC, int NB, int NORM = 0>
__device__ __forceinline__ int draw_site(const SweepArgs &a, bool valid, const SiteIn<NB> &in,
                                         float *Gcol)
{
    int s = 0;
    bool certain = true;
    if constexpr (NORM == 0) {
        // chunks where any lane's prior has a kink take the general path; with
        // few chunks (L <= 32) the mask costs more than the linear path saves
        uint32_t dirty = 0xFFFFFFFFu;
        if (NC >= 8)
            dirty = __reduce_or_sync(0xFFFFFFFFu, valid ? dirty_chunks<NB>(in.xni, a.m.T) : 0u);
        if (valid)
            s = draw_fp32<NC, NB>(a.m, Gcol, kThreads, in, dirty, certain);
    } else {
        if (valid)
            s = draw_fp32_norm<NC, NB, NORM>(a.m, Gcol, kThreads, in, certain);
    }
    return warp_redraw_fp64<NB, NORM>(a.m, valid && !certain, in, s, a.fp64_draws);
}

// One lazy-PCA site update (r, c) at sweep t: draw from x_in, write x_out,
// accumulate after burn-in.  Every lane of the warp must call it (lanes
// outside the image pass through the warp-level steps).
// L2_ONLY: labels and accumulator written by other SMs in the same launch
// are read through L2 (the wavefront kernel).
template <int NC, int NB, int NORM = 0, bool L2_ONLY = false>
__device__ __forceinline__ void pca_site(const SweepArgs &a, int r, int c, uint32_t t, float *Gcol,
                                         const uint32_t *u_s = nullptr)
{
    const bool valid = r < a.H && c < a.W;
    SiteIn<NB> in{};
    if (valid) {
        if (u_s) {
            load_site<NB, L2_ONLY, false>(a, a.xin, r, c, kTagPCA, t, in);
            in.ub = *u_s;
        } else {
            load_site<NB, L2_ONLY>(a, a.xin, r, c, kTagPCA, t, in);
        }
    }
    const int s = draw_site<NC, NB, NORM>(a, valid, in, Gcol);
    if (valid) {
        a.xout[(size_t)r * a.pitch + c] = (uint8_t)s;
        if (accumulate_after(a, t)) {
            float *p = a.acc + (size_t)r * a.W + c;
            *p = (L2_ONLY ? __ldcg(p) : *p) + (float)s;
        }
    }
}


template <int NC, int NB, int NORM>
__global__ void __launch_bounds__(kThreads) pca_direct_kernel(const SweepArgs a)
{
    __shared__ float G_s[NC * kThreads];
    __shared__ __align__(16) uint32_t U_s[kBY * kBX];
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int c = blockIdx.x * kBX + threadIdx.x;
    const int r = blockIdx.y * kBY + threadIdx.y;
    const uint32_t t = sweep_index(a);
    if (threadIdx.y == 0)
        block_uniforms(a, blockIdx.y * kBY, blockIdx.x * kBX, t, U_s);
    __syncthreads();
    pca_site<NC, NB, NORM>(a, r, c, t, G_s + tid, U_s + tid);
}

// Wavefront lazy-PCA over nsweeps sweeps in one persistent launch.  Work
// items (sweep k, tile j) of 4 x 32 sites are taken in increasing order from
// an atomic counter; item (k, j) waits until the 3 x 3 tiles around j have
// finished sweep k - 1 (done[] counts finished sweeps per tile).  The tiles
// it reads (x of sweep k) and overwrites (x of sweep k - 1) are exactly
// those, so no sweep-wide barrier is needed and the tail of one sweep
// overlaps the start of the next.  Every item an item depends on has a
// smaller index and was taken by a block that is resident (the grid is the
// resident capacity), so the waits end; each is bounded anyway (error flag).
// Draws are keyed by (sweep, site): results equal per-sweep launches.
// Tile counters are observed with acquire loads: a waiting lane's label
// reads after the block barrier see what the tile published.  A wait that
// runs out sets *err; the block then takes no further item, and every other
// block stops at its next wait or item.
#ifndef PCAD_WAVE_MIN_BLOCKS
#define PCAD_WAVE_MIN_BLOCKS 8   // resident blocks per SM the register budget targets
#endif

template <int NC, int NB>
__global__ void __launch_bounds__(kThreads, PCAD_WAVE_MIN_BLOCKS) pca_wave_kernel(const SweepArgs a, uint8_t *x0,
                                                           uint8_t *x1, int nsweeps,
                                                           int tiles_x, int tiles_y,
                                                           unsigned int *done,
                                                           unsigned int *grab, int *err)
{
    __shared__ float G_s[NC * kThreads];
    __shared__ __align__(16) uint32_t U_s[kBY * kBX];
    __shared__ unsigned int s_next;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const unsigned int ntiles = (unsigned int)(tiles_x * tiles_y);
    const unsigned int total = ntiles * (unsigned int)nsweeps;
    const uint32_t t0 = sweep_index(a);
    const long long limit = wait_limit(a.wait_ns);
    if (tid == 0)
        s_next = atomicAdd(grab, 1u);
    __syncthreads();
    unsigned int item = s_next;
    while (item < total) {
        const int k = (int)(item / ntiles);
        const int j = (int)(item - (unsigned int)k * ntiles);
        const int ty = j / tiles_x;
        const int tx = j - ty * tiles_x;
        __syncthreads();   // everyone has read s_next
        if (threadIdx.y == 0) {
            // lane 31 fetches the following item (none once a wait of the
            // launch gave up) while lanes 0-8 each wait for one tile of the
            // 3 x 3 neighbourhood to finish sweep k - 1
            if (threadIdx.x == 31)
                s_next = ld_flag(err) ? total : atomicAdd(grab, 1u);
            bool ok = true;
            if (k > 0 && threadIdx.x < 9) {
                const int yy = ty + (int)threadIdx.x / 3 - 1;
                const int xx = tx + (int)threadIdx.x % 3 - 1;
                if (yy >= 0 && yy < tiles_y && xx >= 0 && xx < tiles_x) {
                    const unsigned int *d = done + (size_t)yy * tiles_x + xx;
                    ok = wait_ge(d, (unsigned int)k, ld_acquire_u32(d), err, limit);
                }
            }
            if (!ok)
                atomicExch(err, 1);
            __syncwarp();
        } else if (threadIdx.y == 1) {
            block_uniforms(a, ty * kBY, tx * kBX, t0 + (uint32_t)k, U_s);
        }
        __syncthreads();
        SweepArgs b = a;
        b.xin = (k & 1) ? x1 : x0;
        b.xout = (k & 1) ? x0 : x1;
        pca_site<NC, NB, 0, true>(b, ty * kBY + threadIdx.y, tx * kBX + threadIdx.x,
                                  t0 + (uint32_t)k, G_s + tid, U_s + tid);
        __syncthreads();
        if (tid == 0 && j != a.stall_tile - 1) {
            __threadfence();   // the tile's labels and sums before its counter
            atomicExch(done + j, (unsigned int)(k + 1));
        }
        item = s_next;
    }
}

// Gibbs colour phase q.  A thread owns one "cell": a pair of columns
// (4-neighbourhood, colours by (r + c) mod 2) or a 2x2 block
// (8-neighbourhood, colours by (r mod 2, c mod 2)); it updates the cell's
// site of colour q in place.  No two sites of one colour are neighbours, so
// the phase equals a sequential scan of that colour in any order.  After
// the last phase every site of the cell is final and is accumulated.
template <int NC, int NB>
__global__ void __launch_bounds__(kThreads) gibbs_cb_kernel(const SweepArgs a, int q)
{
    __shared__ float G_s[NC * kThreads];
    __shared__ __align__(16) uint32_t U_s[kBY * 2 * kBX];   // 4 site rows x 64 columns
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int cx = blockIdx.x * kBX + threadIdx.x;
    const int cy = blockIdx.y * kBY + threadIdx.y;
    uint8_t *x = const_cast<uint8_t *>(a.xin);
    int r0, c0, r, c;
    if (NB == 4) {
        r0 = cy;
        c0 = 2 * cx;
        r = r0;
        c = c0 + ((r + q) & 1);
    } else {
        r0 = 2 * cy;
        c0 = 2 * cx;
        r = r0 + (q >> 1);
        c = c0 + (q & 1);
    }
    const bool cell = r0 < a.H && c0 < a.W;
    const bool valid = cell && r < a.H && c < a.W;
    const uint32_t t = sweep_index(a);
    // The block's phase sites lie in 4 rows (one per threadIdx.y) and 64
    // columns: 64 Philox blocks (one per 4 columns), computed by warps 0 and 1
    // (warp w, lane l: row (32 w + l) / 16, columns 4 ((32 w + l) % 16) ..).
    if (threadIdx.y < 2) {
        const int i = (int)threadIdx.y * 32 + (int)threadIdx.x;
        const int ri = i >> 4;
        const int row = NB == 4 ? (int)blockIdx.y * kBY + ri
                                : 2 * ((int)blockIdx.y * kBY + ri) + (q >> 1);
        uint32_t o0, o1, o2, o3;
        philox4x32_10((uint32_t)(16 * (int)blockIdx.x + (i & 15)), (uint32_t)row, t,
                      (kTagGibbs << 24) | (a.chain & 0xFFFFFFu),
                      (uint32_t)(a.seed & 0xFFFFFFFFull), (uint32_t)(a.seed >> 32), o0, o1, o2, o3);
        reinterpret_cast<uint4 *>(U_s)[i] = make_uint4(o0 >> 8, o1 >> 8, o2 >> 8, o3 >> 8);
    }
    __syncthreads();
    SiteIn<NB> in{};
    if (valid) {
        load_site<NB, false, false>(a, x, r, c, kTagGibbs, t, in);
        in.ub = U_s[threadIdx.y * 2 * kBX + (c - 2 * kBX * (int)blockIdx.x)];
    }
    const int s = draw_site<NC, NB>(a, valid, in, G_s + tid);
    if (valid)
        x[(size_t)r * a.pitch + c] = (uint8_t)s;
    if (cell && a.last_phase && accumulate_after(a, t)) {
        const int nr = NB == 4 ? 1 : 2;
#pragma unroll
        for (int dr = 0; dr < nr; ++dr)
#pragma unroll
            for (int dc = 0; dc < 2; ++dc) {
                const int rr = r0 + dr, cc = c0 + dc;
                if (rr < a.H && cc < a.W)
                    a.acc[(size_t)rr * a.W + cc] += (float)x[(size_t)rr * a.pitch + cc];
            }
    }
}

// Batched lazy-PCA sweep over many chains of uneven size and model.  The
// grid is persistent (a multiple of the SM count); each block takes work
// items (tiles of one chain) in the host's order (costliest first) from an
// atomic counter, runs the same per-site code as pca_direct_kernel, and
// dispatches on the chain's chunk class and neighbourhood.  A chain's draws
// depend only on its own (seed, chain id, sweep, row, col), so results are
// bit-identical to running the chain alone.
// One tile of a chain for one (chunk class, neighbourhood) variant; not
// inlined so each variant keeps the single-chain kernel's register budget.
// L2_ONLY: the wavefront variant (labels of other tiles written in the same
// launch).
constexpr int kGroupRows = 4 * kBY;   // rows whose uniforms one pass computes (u_s size)

template <int NC, int NB, bool L2_ONLY>
__device__ __noinline__ void batch_tile(const SweepArgs *sa, int row0, int col0, int rows,
                                        uint32_t t, float *Gcol, uint32_t *u_s)
{
    const SweepArgs &a = *sa;
    const int c = col0 + (int)threadIdx.x;
    const int tid = (int)threadIdx.y * kBX + (int)threadIdx.x;
    // per 16 rows: the uniforms first, warp w the Philox blocks of rows
    // 4w .. 4w + 3 (col0 a multiple of 32; one call per 4 sites), then the
    // sites; every thread of the block takes every barrier
    for (int rb = 0; rb < rows; rb += kGroupRows) {
        if (rb + (int)threadIdx.y * kBY < rows)
            block_uniforms(a, row0 + rb + (int)threadIdx.y * kBY, col0, t,
                           u_s + threadIdx.y * kBY * kBX);
        __syncthreads();
        const int re = min(rows, rb + kGroupRows);
        for (int rr = rb; rr < re; rr += kBY)
            pca_site<NC, NB, 0, L2_ONLY>(a, row0 + rr + (int)threadIdx.y, c, t, Gcol,
                                         u_s + (rr - rb) * kBX + tid);
        __syncthreads();   // u_s is free again
    }
}

template <int NB, bool L2_ONLY = false>
__device__ __forceinline__ void batch_dispatch(const SweepArgs *sa, int ncls, int row0, int col0,
                                               int rows, uint32_t t, float *Gcol, uint32_t *u_s)
{
    switch (ncls) {
    case 1: batch_tile<1, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 2: batch_tile<2, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 3: batch_tile<3, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 4: batch_tile<4, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 5: batch_tile<5, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 8: batch_tile<8, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    case 16: batch_tile<16, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    default: batch_tile<32, NB, L2_ONLY>(sa, row0, col0, rows, t, Gcol, u_s); break;
    }
}


__global__ void __launch_bounds__(kThreads, 8) batch_pca_kernel(const SlotDesc *__restrict__ slots,
                                                             const WorkItem *__restrict__ items,
                                                             int n_items, int *grab,
                                                             uint32_t sweep_off)
{
    __shared__ float G_s[32 * kThreads];
    __shared__ __align__(16) uint32_t U_s[kGroupRows * kBX];   // uniforms of 16 tile rows
    __shared__ int s_item;
    __shared__ uint32_t s_t;
    __shared__ int s_go;
    __shared__ SweepArgs s_args;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const int it = atomicAdd(grab, 1);
            s_item = it;
            s_go = 0;
            if (it < n_items) {
                const SlotDesc &d = slots[items[it].slot];
                const uint32_t t = *d.tdev + sweep_off;
                if (d.active && t < *d.budget) {
                    slot_args(d, t, s_args);
                    s_t = t;
                    s_go = 1;
                }
            }
        }
        __syncthreads();
        if (s_item >= n_items)
            return;
        if (!s_go)
            continue;
        const WorkItem w = items[s_item];
        const int ncls = s_args.last_phase;
        if (s_args.sweep_off == 8u)
            batch_dispatch<8>(&s_args, ncls, w.row0, w.col0, w.rows, s_t, G_s + tid, U_s);
        else
            batch_dispatch<4>(&s_args, ncls, w.row0, w.col0, w.rows, s_t, G_s + tid, U_s);
    }
}

// Wavefront form of the batched sweep: nsweeps sweeps of every chain in one
// persistent launch.  Items (sweep k, tile) are taken in increasing order,
// sweep-major, so each item's 3 x 3 neighbourhood of tiles of the same chain
// at sweep k - 1 was taken earlier by a resident block and the waits end
// (each is bounded anyway: error flag).  A chain whose budget ends inside
// the slice skips its remaining items without waiting; no later item waits
// on a skipped one.  done[g.base + tile] counts the sweeps a tile finished
// in this launch (zeroed before it).
__global__ void __launch_bounds__(kThreads, 8) batch_wave_kernel(
    const SlotDesc *__restrict__ slots, const WaveGeom *__restrict__ geom,
    const WaveItem *__restrict__ items, int n_items, int nsweeps, unsigned int *done,
    unsigned int *grab, int *err)
{
    __shared__ float G_s[32 * kThreads];
    __shared__ __align__(16) uint32_t U_s[kGroupRows * kBX];   // uniforms of 16 tile rows
    __shared__ unsigned int s_next;
    __shared__ int s_go;
    __shared__ uint32_t s_t;
    __shared__ SweepArgs s_args;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const unsigned int total = (unsigned int)n_items * (unsigned int)nsweeps;
    if (tid == 0)
        s_next = atomicAdd(grab, 1u);
    __syncthreads();
    unsigned int item = s_next;
    while (item < total) {
        const int k = (int)(item / (unsigned int)n_items);
        const WaveItem w = items[item - (unsigned int)k * (unsigned int)n_items];
        const WaveGeom gm = geom[w.slot];
        const int ty = w.tile / gm.tiles_x;
        const int tx = w.tile - ty * gm.tiles_x;
        __syncthreads();   // everyone has read s_next and is done with s_args
        if (threadIdx.y == 0) {
            if (threadIdx.x == 31)   // no further item once a wait gave up
                s_next = ld_flag(err) ? total : atomicAdd(grab, 1u);
            const SlotDesc &d = slots[w.slot];
            uint32_t t = 0;
            int go = 0;
            if (threadIdx.x == 0 && d.active) {
                t = *d.tdev + (uint32_t)k;
                go = t < *d.budget;
            }
            go = __shfl_sync(0xFFFFFFFFu, go, 0);
            bool ok = true;
            if (go && k > 0 && threadIdx.x < 9) {
                const int yy = ty + (int)threadIdx.x / 3 - 1;
                const int xx = tx + (int)threadIdx.x % 3 - 1;
                if (yy >= 0 && yy < gm.tiles_y && xx >= 0 && xx < gm.tiles_x) {
                    const unsigned int *c = done + gm.base + yy * gm.tiles_x + xx;
                    ok = wait_ge(c, (unsigned int)k, ld_acquire_u32(c), err, kWaitLimitNs);
                }
            }
            if (!ok)
                atomicExch(err, 1);
            if (threadIdx.x == 0) {
                if (go) {
                    slot_args(d, t, s_args);
                    s_t = t;
                }
                s_go = go;
            }
            __syncwarp();
        }
        __syncthreads();
        if (s_go) {
            const int row0 = ty * gm.rows;
            const int rows = min(gm.rows, (s_args.H - row0 + kBY - 1) / kBY * kBY);
            if (s_args.sweep_off == 8u)
                batch_dispatch<8, true>(&s_args, s_args.last_phase, row0, tx * kBX, rows, s_t,
                                        G_s + tid, U_s);
            else
                batch_dispatch<4, true>(&s_args, s_args.last_phase, row0, tx * kBX, rows, s_t,
                                        G_s + tid, U_s);
            __syncthreads();
            if (tid == 0) {
                __threadfence();   // the tile's labels and sums before its counter
                atomicExch(done + gm.base + w.tile, (unsigned int)(k + 1));
            }
        }
        item = s_next;
    }
}

__global__ void batch_advance_kernel(const SlotDesc *slots, int n_slots, uint32_t n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_slots && slots[i].active) {
        const uint32_t t = *slots[i].tdev, b = *slots[i].budget;
        if (t < b)
            *slots[i].tdev = t + (b - t < n ? b - t : n);
    }
}

template <int NC, int NB>
cudaError_t launch_pca_t(const SweepArgs &a, cudaStream_t st)
{
    dim3 block(kBX, kBY);
    dim3 grid((a.W + kBX - 1) / kBX, (a.H + kBY - 1) / kBY);
    if (a.m.norm == 1)
        pca_direct_kernel<NC, NB, 1><<<grid, block, 0, st>>>(a);
    else if (a.m.norm == 2)
        pca_direct_kernel<NC, NB, 2><<<grid, block, 0, st>>>(a);
    else
        pca_direct_kernel<NC, NB, 0><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NC, int NB>
cudaError_t launch_gibbs_t(const SweepArgs &a, int q, cudaStream_t st)
{
    dim3 block(kBX, kBY);
    const int cells_x = (a.W + 1) / 2;
    const int cells_y = NB == 4 ? a.H : (a.H + 1) / 2;
    dim3 grid((cells_x + kBX - 1) / kBX, (cells_y + kBY - 1) / kBY);
    gibbs_cb_kernel<NC, NB><<<grid, block, 0, st>>>(a, q);
    return cudaGetLastError();
}

template <int NB>
cudaError_t dispatch_pca(const SweepArgs &a, cudaStream_t st)
{
    switch (chunk_class(a.m.L)) {
    case 1: return launch_pca_t<1, NB>(a, st);
    case 2: return launch_pca_t<2, NB>(a, st);
    case 3: return launch_pca_t<3, NB>(a, st);
    case 4: return launch_pca_t<4, NB>(a, st);
    case 5: return launch_pca_t<5, NB>(a, st);
    case 8: return launch_pca_t<8, NB>(a, st);
    case 16: return launch_pca_t<16, NB>(a, st);
    default: return launch_pca_t<32, NB>(a, st);
    }
}

template <int NB>
cudaError_t dispatch_gibbs(const SweepArgs &a, int q, cudaStream_t st)
{
    switch (chunk_class(a.m.L)) {
    case 1: return launch_gibbs_t<1, NB>(a, q, st);
    case 2: return launch_gibbs_t<2, NB>(a, q, st);
    case 3: return launch_gibbs_t<3, NB>(a, q, st);
    case 4: return launch_gibbs_t<4, NB>(a, q, st);
    case 5: return launch_gibbs_t<5, NB>(a, q, st);
    case 8: return launch_gibbs_t<8, NB>(a, q, st);
    case 16: return launch_gibbs_t<16, NB>(a, q, st);
    default: return launch_gibbs_t<32, NB>(a, q, st);
    }
}

}  // namespace

int chunk_class(int L)
{
    const int nc = (L + kChunk - 1) / kChunk;
    if (nc <= 5)
        return nc;
    if (nc <= 8)
        return 8;
    if (nc <= 16)
        return 16;
    return 32;
}

namespace {
__global__ void advance_kernel(uint32_t *counter, uint32_t n)
{
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *counter += n;
}
}  // namespace

cudaError_t launch_advance(uint32_t *counter, uint32_t n, cudaStream_t s)
{
    advance_kernel<<<1, 32, 0, s>>>(counter, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_sweep(const SlotDesc *slots, const WorkItem *items, int n_items,
                               int *grab, uint32_t sweep_off, int grid, cudaStream_t s)
{
    batch_pca_kernel<<<grid, dim3(kBX, kBY), 0, s>>>(slots, items, n_items, grab, sweep_off);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(const SlotDesc *slots, int n_slots, uint32_t n, cudaStream_t s)
{
    if (n_slots > 0)
        batch_advance_kernel<<<(n_slots + 127) / 128, 128, 0, s>>>(slots, n_slots, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_wave(const SlotDesc *slots, const WaveGeom *geom, const WaveItem *items,
                              int n_items, int nsweeps, unsigned int *done, unsigned int *grab,
                              int *err, int grid, cudaStream_t s)
{
    const long long total = (long long)n_items * nsweeps;
    if (total <= 0)
        return cudaSuccess;
    if (total >= (1ll << 32))
        return cudaErrorInvalidValue;
    batch_wave_kernel<<<(int)(total < grid ? total : grid), dim3(kBX, kBY), 0, s>>>(
        slots, geom, items, n_items, nsweeps, done, grab, err);
    return cudaGetLastError();
}

int batch_wave_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_wave_kernel, kThreads, 0) !=
        cudaSuccess)
        nb = 1;
    return nb > 0 ? nb : 1;
}

int batch_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_pca_kernel, kThreads, 0) !=
        cudaSuccess)
        nb = 1;
    return nb > 0 ? nb : 1;
}

namespace {

template <int NC, int NB>
cudaError_t launch_wave_t(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int nsweeps,
                          unsigned int *done, unsigned int *grab, int *err, cudaStream_t st)
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
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pca_wave_kernel<NC, NB>, kThreads,
                                                          0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = n;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (a.W + kBX - 1) / kBX;
    const int tiles_y = (a.H + kBY - 1) / kBY;
    const long long items = (long long)tiles_x * tiles_y * nsweeps;
    if (items <= 0)
        return cudaSuccess;
    // at most the resident capacity: every block that takes an item runs
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(items < cap ? items : cap);
    pca_wave_kernel<NC, NB><<<grid, dim3(kBX, kBY), 0, st>>>(a, x0, x1, nsweeps, tiles_x,
                                                            tiles_y, done, grab, err);
    return cudaGetLastError();
}

template <int NB>
cudaError_t dispatch_wave(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int n, unsigned int *done,
                          unsigned int *grab, int *err, cudaStream_t st)
{
    switch (chunk_class(a.m.L)) {
    case 1: return launch_wave_t<1, NB>(a, x0, x1, n, done, grab, err, st);
    case 2: return launch_wave_t<2, NB>(a, x0, x1, n, done, grab, err, st);
    case 3: return launch_wave_t<3, NB>(a, x0, x1, n, done, grab, err, st);
    case 4: return launch_wave_t<4, NB>(a, x0, x1, n, done, grab, err, st);
    case 5: return launch_wave_t<5, NB>(a, x0, x1, n, done, grab, err, st);
    case 8: return launch_wave_t<8, NB>(a, x0, x1, n, done, grab, err, st);
    case 16: return launch_wave_t<16, NB>(a, x0, x1, n, done, grab, err, st);
    default: return launch_wave_t<32, NB>(a, x0, x1, n, done, grab, err, st);
    }
}

}  // namespace

int wave_tiles(int H, int W)
{
    return ((W + kBX - 1) / kBX) * ((H + kBY - 1) / kBY);
}

cudaError_t launch_pca_wave(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int nsweeps,
                            unsigned int *done, unsigned int *grab, int *err, cudaStream_t st)
{
    if (a.m.norm != 0)
        return cudaErrorInvalidValue;   // the wavefront kernel runs the L0 price
    return a.m.nbhd == 8 ? dispatch_wave<8>(a, x0, x1, nsweeps, done, grab, err, st)
                         : dispatch_wave<4>(a, x0, x1, nsweeps, done, grab, err, st);
}

cudaError_t launch_pca_sweep(const SweepArgs &a, cudaStream_t st)
{
    return a.m.nbhd == 8 ? dispatch_pca<8>(a, st) : dispatch_pca<4>(a, st);
}

cudaError_t launch_gibbs_phase(const SweepArgs &a, int q, cudaStream_t st)
{
    return a.m.nbhd == 8 ? dispatch_gibbs<8>(a, q, st) : dispatch_gibbs<4>(a, q, st);
}

}  // namespace pcad
