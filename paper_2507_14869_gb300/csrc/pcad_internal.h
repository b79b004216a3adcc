// Internal declarations shared by the runtime (capi.cu) and the kernels.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/pcaden.h"
#include "pcad_device.cuh"

namespace pcad {

// One sweep (PCA) or one colour phase (Gibbs) over one image.
struct SweepArgs {
    const uint8_t *xin;       // previous labels (PCA) / labels updated in place (Gibbs)
    uint8_t *xout;            // next labels (PCA); unused by Gibbs
    const uint8_t *g;         // observation
    float *acc;               // posterior-mean accumulator (H x W, row stride W)
    unsigned long long *fp64_draws;  // counter of FP64 re-evaluations
    const uint32_t *sweep_base;  // device sweep counter of the chain
    uint64_t seed;
    int H, W, pitch;          // pitch: bytes between label rows (x and g)
    uint32_t sweep_off;       // this update's sweep index = *sweep_base + sweep_off
    uint32_t chain;
    int burn_in;              // sweeps not accumulated
    int last_phase;           // Gibbs: this phase completes the sweep
    int row_off;              // global row of local row 0 (row bands): Philox rows are global
    long long wait_ns;        // limit of each bounded device wait (0: kWaitLimitNs)
    int stall_tile;           // test aid: wavefront tile stall_tile - 1 never publishes (0: off)
    DevModel m;
};

__device__ __forceinline__ uint32_t sweep_index(const SweepArgs &a)
{
    return *a.sweep_base + a.sweep_off;
}

// Accumulate after the k-th completed sweep (k = index + 1) when k > burn_in.
__device__ __forceinline__ bool accumulate_after(const SweepArgs &a, uint32_t t)
{
    return (long long)t + 1 > (long long)a.burn_in;
}

// Inputs of site (r, c) from the labels x at sweep t.  Neighbour order:
// up, down, left, right, then the four diagonals; a neighbour outside the
// image is "missing" (label 1024).
// L2_ONLY: the labels may have been written by other SMs during the same
// launch, so they are read through L2 (ld.global.cg), never from a possibly
// stale L1 line.
template <int NB, bool L2_ONLY = false, bool UNIFORM = true>
__device__ __forceinline__ void load_site(const SweepArgs &a, const uint8_t *__restrict__ x, int r,
                                          int c, uint32_t tag, uint32_t t, SiteIn<NB> &in)
{
    constexpr int dr[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
    constexpr int dc[8] = {0, 0, -1, 1, -1, 1, -1, 1};
    const auto ld = [&](size_t i) -> int { return L2_ONLY ? (int)__ldcg(x + i) : (int)x[i]; };
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int rr = r + dr[j];
        const int cc = c + dc[j];
        const bool inside = rr >= 0 && rr < a.H && cc >= 0 && cc < a.W;
        in.xni[j] = inside ? ld((size_t)rr * a.pitch + cc) : kMissingLabelI;
    }
    const size_t idx = (size_t)r * a.pitch + c;
    in.xi = ld(idx);
    in.g = a.g[idx];
    if constexpr (UNIFORM)
        in.ub = site_u24(a.seed, a.chain, tag, t, (uint32_t)(r + a.row_off), (uint32_t)c);
}

// The uniforms of a 4 x 32 block of sites (rows r0.., columns c0.., c0 a
// multiple of 4): lane l of the calling warp computes the Philox block of row
// r0 + l / 8, columns c0 + 4 (l % 8) .. + 3 (one call serves 4 sites) into
// u_s[32 * (l / 8) + 4 (l % 8) ..], i.e. u_s[32 * row + column].
__device__ __forceinline__ void block_uniforms(const SweepArgs &a, int r0, int c0, uint32_t t,
                                               uint32_t *u_s)
{
    const int l = (int)(threadIdx.x & 31);
    uint32_t o0, o1, o2, o3;
    philox4x32_10((uint32_t)((c0 >> 2) + (l & 7)), (uint32_t)(r0 + a.row_off + (l >> 3)), t,
                  (kTagPCA << 24) | (a.chain & 0xFFFFFFu), (uint32_t)(a.seed & 0xFFFFFFFFull),
                  (uint32_t)(a.seed >> 32), o0, o1, o2, o3);
    reinterpret_cast<uint4 *>(u_s)[l] = make_uint4(o0 >> 8, o1 >> 8, o2 >> 8, o3 >> 8);
}

// *counter += n (one thread).
cudaError_t launch_advance(uint32_t *counter, uint32_t n, cudaStream_t s);

// Number of 8-label chunks rounded up to an instantiated size.
int chunk_class(int L);

// Launch one PCA sweep (xin -> xout) on `stream`.
cudaError_t launch_pca_sweep(const SweepArgs &a, cudaStream_t stream);

// Launch Gibbs colour phase q (0..ncolours-1) in place on a.xin.  When
// a.accumulate is set, the phase must be the last of the sweep.
cudaError_t launch_gibbs_phase(const SweepArgs &a, int q, cudaStream_t stream);

// acc / n -> mean (H x W floats)
cudaError_t launch_mean(const float *acc, float n, float *mean, long count, cudaStream_t s);

// labels (pitched) -> float plane (label units)
cudaError_t launch_labels_to_float(const uint8_t *x, int pitch, int H, int W, float *out,
                                   cudaStream_t s);

// Metrics: est (H x W floats, label units), clean (H x W bytes, contiguous).
// out[0] = PSNR dB, out[1] = SSIM (device doubles).  scratch: >= 8 doubles.
cudaError_t launch_metrics(const float *est, const uint8_t *clean, int H, int W, int L,
                           double *scratch, double *out, cudaStream_t s);

// Validate every label < L (returns count of bad labels into *bad, device int).
cudaError_t launch_check_labels(const uint8_t *x, int pitch, int H, int W, int L, int *bad,
                                cudaStream_t s);

// One chain of a batched or served launch (device memory, filled by the host).
// The state after t sweeps lives in x[t & 1]; *tdev is the chain's sweep
// counter and *budget the sweep count it stops at.
struct SlotDesc {
    const uint8_t *g;
    uint8_t *x[2];
    float *acc;
    uint32_t *tdev;
    const uint32_t *budget;
    unsigned long long *fp64_draws;
    uint64_t seed;
    int H, W, pitch;
    uint32_t chain;
    int burn_in;
    int ncls;          // chunk_class(L)
    int nbhd;
    int active;        // 0: skip (free serving slot)
    DevModel m;
    const float *tctab;   // tensor-core sweep: outside-window chunk sums of the model
};

// Chain descriptor -> sweep arguments of sweep t (the chunk class travels in
// last_phase and the neighbourhood in sweep_off, which the tile code does
// not read).
__device__ __forceinline__ void slot_args(const SlotDesc &d, uint32_t t, SweepArgs &a)
{
    a = SweepArgs{};
    a.xin = d.x[t & 1u];
    a.xout = d.x[(t + 1u) & 1u];
    a.g = d.g;
    a.acc = d.acc;
    a.fp64_draws = d.fp64_draws;
    a.seed = d.seed;
    a.H = d.H;
    a.W = d.W;
    a.pitch = d.pitch;
    a.chain = d.chain;
    a.burn_in = d.burn_in;
    a.last_phase = d.ncls;
    a.sweep_off = (uint32_t)d.nbhd;
    a.m = d.m;
}

// A tile of `rows` x 32 sites of one slot.
struct WorkItem {
    int slot;
    int row0, col0;
    int rows;
};

// One sweep (index *tdev + sweep_off for every slot) over all work items:
// persistent blocks grab items through *grab (zeroed before the launch).
cudaError_t launch_batch_sweep(const SlotDesc *slots, const WorkItem *items, int n_items,
                               int *grab, uint32_t sweep_off, int grid, cudaStream_t s);

// Tile grid of one slot for the wavefront batch kernel: tiles of `rows`
// (a multiple of 4) x 32 sites, row-major; tile j's counter is done[base + j].
struct WaveGeom {
    int base;
    int tiles_x, tiles_y;
    int rows;
};

// One tile of one slot (one sweep of it; the list is repeated per sweep).
struct WaveItem {
    int slot;
    int tile;
};

// nsweeps sweeps (indices *tdev + 0 .. nsweeps - 1 of every active slot,
// each stopping at its budget) in one persistent launch of at most `grid`
// blocks (the resident capacity, batch_wave_blocks_per_sm() x SMs); *grab
// and done[] (every slot's tiles) are zeroed before it.  *err is set when a
// bounded wait for a neighbour tile gives up.
cudaError_t launch_batch_wave(const SlotDesc *slots, const WaveGeom *geom, const WaveItem *items,
                              int n_items, int nsweeps, unsigned int *done, unsigned int *grab,
                              int *err, int grid, cudaStream_t s);
int batch_wave_blocks_per_sm();

// For every active slot: *tdev += min(n, *budget - *tdev).
cudaError_t launch_batch_advance(const SlotDesc *slots, int n_slots, uint32_t n, cudaStream_t s);

// Resident 128-thread blocks per SM of the batch kernel.
int batch_blocks_per_sm();

// Temporally blocked PCA: k (1..8) sweeps per launch from the plane behind
// xmap into a.xout; sweep indices *a.sweep_base + a.sweep_off + 0..k-1.
// *err is set when a bounded wait for the tile loads gives up.
cudaError_t launch_pca_tb(const CUtensorMap &xmap, const CUtensorMap &gmap, const SweepArgs &a,
                          int k, int *err, cudaStream_t s);

// Posterior energy H(x) = pair_c * pair_sum + data term, from the integer
// sums of energy.cu: data term = data_sum / two_s2 (Gaussian),
// lf_same * (n_sites - data_sum) + lf_diff * data_sum (flip) or 0 (none).
struct EnergyCoef {
    int potts, T, gauss, nbhd;
    int none;            // no likelihood: data term 0
    double pair_c;       // -c_P (Potts) or c_T (truncated linear)
    double two_s2;       // 2 sigma^2
    double lf_same;      // -ln(1 - p)
    double lf_diff;      // -ln p
    unsigned long long n_sites;
};
EnergyCoef energy_coef(const pcad_model &m, long n_sites);

// Minimum-energy tracking state (device pointers; trace == nullptr: off).
struct EnergyTrack {
    double *trace;                  // H after each tracked sweep
    int cap;
    unsigned int *n;                // entries recorded
    double *best;                   // lowest H so far (+inf initially)
    unsigned long long *best_sweep; // completed sweeps when it was reached
    int *flag;                      // this sweep set a new minimum
    uint8_t *xb;                    // the lowest-energy state (same pitch as x)
};

// sums (2 x u64, zero on entry, zero again on return) <- integer sums of
// labelling x; out[0..2] <- H, pair sum, data sum (when out != nullptr); with
// tracking, record H as the energy after sweep *tdev + sweep_off.
cudaError_t launch_energy(const uint8_t *x, const uint8_t *g, int H, int W, int pitch,
                          const EnergyCoef &k, unsigned long long *sums, double *out,
                          const EnergyTrack &tr, const uint32_t *tdev, uint32_t sweep_off,
                          cudaStream_t s);

// Wavefront lazy-PCA: nsweeps sweeps in one persistent launch from plane x0
// (sweep index *a.sweep_base + a.sweep_off + k reads x[k & 1] of {x0, x1});
// a tile starts sweep k once the 3 x 3 neighbouring tiles finished sweep
// k - 1.  done (one counter per 4 x 32 tile) and grab (the work counter)
// must be zero on entry; *err is set if a bounded dependency wait gives up.
cudaError_t launch_pca_wave(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int nsweeps,
                            unsigned int *done, unsigned int *grab, int *err, cudaStream_t s);
int wave_tiles(int H, int W);

// Tensor-core lazy-PCA sweeps (windowed prior sums by tcgen05.mma), run as
// a wavefront like launch_pca_wave: nsweeps sweeps from plane x0, done (one
// counter per 4 x 32 tile) and grab zero on entry.  Eligible models: L in
// [kTcMinLabels, 256], truncation T <= kTcMaxT (the 128-label window then
// holds every tent of a 64-bin histogram), L0 price.  *err is set (1: a
// bounded wait gave up, 2: misaligned shared memory).
constexpr int kTcMinLabels = 64;
constexpr int kTcMaxT = 33;
bool pca_tc_eligible(const DevModel &m);
// budget (optional): sweeps with index >= *budget are skipped.  par_from_t:
// x0 / x1 are the planes of even / odd sweep indices (else of sweeps 0 / 1
// of the launch).
cudaError_t launch_pca_tc(const SweepArgs &a, uint8_t *x0, uint8_t *x1, int nsweeps,
                          unsigned int *done, unsigned int *grab, int *err, cudaStream_t s,
                          const uint32_t *budget = nullptr, bool par_from_t = false);
// nsweeps checkerboard Gibbs sweeps (4-neighbourhood, 2 colour phases each)
// of one chain in place on x, on the same tensor-core kernel: 8 x 32 tiles,
// one counter per tile in done[] (at least ceil(H / 8) * ceil(W / 32)
// zeroed entries), grab zeroed.
cudaError_t launch_gibbs_tc(const SweepArgs &a, uint8_t *x, int nsweeps, unsigned int *done,
                            unsigned int *grab, int *err, cudaStream_t s);

// Models the automatic kernel choice gives the tensor-core sweep: eligible
// and L >= kTcAutoLabels (on GB300 it measured 1.4-1.6x the CUDA-core
// kernels at L = 256, level at L = 128 and slower below: the window's work
// does not shrink with L).
constexpr int kTcAutoLabels = 192;
bool pca_tc_auto(const DevModel &m);

// The outside-window chunk sums of a model, as the batched tensor-core
// sweep reads them: tc_table_floats(L) floats (16-byte aligned), written by
// launch_tc_table.
int tc_table_floats(int L);
cudaError_t launch_tc_table(const DevModel &m, float *out, cudaStream_t s);

// The CUDA-core windowed sweep (the tensor-core sweep's weights, tent sums
// from a byte table over each site's hull of labels, outside chunks from
// ftab = launch_tc_table's table): one sweep a.xin -> a.xout, or (x0 set)
// from the plane of the sweep index's parity (x0 even, x1 odd) to the
// other, skipped at or past *budget (budget optional).  Models with
// kWinMinLabels <= L <= 256, 1 <= T <= kTcMaxT, nbhd T <= 255, the L0 price.
constexpr int kWinMinLabels = 9;
// The automatic kernel choice (chains, batches, the server) takes the
// windowed sweeps from this many labels on (below, the small-label or
// per-sweep CUDA-core kernels measured as fast or faster on GB300).
constexpr int kWinAutoMinLabels = 32;
bool pca_win_eligible(const DevModel &m);
cudaError_t launch_pca_win(const SweepArgs &a, const float *ftab, cudaStream_t s,
                           uint8_t *x0 = nullptr, uint8_t *x1 = nullptr,
                           const uint32_t *budget = nullptr);
// The windowed sweep as one persistent wavefront launch of nsweeps sweeps
// (planes x0 for even, x1 for odd sweeps of the launch, or by the parity of
// the sweep index with par_from_t): tiles of 4 x 32 sites, counters done[]
// (ceil(H / 4) * ceil(W / 32) zeroed entries), grab zeroed, *err set when a
// bounded dependency wait gave up; budget (optional): sweeps at or past
// *budget are skipped.
cudaError_t launch_pca_winw(const SweepArgs &a, const float *ftab, uint8_t *x0, uint8_t *x1,
                            int nsweeps, unsigned int *done, unsigned int *grab, int *err,
                            cudaStream_t s, const uint32_t *budget = nullptr,
                            bool par_from_t = false);
// nsweeps checkerboard Gibbs sweeps in place on x with the windowed draw as
// one wavefront launch of colour phases: tiles of 64 columns x 4 (8 for 8
// neighbours) rows, counters done[] (one zeroed entry per tile), grab
// zeroed, *err as launch_pca_winw's.
cudaError_t launch_gibbs_winw(const SweepArgs &a, const float *ftab, uint8_t *x, int nsweeps,
                              unsigned int *done, unsigned int *grab, int *err, cudaStream_t s);
// Checkerboard Gibbs colour phase q (0..nbhd/2 - 1) in place on a.xin with
// the windowed draw; a.last_phase: accumulate the cells after it.
cudaError_t launch_gibbs_win(const SweepArgs &a, int q, const float *ftab, cudaStream_t s);

// Batched tensor-core sweeps: nsweeps sweeps of every slot listed in items
// (tiles of 4 rows x 32 sites of the slot's grid in geom, rows = 4) in one
// wavefront launch; slot s runs sweeps t_arr[s] + k while below
// budget_arr[s] (the arrays behind its descriptor's tdev and budget).
// Every slot of a launch has truncation T, neighbourhood nbhd, L % 8 != 0
// exactly when lmask, at most nc_max chunks, a tensor-core eligible model
// and its table in tctab.  done (every tile) and grab zero on entry.
cudaError_t launch_batch_tc(const SlotDesc *slots, const uint32_t *t_arr,
                            const uint32_t *budget_arr, const WaveGeom *geom,
                            const WaveItem *items, int n_items, int nsweeps, int T, int nbhd,
                            bool lmask, int nc_max, unsigned int *done, unsigned int *grab,
                            int *err, cudaStream_t s);

// TMA descriptor of a uint8 plane (box 96 x 48); false if the driver refuses.
bool encode_plane_map(CUtensorMap *map, void *base, int H, int W, int pitch);

// Small label counts (kSmallMinLabels <= L <= kSmallMaxLabels, gam <= 0,
// alpha <= 0, L0 price): one-launch-per-sweep kernel with the prior sums of
// all labels from a pair table (ptab_words() words, built by launch_ptab for
// the truncation T; the model's ptab points at it).
constexpr int kSmallMinLabels = 3;
constexpr int kSmallMaxLabels = 16;
// From this many sites a small-label chain sweeps on TMA-loaded tiles
// (launch_pca_small_tma) instead of 16 x 32 staged tiles.
constexpr long long kSmallTmaMinSites = 1ll << 23;
int ptab_words();
cudaError_t launch_ptab(int T, uint32_t *out, cudaStream_t s);
bool pca_small_eligible(const DevModel &m);
// One small-label sweep a.xin -> a.xout on TMA-loaded tiles (persistent,
// double-buffered): xmap, gmap the maps of a.xin and of the observation
// (encode_plane_map); the data term from a table, so observations g < L; a
// bounded wait that runs out sets *err.
cudaError_t launch_pca_small_tma(const CUtensorMap &xmap, const CUtensorMap &gmap,
                                 const SweepArgs &a, int *err, cudaStream_t s);
// x0 / x1 (optional): the planes of even / odd sweep indices, used in place of
// a.xin / a.xout; budget (optional): sweeps with index >= *budget are skipped;
// aq: the data term from a table of the observations g < 16 (observations
// checked against L: chains use it).
cudaError_t launch_pca_small(const SweepArgs &a, cudaStream_t s, uint8_t *x0 = nullptr,
                             uint8_t *x1 = nullptr, const uint32_t *budget = nullptr,
                             bool aq = false);

// Whole chains of small two-label images in one CTA (state in shared
// memory): L = 2, 4 or 8 neighbours, the thresholds table m.btab built, at
// most 4096 quads of 4 sites (H * ceil(W / 4)) and 200 KB of shared memory.
// nsweeps sweeps from plane x_in (the current state) in one launch; the
// final state goes to x_out (x_in itself for Gibbs, the other plane when
// nsweeps is odd for PCA).
bool resident_eligible(const DevModel &m, int H, int W);
// Two-label PCA sweep a.xin -> a.xout with the threshold table m.btab, one
// launch per sweep (any image size; the planes read and written as words).
// x0 / x1 (optional): the planes of even / odd sweep indices, used in place
// of a.xin / a.xout; budget (optional): sweeps with index >= *budget are
// skipped.
bool binary_eligible(const DevModel &m);
cudaError_t launch_pca_binary(const SweepArgs &a, cudaStream_t s, uint8_t *x0 = nullptr,
                              uint8_t *x1 = nullptr, const uint32_t *budget = nullptr);
// AUTO takes it for two-label images of this many sites and more.
constexpr long long kBinaryAutoMinSites = 1ll << 18;
cudaError_t launch_resident(const SweepArgs &a, const uint8_t *x_in, uint8_t *x_out, int nsweeps,
                            bool gibbs, cudaStream_t s);
// The two-label draw thresholds of every site configuration (L = 2), from
// the model's FP32 draw and FP64 re-draw; btab_bytes() of device memory.
int btab_bytes();
cudaError_t launch_btab(const DevModel &m, uint4 *out, cudaStream_t s);
// Batched form: whether a two-label chain of this size runs resident, its
// shared memory, and one launch of `count` chains (slot indices idx[0..count),
// all with nbhd neighbours, tables at tabs + b * btab_bytes()) for n sweeps
// below each slot's budget, smem the largest of their resident_smem_bytes.
bool resident_fits(int L, int nbhd, int H, int W);
int resident_smem_bytes(int nbhd, int H, int W);
cudaError_t launch_resident_batch(const SlotDesc *slots, const int *idx, const uint4 *tabs,
                                  int count, int nbhd, int n, int smem, cudaStream_t s);

// Largest row offset of a band chain (Philox rows are 32-bit).
constexpr int kMaxRowOffset = 1 << 30;

// Accessors of a chain for the row-band runner: the plane holding the
// current state (stream-ordered: valid for work queued after the chain's
// last run), its row pitch and the chain's stream.
uint8_t *chain_state(pcad_chain *ch);
int chain_pitch(const pcad_chain *ch);
cudaStream_t chain_stream(const pcad_chain *ch);

// Model validation, host tables and error reporting shared by the entry points.
pcad_status check_model(const pcad_model *m);
void model_tables(const pcad_model &m, double *ta64, std::vector<double> &pr64, DevModel &dm);
pcad_status set_error(pcad_status st, const char *msg);

}  // namespace pcad
