// Batched chains and the continuous-batching server.
//
// Both keep one SlotDesc per chain in device memory (pointers, size, model,
// the chain's own sweep counter and sweep budget) and a work list of tiles
// (rows x 32 sites of one chain), and advance every active chain by one sweep
// per launch of the persistent batch kernel.  A chain's state after t sweeps
// lives in x[t & 1] and its draws are keyed by its own (seed, chain id,
// sweep, row, col), so a chain gives the same labels whatever else shares
// the launch.
//
// pcad_batch: a fixed set of chains run in lockstep; sweeps are issued in
// slices of 8, 16 or 32 sweeps captured once into a CUDA graph (a wavefront
// slice is one persistent launch, so the slice length is the number of
// sweeps per launch).  At creation an optional autotuner times the tile
// height, the work-list order and the slice length on the batch itself and
// caches the choice per batch signature.
//
// pcad_server: requests of different sizes, models and sweep budgets are
// admitted into free slots while the HBM budget allows, run slice by slice
// next to whatever else is active, and leave when their budget is spent; the
// caller collects results with pcad_server_poll.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "pcad_internal.h"

using namespace pcad;

namespace {

constexpr int kSlice = 16;        // default sweeps per batch slice (one graph)
constexpr int kMaxSlice = 32;     // longest slice (sizes the per-sweep work counters)
constexpr int kOrderWave = 2;     // batch work order: one wavefront launch per slice
// Tile height of the server's wavefront launches: 4 rows keep the slice's
// critical path (one tile after another through its sweeps) short when
// few tiles are active; 8 rows halve the per-tile synchronisation once the
// active set has at least 4 tiles of 4 rows per resident block (measured on
// single requests of 300^2..1376^2 and on a 50 req/s mix).
constexpr int kServeTallTiles = 4;
// SRPT server: least estimated GPU time of a full slice of the run set.
constexpr double kMinSliceSeconds = 1e-3;
constexpr size_t kAlign = 256;
constexpr int kTableBytes = 4096;  // 511 doubles

size_t al(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

#define B_TRY(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return set_error(PCAD_ECUDA, cudaGetErrorString(e_));                     \
    } while (0)

pcad_status check_job(const pcad_job &j)
{
    if (!j.g_host)
        return set_error(PCAD_EINVAL, "job observation is NULL");
    if (j.H < 1 || j.W < 1 || j.H > 65535 || j.W > 65535 || j.g_pitch < j.W)
        return set_error(PCAD_EINVAL, "job size or pitch outside the limits");
    if (j.burn_in < 0 || j.chain_id >= (1u << 24))
        return set_error(PCAD_EINVAL, "job burn_in < 0 or chain id >= 2^24");
    pcad_status st = check_model(&j.model);
    if (st != PCAD_OK)
        return st;
    if (j.model.sampler != PCAD_SAMPLER_PCA)
        return set_error(PCAD_EINVAL, "batches and the server run the PCA sampler");
    if (j.model.inertia_norm != 0 && j.model.L > 2 && j.model.inertia > 0.0f)
        return set_error(PCAD_EINVAL, "batches and the server run the L0 inertia price only");
    // observations are labels, as for chains: the two-label and small-label
    // kernels index their tables by g
    if (j.model.L < 256) {
        for (int r = 0; r < j.H; ++r) {
            const uint8_t *row = j.g_host + (size_t)r * j.g_pitch;
            uint8_t mx = 0;
            for (int c = 0; c < j.W; ++c)
                mx = row[c] > mx ? row[c] : mx;
            if (mx >= j.model.L)
                return set_error(PCAD_EINVAL, "observed labels are >= L");
        }
    }
    return PCAD_OK;
}

// Per-chain device layout inside one allocation.
struct SlotMem {
    size_t x0, x1, g, acc, ta, pr, tab, end;   // tab == end: no tensor-core table
};

// Whether a model's slot keeps an outside-chunk table: the models of the
// batched tensor-core sweep (the automatic kernel rule of the chains) and
// those the windowed sweep takes when their image is large.
bool model_tc(const pcad_model &m)
{
    double ta64[511];
    std::vector<double> pr64;
    DevModel dm{};
    model_tables(m, ta64, pr64, dm);
    return m.sampler == PCAD_SAMPLER_PCA && (pca_tc_auto(dm) || pca_win_eligible(dm));
}

SlotMem slot_layout(int H, int W, int pitch, size_t pr_bytes, size_t tab_bytes, size_t base)
{
    SlotMem s;
    const size_t plane = al((size_t)pitch * H);
    s.x0 = base;
    s.x1 = s.x0 + plane;
    s.g = s.x1 + plane;
    s.acc = s.g + plane;
    s.ta = s.acc + al((size_t)H * W * sizeof(float));
    s.pr = s.ta + kTableBytes;
    s.tab = s.pr + al(pr_bytes);
    s.end = s.tab + al(tab_bytes);
    return s;
}

SlotMem job_layout(const pcad_job &j, int pitch, size_t base)
{
    const int T = j.model.pair == PCAD_PAIR_POTTS ? 1 : j.model.pair_T;
    const size_t tab = model_tc(j.model) ? (size_t)tc_table_floats(j.model.L) * sizeof(float) : 0;
    return slot_layout(j.H, j.W, pitch, (size_t)(j.model.nbhd * T + 1) * sizeof(double), tab,
                       base);
}

size_t slot_bytes(const pcad_job &j)
{
    return job_layout(j, (int)((j.W + 15) / 16 * 16), 0).end;
}

// Build a slot: copy g, x0 <- g, acc <- 0, tables; fill the descriptor.
pcad_status init_slot(const pcad_job &j, char *base, const SlotMem &sm, int pitch,
                      uint32_t *tdev, const uint32_t *budget, unsigned long long *fp64,
                      cudaStream_t s, SlotDesc &d)
{
    double ta64[511];
    std::vector<double> pr64;
    DevModel dm{};
    model_tables(j.model, ta64, pr64, dm);
    B_TRY(cudaMemcpy2DAsync(base + sm.g, pitch, j.g_host, j.g_pitch, j.W, j.H,
                            cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpy2DAsync(base + sm.x0, pitch, base + sm.g, pitch, j.W, j.H,
                            cudaMemcpyDeviceToDevice, s));
    B_TRY(cudaMemsetAsync(base + sm.acc, 0, (size_t)j.H * j.W * sizeof(float), s));
    B_TRY(cudaMemcpyAsync(base + sm.ta, ta64, sizeof(ta64), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(base + sm.pr, pr64.data(), pr64.size() * sizeof(double),
                          cudaMemcpyHostToDevice, s));
    dm.ta64 = (const double *)(base + sm.ta);
    dm.pr64 = (const double *)(base + sm.pr);
    d = SlotDesc{};
    d.g = (const uint8_t *)(base + sm.g);
    d.x[0] = (uint8_t *)(base + sm.x0);
    d.x[1] = (uint8_t *)(base + sm.x1);
    d.acc = (float *)(base + sm.acc);
    d.tdev = tdev;
    d.budget = budget;
    d.fp64_draws = fp64;
    d.seed = j.seed;
    d.H = j.H;
    d.W = j.W;
    d.pitch = pitch;
    d.chain = j.chain_id;
    d.burn_in = j.burn_in;
    d.ncls = chunk_class(j.model.L);
    d.nbhd = j.model.nbhd;
    d.active = 1;
    d.m = dm;
    d.tctab = nullptr;
    if (sm.end > sm.tab && (pca_tc_auto(dm) || pca_win_eligible(dm))) {
        d.tctab = (const float *)(base + sm.tab);
        B_TRY(launch_tc_table(dm, (float *)(base + sm.tab), s));
    }
    return PCAD_OK;
}

// Work list: tiles of `rows` x 32; LPT order puts the costliest tiles first.
std::vector<WorkItem> make_items(const std::vector<SlotDesc> &d, const std::vector<int> &active,
                                 int rows, bool lpt)
{
    std::vector<WorkItem> items;
    std::vector<long> cost;
    for (int i : active) {
        for (int r0 = 0; r0 < d[i].H; r0 += rows)
            for (int c0 = 0; c0 < d[i].W; c0 += 32) {
                items.push_back(WorkItem{i, r0, c0, std::min(rows, ((d[i].H - r0 + 3) / 4) * 4)});
                cost.push_back((long)d[i].ncls * 8 + 4);
            }
    }
    if (lpt) {
        std::vector<size_t> idx(items.size());
        for (size_t k = 0; k < idx.size(); ++k)
            idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
            return cost[a] * items[a].rows > cost[b] * items[b].rows;
        });
        std::vector<WorkItem> out(items.size());
        for (size_t k = 0; k < idx.size(); ++k)
            out[k] = items[idx[k]];
        items.swap(out);
    }
    return items;
}

int grid_size()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * batch_blocks_per_sm();
}

// Wavefront work list in device memory: per-slot tile grids, the tiles of
// one sweep and one done counter per tile, in one allocation (regrown).
struct WaveBuf {
    void *mem = nullptr;
    size_t cap = 0;
    WaveGeom *geom = nullptr;
    WaveItem *items = nullptr;
    unsigned int *done = nullptr;
    int n_items = 0, n_tiles = 0;
};

// Fill `wb` for the given slots: slots in decreasing per-site cost, each
// slot's tiles row-major, so a tile's neighbours are taken shortly before
// or after it.  geom has one entry per slot of `d` (unused ones empty).
pcad_status wave_upload(WaveBuf &wb, const std::vector<SlotDesc> &d, std::vector<int> active,
                        int rows, cudaStream_t st)
{
    std::stable_sort(active.begin(), active.end(),
                     [&](int a, int b) { return d[a].ncls > d[b].ncls; });
    std::vector<WaveGeom> geom(d.size(), WaveGeom{0, 0, 0, rows});
    std::vector<WaveItem> items;
    long tiles = 0;
    for (int i : active) {
        WaveGeom g{(int)tiles, (d[i].W + 31) / 32, (d[i].H + rows - 1) / rows, rows};
        geom[i] = g;
        for (int j = 0; j < g.tiles_x * g.tiles_y; ++j)
            items.push_back(WaveItem{i, j});
        tiles += (long)g.tiles_x * g.tiles_y;
        if (tiles > (1l << 30))
            return set_error(PCAD_EINVAL, "too many tiles for one wavefront launch");
    }
    const size_t need = al(geom.size() * sizeof(WaveGeom)) + al(items.size() * sizeof(WaveItem)) +
                        al((size_t)tiles * sizeof(unsigned int));
    if (need > wb.cap) {
        if (wb.mem)
            B_TRY(cudaFreeAsync(wb.mem, st));
        wb.mem = nullptr;
        wb.cap = std::max(need, 2 * wb.cap);
        B_TRY(cudaMallocAsync(&wb.mem, wb.cap, st));
    }
    char *p = (char *)wb.mem;
    wb.geom = (WaveGeom *)p;
    p += al(geom.size() * sizeof(WaveGeom));
    wb.items = (WaveItem *)p;
    p += al(items.size() * sizeof(WaveItem));
    wb.done = (unsigned int *)p;
    B_TRY(cudaMemcpyAsync(wb.geom, geom.data(), geom.size() * sizeof(WaveGeom),
                          cudaMemcpyHostToDevice, st));
    if (!items.empty())
        B_TRY(cudaMemcpyAsync(wb.items, items.data(), items.size() * sizeof(WaveItem),
                              cudaMemcpyHostToDevice, st));
    wb.n_items = (int)items.size();
    wb.n_tiles = (int)tiles;
    return PCAD_OK;
}

// One wavefront launch of n sweeps over the list (counters zeroed first).
pcad_status wave_issue(const WaveBuf &wb, const SlotDesc *slots, int n, int *grab, int *err,
                       int grid, cudaStream_t st)
{
    B_TRY(cudaMemsetAsync(grab, 0, sizeof(int), st));
    B_TRY(cudaMemsetAsync(wb.done, 0, (size_t)wb.n_tiles * sizeof(unsigned int), st));
    B_TRY(launch_batch_wave(slots, wb.geom, wb.items, wb.n_items, n, wb.done,
                            (unsigned int *)grab, err, grid, st));
    return PCAD_OK;
}

int wave_grid()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * batch_wave_blocks_per_sm();
}

// Slots on the tensor-core sweep.  Large images (at least kTcBigTiles tiles
// of 4 x 32 sites, two per resident warpgroup) fill the GPU alone and run
// the one-chain kernel, one launch per slot and slice (its arguments are
// baked into the launch, its planes follow the device sweep counter); the
// others share one batched launch per (truncation, neighbourhood,
// L % 8 != 0) group, where the per-item staging of a chain's arguments
// costs less than the idle GPU of a small one-chain launch.
constexpr long kTcBigTiles = 1216;

struct TcGroup {
    int T = 0, nbhd = 0;
    bool lmask = false;
    int nc_max = 0;
    WaveBuf wb;
};

// Chains the windowed sweep takes run it as their own launches, as the
// chain API does for such images: from kWinBigBlocks blocks of 4 x 32 sites
// per multiprocessor one launch per sweep, from kWinWaveBlocks one
// wavefront launch per slice (on GB300 1.3-1.5x the tensor-core sweep
// there); planes by the device sweep counter, budget-aware.
constexpr long kWinBigBlocks = 100;
constexpr long kWinWaveBlocks = 8;

struct TcSet {
    std::vector<TcGroup> groups;
    std::vector<int> win;          // slots on the windowed sweep, launched one at a time
    std::vector<int> winw;         // slots on the windowed wavefront, launched one at a time
    std::vector<int> big;          // slots launched one at a time
    unsigned int *ctr = nullptr;   // their tile counters and work counter (regrown)
    long ctr_cap = 0;
};

// Split `active` into the tensor-core slots (those with a table: large ones
// one by one, the others by group) and the rest (returned).
pcad_status tc_set_build(TcSet &ts, const std::vector<SlotDesc> &d,
                         const std::vector<int> &active, std::vector<int> &rest, cudaStream_t st)
{
    std::vector<std::vector<int>> members(ts.groups.size());
    rest.clear();
    ts.big.clear();
    ts.win.clear();
    ts.winw.clear();
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long big_tiles = 0;
    for (int i : active) {
        if (!d[i].tctab) {
            rest.push_back(i);
            continue;
        }
        const long tiles = (long)((d[i].W + 31) / 32) * ((d[i].H + 3) / 4);
        if (sms > 0 && tiles >= kWinWaveBlocks * sms && (d[i].H + 3) / 4 <= 65535 &&
            pca_win_eligible(d[i].m) && d[i].m.L >= kWinAutoMinLabels) {
            if (tiles >= kWinBigBlocks * sms) {
                ts.win.push_back(i);
            } else {
                ts.winw.push_back(i);
                big_tiles = std::max(big_tiles, tiles);
            }
            continue;
        }
        if (!pca_tc_auto(d[i].m)) {   // a table for the windowed sweep only
            rest.push_back(i);
            continue;
        }
        if (tiles >= kTcBigTiles) {
            ts.big.push_back(i);
            big_tiles = std::max(big_tiles, tiles);
            continue;
        }
        const bool lm = (d[i].m.L % kChunk) != 0;
        size_t gi = 0;
        while (gi < ts.groups.size() && !(ts.groups[gi].T == d[i].m.T &&
                                          ts.groups[gi].nbhd == d[i].nbhd &&
                                          ts.groups[gi].lmask == lm))
            ++gi;
        if (gi == ts.groups.size()) {
            ts.groups.emplace_back();
            ts.groups.back().T = d[i].m.T;
            ts.groups.back().nbhd = d[i].nbhd;
            ts.groups.back().lmask = lm;
            members.emplace_back();
        }
        members[gi].push_back(i);
    }
    for (size_t gi = 0; gi < ts.groups.size(); ++gi) {
        int ncm = 1;
        for (int i : members[gi])
            ncm = std::max(ncm, (d[i].m.L + kChunk - 1) / kChunk);
        ts.groups[gi].nc_max = ncm;
        pcad_status s = wave_upload(ts.groups[gi].wb, d, members[gi], 4, st);
        if (s != PCAD_OK)
            return s;
    }
    if (big_tiles + 1 > ts.ctr_cap) {
        if (ts.ctr)
            B_TRY(cudaFreeAsync(ts.ctr, st));
        ts.ctr = nullptr;
        ts.ctr_cap = std::max(big_tiles + 1, 2 * ts.ctr_cap);
        B_TRY(cudaMallocAsync((void **)&ts.ctr, (size_t)ts.ctr_cap * sizeof(unsigned int), st));
    }
    return PCAD_OK;
}

// The tensor-core launches of n sweeps: one per large slot (desc: the host
// copies of the descriptors), one per non-empty group.
pcad_status tc_set_issue(const TcSet &ts, const std::vector<SlotDesc> &desc,
                         const SlotDesc *slots, const uint32_t *t_arr, const uint32_t *budget_arr,
                         int n, int *grab, int *err, cudaStream_t st)
{
    for (int i : ts.win) {
        const SlotDesc &d = desc[i];
        SweepArgs a{};
        a.g = d.g;
        a.acc = d.acc;
        a.fp64_draws = d.fp64_draws;
        a.sweep_base = d.tdev;
        a.seed = d.seed;
        a.H = d.H;
        a.W = d.W;
        a.pitch = d.pitch;
        a.chain = d.chain;
        a.burn_in = d.burn_in;
        a.m = d.m;
        for (int k = 0; k < n; ++k) {
            a.sweep_off = (uint32_t)k;
            B_TRY(launch_pca_win(a, d.tctab, st, d.x[0], d.x[1], d.budget));
        }
    }
    for (int i : ts.winw) {
        const SlotDesc &d = desc[i];
        SweepArgs a{};
        a.g = d.g;
        a.acc = d.acc;
        a.fp64_draws = d.fp64_draws;
        a.sweep_base = d.tdev;
        a.seed = d.seed;
        a.H = d.H;
        a.W = d.W;
        a.pitch = d.pitch;
        a.chain = d.chain;
        a.burn_in = d.burn_in;
        a.m = d.m;
        const size_t tiles = (size_t)((d.W + 31) / 32) * ((d.H + 3) / 4);
        B_TRY(cudaMemsetAsync(ts.ctr, 0, (tiles + 1) * sizeof(unsigned int), st));
        B_TRY(launch_pca_winw(a, d.tctab, d.x[0], d.x[1], n, ts.ctr, ts.ctr + tiles, err, st,
                              d.budget, true));
    }
    for (int i : ts.big) {
        const SlotDesc &d = desc[i];
        SweepArgs a{};
        a.g = d.g;
        a.acc = d.acc;
        a.fp64_draws = d.fp64_draws;
        a.sweep_base = d.tdev;
        a.seed = d.seed;
        a.H = d.H;
        a.W = d.W;
        a.pitch = d.pitch;
        a.chain = d.chain;
        a.burn_in = d.burn_in;
        a.m = d.m;
        const size_t tiles = (size_t)((d.W + 31) / 32) * ((d.H + 3) / 4);
        B_TRY(cudaMemsetAsync(ts.ctr, 0, (tiles + 1) * sizeof(unsigned int), st));
        B_TRY(launch_pca_tc(a, d.x[0], d.x[1], n, ts.ctr, ts.ctr + tiles, err, st, d.budget,
                            true));
    }
    for (const TcGroup &g : ts.groups) {
        if (g.wb.n_items == 0)
            continue;
        B_TRY(cudaMemsetAsync(grab, 0, sizeof(int), st));
        B_TRY(cudaMemsetAsync(g.wb.done, 0, (size_t)g.wb.n_tiles * sizeof(unsigned int), st));
        B_TRY(launch_batch_tc(slots, t_arr, budget_arr, g.wb.geom, g.wb.items, g.wb.n_items, n,
                              g.T, g.nbhd, g.lmask, g.nc_max, g.wb.done, (unsigned int *)grab,
                              err, st));
    }
    return PCAD_OK;
}

// Large chains with small-label models (3 <= L <= 16, c >= 0) run the
// small-label kernel, one launch per chain and sweep: a chain of at least
// kSmallBigTiles tiles of 16 x 32 sites fills the GPU alone, and the
// small-label kernel measured about twice the batched CUDA-core kernel's
// rate at L = 16 on GB300.  Planes follow the device sweep counter and each
// launch skips sweeps at or past the chain's budget, so a captured slice
// stays valid for any start.  One pair table per distinct truncation T.
constexpr long kSmallBigTiles = 1216;
// Two-label chains of at least kBinBigSites sites (one wave of the
// two-label sweep's 16 x 128-site tiles at 8 blocks per SM) run the
// two-label sweep the same way, each with its own threshold table.
constexpr long kBinBigSites = 1216L * 16 * 128;

struct SmallSet {
    std::vector<int> big;          // slots launched one at a time
    std::vector<int> table_T;      // T of each pair table
    uint32_t *tables = nullptr;    // the pair tables, ptab_words() words each
    size_t cap = 0;                // tables allocated
    std::vector<int> bin;          // two-label slots launched one at a time
    uint4 *btabs = nullptr;        // their threshold tables, same order
    size_t bcap = 0;               // tables allocated
};

size_t bin_tab_entries()
{
    return (size_t)btab_bytes() / sizeof(uint4);
}

// Split `in` into the small-label slots launched one at a time and the rest.
pcad_status small_set_build(SmallSet &ss, const std::vector<SlotDesc> &d,
                            const std::vector<int> &in, std::vector<int> &rest, cudaStream_t st)
{
    ss.big.clear();
    ss.table_T.clear();
    ss.bin.clear();
    rest.clear();
    for (int i : in) {
        DevModel m = d[i].m;
        m.ptab = reinterpret_cast<const uint32_t *>(&ss);   // eligibility of the model only
        m.btab = reinterpret_cast<const uint4 *>(&ss);
        const long tiles = (long)((d[i].W + 31) / 32) * ((d[i].H + 15) / 16);
        if (tiles >= kSmallBigTiles && pca_small_eligible(m)) {
            ss.big.push_back(i);
            if (std::find(ss.table_T.begin(), ss.table_T.end(), m.T) == ss.table_T.end())
                ss.table_T.push_back(m.T);
        } else if ((long)d[i].H * d[i].W >= kBinBigSites && binary_eligible(m)) {
            ss.bin.push_back(i);
        } else {
            rest.push_back(i);
        }
    }
    if (ss.bin.size() > ss.bcap) {
        if (ss.btabs)
            B_TRY(cudaFreeAsync(ss.btabs, st));
        ss.btabs = nullptr;
        ss.bcap = std::max(ss.bin.size(), 2 * ss.bcap);
        B_TRY(cudaMallocAsync((void **)&ss.btabs, ss.bcap * bin_tab_entries() * sizeof(uint4), st));
    }
    for (size_t p = 0; p < ss.bin.size(); ++p)
        B_TRY(launch_btab(d[ss.bin[p]].m, ss.btabs + p * bin_tab_entries(), st));
    if (ss.table_T.size() > ss.cap) {
        if (ss.tables)
            B_TRY(cudaFreeAsync(ss.tables, st));
        ss.tables = nullptr;
        ss.cap = std::max(ss.table_T.size(), 2 * ss.cap);
        B_TRY(cudaMallocAsync((void **)&ss.tables, ss.cap * ptab_words() * sizeof(uint32_t), st));
    }
    for (size_t k = 0; k < ss.table_T.size(); ++k)
        B_TRY(launch_ptab(ss.table_T[k], ss.tables + k * ptab_words(), st));
    return PCAD_OK;
}

// n sweeps of every small-label slot launched one at a time.
pcad_status small_set_issue(const SmallSet &ss, const std::vector<SlotDesc> &desc, int n,
                            cudaStream_t st)
{
    for (int i : ss.big) {
        const SlotDesc &d = desc[i];
        SweepArgs a{};
        a.g = d.g;
        a.acc = d.acc;
        a.fp64_draws = d.fp64_draws;
        a.sweep_base = d.tdev;
        a.seed = d.seed;
        a.H = d.H;
        a.W = d.W;
        a.pitch = d.pitch;
        a.chain = d.chain;
        a.burn_in = d.burn_in;
        a.m = d.m;
        const size_t k = std::find(ss.table_T.begin(), ss.table_T.end(), d.m.T) - ss.table_T.begin();
        a.m.ptab = ss.tables + k * ptab_words();
        for (int s = 0; s < n; ++s) {
            a.sweep_off = (uint32_t)s;
            B_TRY(launch_pca_small(a, st, d.x[0], d.x[1], d.budget));
        }
    }
    for (size_t p = 0; p < ss.bin.size(); ++p) {
        const SlotDesc &d = desc[ss.bin[p]];
        SweepArgs a{};
        a.g = d.g;
        a.acc = d.acc;
        a.fp64_draws = d.fp64_draws;
        a.sweep_base = d.tdev;
        a.seed = d.seed;
        a.H = d.H;
        a.W = d.W;
        a.pitch = d.pitch;
        a.chain = d.chain;
        a.burn_in = d.burn_in;
        a.m = d.m;
        a.m.btab = ss.btabs + p * bin_tab_entries();
        for (int s = 0; s < n; ++s) {
            a.sweep_off = (uint32_t)s;
            B_TRY(launch_pca_binary(a, st, d.x[0], d.x[1], d.budget));
        }
    }
    return PCAD_OK;
}

// The threshold table of two-label slot i again (its coefficients changed);
// no-op for other slots.
pcad_status small_set_retable(const SmallSet &ss, const SlotDesc &d, int i, cudaStream_t st)
{
    for (size_t p = 0; p < ss.bin.size(); ++p)
        if (ss.bin[p] == i)
            B_TRY(launch_btab(d.m, ss.btabs + p * bin_tab_entries(), st));
    return PCAD_OK;
}

// Two-label chains small enough to keep their state in one CTA's shared
// memory (64 x 64 and the like) run the resident kernel: one launch per
// neighbourhood holds every such chain, one CTA each, for all the sweeps of
// a slice.  Each chain has its own threshold table (it follows the chain's
// coefficients).
struct ResSet {
    std::vector<int> slots[2];     // chains with 4 and with 8 neighbours
    int smem[2] = {0, 0};          // shared memory of each launch
    int *d_idx = nullptr;          // slot indices: slots[0], then slots[1]
    uint4 *tabs = nullptr;         // one threshold table per chain, same order
    size_t cap = 0;                // chains the buffers hold
};

size_t res_tab_entries()
{
    return (size_t)btab_bytes() / sizeof(uint4);
}

// Split `in` into the resident two-label chains and the rest; build their
// tables (kept when the set is unchanged).
pcad_status res_set_build(ResSet &rs, const std::vector<SlotDesc> &d, const std::vector<int> &in,
                          std::vector<int> &rest, cudaStream_t st)
{
    std::vector<int> sl[2];
    int smem[2] = {0, 0};
    rest.clear();
    for (int i : in) {
        if (resident_fits(d[i].m.L, d[i].nbhd, d[i].H, d[i].W)) {
            const int k = d[i].nbhd == 8 ? 1 : 0;
            sl[k].push_back(i);
            smem[k] = std::max(smem[k], resident_smem_bytes(d[i].nbhd, d[i].H, d[i].W));
        } else {
            rest.push_back(i);
        }
    }
    if (sl[0] == rs.slots[0] && sl[1] == rs.slots[1] && (rs.tabs || sl[0].size() + sl[1].size() == 0))
        return PCAD_OK;
    rs.slots[0] = sl[0];
    rs.slots[1] = sl[1];
    rs.smem[0] = smem[0];
    rs.smem[1] = smem[1];
    std::vector<int> idx(sl[0]);
    idx.insert(idx.end(), sl[1].begin(), sl[1].end());
    if (idx.size() > rs.cap) {
        if (rs.d_idx)
            B_TRY(cudaFreeAsync(rs.d_idx, st));
        if (rs.tabs)
            B_TRY(cudaFreeAsync(rs.tabs, st));
        rs.d_idx = nullptr;
        rs.tabs = nullptr;
        rs.cap = std::max(idx.size(), 2 * rs.cap);
        B_TRY(cudaMallocAsync((void **)&rs.d_idx, rs.cap * sizeof(int), st));
        B_TRY(cudaMallocAsync((void **)&rs.tabs, rs.cap * res_tab_entries() * sizeof(uint4), st));
    }
    if (idx.empty())
        return PCAD_OK;
    B_TRY(cudaMemcpyAsync(rs.d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice,
                          st));
    for (size_t p = 0; p < idx.size(); ++p)
        B_TRY(launch_btab(d[idx[p]].m, rs.tabs + p * res_tab_entries(), st));
    return PCAD_OK;
}

// The table of slot i again (its coefficients changed); no-op for other slots.
pcad_status res_set_retable(const ResSet &rs, const SlotDesc &d, int i, cudaStream_t st)
{
    size_t p = 0;
    for (int k = 0; k < 2; ++k)
        for (int j : rs.slots[k]) {
            if (j == i)
                B_TRY(launch_btab(d.m, rs.tabs + p * res_tab_entries(), st));
            ++p;
        }
    return PCAD_OK;
}

pcad_status res_set_issue(const ResSet &rs, const SlotDesc *d_slots, int n, cudaStream_t st)
{
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        const int cnt = (int)rs.slots[k].size();
        if (cnt > 0)
            B_TRY(launch_resident_batch(d_slots, rs.d_idx + off, rs.tabs + off * res_tab_entries(),
                                        cnt, k ? 8 : 4, n, rs.smem[k], st));
        off += (size_t)cnt;
    }
    return PCAD_OK;
}

void res_set_free(ResSet &rs, cudaStream_t st)
{
    if (rs.d_idx)
        cudaFreeAsync(rs.d_idx, st);
    if (rs.tabs)
        cudaFreeAsync(rs.tabs, st);
    rs = ResSet{};
}

void small_set_free(SmallSet &ss, cudaStream_t st)
{
    if (ss.tables)
        cudaFreeAsync(ss.tables, st);
    if (ss.btabs)
        cudaFreeAsync(ss.btabs, st);
    ss.tables = nullptr;
    ss.btabs = nullptr;
    ss.cap = 0;
    ss.bcap = 0;
    ss.big.clear();
    ss.bin.clear();
    ss.table_T.clear();
}

void tc_set_free(TcSet &ts, cudaStream_t st)
{
    for (TcGroup &g : ts.groups)
        if (g.wb.mem)
            cudaFreeAsync(g.wb.mem, st);
    ts.groups.clear();
    if (ts.ctr)
        cudaFreeAsync(ts.ctr, st);
    ts.ctr = nullptr;
    ts.ctr_cap = 0;
}

struct TuneKey {
    int n;
    long sites[33];
    bool operator<(const TuneKey &o) const
    {
        if (n != o.n)
            return n < o.n;
        return memcmp(sites, o.sites, sizeof(sites)) < 0;
    }
};
struct TuneVal {
    int rows;
    int lpt;
    int slice;
    float ms;     // per sweep
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

// ------------------------------------------------------------------- batch

struct pcad_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    void *block = nullptr;
    std::vector<pcad_job> jobs;      // g_host pointers are not kept valid (set to NULL)
    std::vector<SlotMem> mem;
    std::vector<SlotDesc> desc;
    SlotDesc *d_slots = nullptr;
    WorkItem *d_items = nullptr;
    int n_items = 0;
    int *d_grab = nullptr;
    uint32_t *d_t = nullptr, *d_budget = nullptr;
    unsigned long long *d_fp64 = nullptr;
    float *d_plane = nullptr;
    size_t plane_floats = 0;
    uint64_t t = 0;
    int grid = 0;
    int rows = 4;
    int lpt = 1;                     // work order: 0 image, 1 costliest first, 2 wavefront
    int slice = kSlice;              // sweeps per captured slice (per wavefront launch)
    WaveBuf wb;                      // order 2: the wavefront work list
    int wgrid = 0;
    int *d_err = nullptr;            // wavefront launches: bounded-wait flag
    TcSet tc;                        // chains on the tensor-core sweep
    SmallSet small;                  // large small-label chains, launched one at a time
    ResSet res;                      // small two-label chains, one CTA each
    float tune_ms = 0.0f;
    cudaGraphExec_t graph = nullptr;
};

namespace {

pcad_status batch_set_items(pcad_batch *b, int rows, int lpt, int slice)
{
    std::vector<int> all(b->n), not_res, others, active;
    for (int i = 0; i < b->n; ++i)
        all[i] = i;
    // small two-label chains run resident, chains with a tensor-core table
    // on the batched tensor-core sweep, large small-label chains on their
    // own launches; the tiling below applies to the others
    pcad_status st0 = res_set_build(b->res, b->desc, all, not_res, b->stream);
    if (st0 == PCAD_OK)
        st0 = tc_set_build(b->tc, b->desc, not_res, others, b->stream);
    if (st0 == PCAD_OK)
        st0 = small_set_build(b->small, b->desc, others, active, b->stream);
    if (st0 != PCAD_OK)
        return st0;
    if (lpt == kOrderWave) {
        pcad_status st = wave_upload(b->wb, b->desc, active, rows, b->stream);
        if (st != PCAD_OK)
            return st;
    } else {
        std::vector<WorkItem> items = make_items(b->desc, active, rows, lpt != 0);
        if (items.empty())
            items.push_back(WorkItem{0, 0, 0, 0});   // placeholder: never launched
        if ((int)items.size() > b->n_items && b->d_items) {
            B_TRY(cudaFreeAsync(b->d_items, b->stream));
            b->d_items = nullptr;
        }
        if (!b->d_items)
            B_TRY(cudaMallocAsync((void **)&b->d_items, items.size() * sizeof(WorkItem),
                                  b->stream));
        B_TRY(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                              cudaMemcpyHostToDevice, b->stream));
        b->n_items = active.empty() ? 0 : (int)items.size();
    }
    b->rows = rows;
    b->lpt = lpt;
    b->slice = slice;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PCAD_OK;
}

pcad_status batch_issue_slice(pcad_batch *b, cudaStream_t s)
{
    const int n = b->slice;
    pcad_status st0 = res_set_issue(b->res, b->d_slots, n, s);
    if (st0 == PCAD_OK)
        st0 = tc_set_issue(b->tc, b->desc, b->d_slots, b->d_t, b->d_budget, n, b->d_grab,
                           b->d_err, s);
    if (st0 == PCAD_OK)
        st0 = small_set_issue(b->small, b->desc, n, s);
    if (st0 != PCAD_OK)
        return st0;
    if (b->lpt == kOrderWave) {
        pcad_status st = wave_issue(b->wb, b->d_slots, n, b->d_grab, b->d_err, b->wgrid, s);
        if (st != PCAD_OK)
            return st;
    } else if (b->n_items > 0) {
        B_TRY(cudaMemsetAsync(b->d_grab, 0, n * sizeof(int), s));
        for (int k = 0; k < n; ++k)
            B_TRY(launch_batch_sweep(b->d_slots, b->d_items, b->n_items, b->d_grab + k,
                                     (uint32_t)k, b->grid, s));
    }
    B_TRY(launch_batch_advance(b->d_slots, b->n, (uint32_t)n, s));
    return PCAD_OK;
}

pcad_status batch_graph(pcad_batch *b)
{
    cudaStream_t cap;
    B_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    pcad_status st = PCAD_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = batch_issue_slice(b, cap);
        e = cudaStreamEndCapture(cap, &g);
    }
    if (st == PCAD_OK && e != cudaSuccess)
        st = set_error(PCAD_ECUDA, cudaGetErrorString(e));
    if (st == PCAD_OK) {
        e = cudaGraphInstantiate(&b->graph, g, 0);
        if (e != cudaSuccess)
            st = set_error(PCAD_ECUDA, cudaGetErrorString(e));
    }
    if (g)
        cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return st;
}

pcad_status batch_run_sweeps(pcad_batch *b, int nsweeps)
{
    std::vector<uint32_t> bud(b->n, (uint32_t)(b->t + nsweeps));
    B_TRY(cudaMemcpyAsync(b->d_budget, bud.data(), bud.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, b->stream));
    if (!b->graph) {
        pcad_status st = batch_graph(b);
        if (st != PCAD_OK)
            return st;
    }
    for (int left = nsweeps; left > 0; left -= b->slice)
        B_TRY(cudaGraphLaunch(b->graph, b->stream));
    b->t += (uint64_t)nsweeps;
    return PCAD_OK;
}

pcad_status batch_reset_state(pcad_batch *b)
{
    // x0 <- g and acc <- 0 for every slot, counters to zero
    for (int i = 0; i < b->n; ++i) {
        const SlotDesc &d = b->desc[i];
        B_TRY(cudaMemcpy2DAsync(d.x[0], d.pitch, d.g, d.pitch, d.W, d.H, cudaMemcpyDeviceToDevice,
                                b->stream));
        B_TRY(cudaMemsetAsync(d.acc, 0, (size_t)d.H * d.W * sizeof(float), b->stream));
    }
    B_TRY(cudaMemsetAsync(b->d_t, 0, b->n * sizeof(uint32_t), b->stream));
    B_TRY(cudaMemsetAsync(b->d_fp64, 0, b->n * sizeof(unsigned long long), b->stream));
    b->t = 0;
    return PCAD_OK;
}

// Synchronise the stream and report a wavefront wait that gave up.
pcad_status batch_check_err(pcad_batch *b)
{
    int err = 0;
    B_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    if (err != 0)
        return set_error(PCAD_ETIMEOUT, "wavefront wait for a neighbour tile gave up");
    return PCAD_OK;
}

pcad_status batch_autotune(pcad_batch *b)
{
    TuneKey key{};
    key.n = b->n;
    for (const SlotDesc &d : b->desc)
        key.sites[std::min(d.ncls, 32)] += (long)d.H * d.W;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->tune_ms = it->second.ms;
            return batch_set_items(b, it->second.rows, it->second.lpt, it->second.slice);
        }
    }
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    // per-sweep launches with 4/8/16-row tiles in cost or image order
    // (16-sweep graphs), and the wavefront with 4/8-row tiles and 8, 16 or 32
    // sweeps per launch; compared per sweep
    const int cands[12][3] = {{4, 1, 16},          {8, 1, 16},          {16, 1, 16},
                              {4, 0, 16},          {8, 0, 16},          {16, 0, 16},
                              {4, kOrderWave, 8},  {8, kOrderWave, 8},  {4, kOrderWave, 16},
                              {8, kOrderWave, 16}, {4, kOrderWave, 32}, {8, kOrderWave, 32}};
    TuneVal best{4, 1, kSlice, 1e30f};
    pcad_status st = PCAD_OK;
    for (const auto &c : cands) {
        const int r = c[0], lpt = c[1], sl = c[2];
        st = batch_set_items(b, r, lpt, sl);
        if (st != PCAD_OK)
            break;
        st = batch_run_sweeps(b, sl);   // warm + graph
        if (st == PCAD_OK && cudaEventRecord(e0, b->stream) != cudaSuccess)
            st = set_error(PCAD_ECUDA, "event record");
        if (st == PCAD_OK)
            st = batch_run_sweeps(b, sl);
        if (st == PCAD_OK && cudaEventRecord(e1, b->stream) != cudaSuccess)
            st = set_error(PCAD_ECUDA, "event record");
        float ms = 0.0f;
        if (st == PCAD_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = set_error(PCAD_ECUDA, "event timing");
        if (st == PCAD_OK)
            st = batch_check_err(b);
        if (st == PCAD_OK && ms / sl < best.ms)
            best = TuneVal{r, lpt, sl, ms / sl};
        if (st == PCAD_OK)
            st = batch_reset_state(b);
        if (st != PCAD_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PCAD_OK)
        return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    b->tune_ms = best.ms;
    return batch_set_items(b, best.rows, best.lpt, best.slice);
}

}  // namespace

extern "C" {

pcad_status pcad_batch_create(const pcad_job *jobs, int n, int autotune, void *cuda_stream,
                              pcad_batch **out)
{
    if (!out)
        return set_error(PCAD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!jobs || n < 1)
        return set_error(PCAD_EINVAL, "need at least one job");
    size_t total = 0;
    std::vector<SlotMem> mem(n);
    size_t max_plane = 1;
    for (int i = 0; i < n; ++i) {
        pcad_status st = check_job(jobs[i]);
        if (st != PCAD_OK)
            return st;
        const int pitch = (jobs[i].W + 15) / 16 * 16;
        mem[i] = job_layout(jobs[i], pitch, total);
        total = mem[i].end;
        max_plane = std::max(max_plane, (size_t)jobs[i].H * jobs[i].W);
    }
    const size_t off_desc = total;
    total += al(n * sizeof(SlotDesc));
    const size_t off_ctr = total;
    total += al(n * (2 * sizeof(uint32_t) + sizeof(unsigned long long)));
    const size_t off_grab = total;
    total += al((kMaxSlice + 1) * sizeof(int));   // grab counters, wavefront error flag
    const size_t off_plane = total;
    total += al(max_plane * sizeof(float));

    pcad_batch *b = new pcad_batch();
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMallocAsync(&b->block, total, b->stream);
    if (e != cudaSuccess) {
        delete b;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? PCAD_ENOMEM : PCAD_ECUDA,
                         cudaGetErrorString(e));
    }
    char *base = (char *)b->block;
    b->mem = mem;
    b->d_slots = (SlotDesc *)(base + off_desc);
    unsigned long long *fp64 = (unsigned long long *)(base + off_ctr);
    b->d_fp64 = fp64;
    b->d_t = (uint32_t *)(fp64 + n);
    b->d_budget = b->d_t + n;
    b->d_grab = (int *)(base + off_grab);
    b->d_plane = (float *)(base + off_plane);
    b->plane_floats = max_plane;
    b->d_err = b->d_grab + kMaxSlice;
    b->grid = grid_size();
    b->wgrid = wave_grid();
    b->desc.resize(n);
    auto bail = [&](pcad_status st) {
        if (b->d_items)
            cudaFreeAsync(b->d_items, b->stream);
        if (b->wb.mem)
            cudaFreeAsync(b->wb.mem, b->stream);
        tc_set_free(b->tc, b->stream);
        small_set_free(b->small, b->stream);
        res_set_free(b->res, b->stream);
        cudaFreeAsync(b->block, b->stream);
        cudaStreamSynchronize(b->stream);
        delete b;
        return st;
    };
    e = cudaMemsetAsync(base + off_ctr, 0, al(n * 16), b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    if (e != cudaSuccess)
        return bail(set_error(PCAD_ECUDA, cudaGetErrorString(e)));
    for (int i = 0; i < n; ++i) {
        const int pitch = (jobs[i].W + 15) / 16 * 16;
        pcad_status st = init_slot(jobs[i], base, mem[i], pitch, b->d_t + i, b->d_budget + i,
                                   fp64 + i, b->stream, b->desc[i]);
        if (st != PCAD_OK)
            return bail(st);
        b->jobs.push_back(jobs[i]);
        b->jobs.back().g_host = nullptr;
    }
    e = cudaMemcpyAsync(b->d_slots, b->desc.data(), n * sizeof(SlotDesc), cudaMemcpyHostToDevice,
                        b->stream);
    if (e != cudaSuccess)
        return bail(set_error(PCAD_ECUDA, cudaGetErrorString(e)));
    pcad_status st = autotune ? batch_autotune(b) : batch_set_items(b, 4, 1, kSlice);
    if (st == PCAD_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
        st = set_error(PCAD_ECUDA, "batch set-up failed");
    if (st != PCAD_OK)
        return bail(st);
    *out = b;
    return PCAD_OK;
}

pcad_status pcad_batch_run(pcad_batch *b, int nsweeps)
{
    if (!b || nsweeps < 0)
        return set_error(PCAD_EINVAL, "bad batch or sweep count");
    if (nsweeps == 0)
        return PCAD_OK;
    if (b->t + (uint64_t)nsweeps > 0xFFFFFFFFull)
        return set_error(PCAD_EINVAL, "sweep counter would exceed 2^32");
    for (const pcad_job &j : b->jobs) {
        const uint64_t t1 = b->t + nsweeps;
        const uint64_t acc = t1 > (uint64_t)j.burn_in ? t1 - j.burn_in : 0;
        if ((uint64_t)(j.model.L - 1) * acc >= (1ull << 24))
            return set_error(PCAD_EINVAL, "accumulator would leave the exact FP32 range");
    }
    return batch_run_sweeps(b, nsweeps);
}

pcad_status pcad_batch_set_model(pcad_batch *b, int i, const pcad_model *m)
{
    if (!b || i < 0 || i >= b->n)
        return set_error(PCAD_EINVAL, "bad batch or chain index");
    pcad_status st = check_model(m);
    if (st != PCAD_OK)
        return st;
    const pcad_model &o = b->jobs[i].model;
    const int To = o.pair == PCAD_PAIR_POTTS ? 1 : o.pair_T;
    const int Tn = m->pair == PCAD_PAIR_POTTS ? 1 : m->pair_T;
    if (m->L != o.L || m->nbhd != o.nbhd || m->pair != o.pair || Tn != To ||
        m->noise != o.noise || m->sampler != o.sampler || m->inertia_norm != o.inertia_norm)
        return set_error(PCAD_EINVAL, "set_model changes coefficients only (L, nbhd, pair, "
                                      "pair_T, noise and sampler stay)");
    double ta64[511];
    std::vector<double> pr64;
    DevModel dm{};
    model_tables(*m, ta64, pr64, dm);
    char *base = (char *)b->block;
    const SlotMem &sm = b->mem[i];
    // stream-ordered: sweeps queued before use the old model; the launches
    // read the descriptor from device memory, so captured graphs stay valid
    B_TRY(cudaMemcpyAsync(base + sm.ta, ta64, sizeof(ta64), cudaMemcpyHostToDevice, b->stream));
    B_TRY(cudaMemcpyAsync(base + sm.pr, pr64.data(), pr64.size() * sizeof(double),
                          cudaMemcpyHostToDevice, b->stream));
    dm.ta64 = (const double *)(base + sm.ta);
    dm.pr64 = (const double *)(base + sm.pr);
    b->desc[i].m = dm;
    if (b->desc[i].tctab)   // the tensor-core sweep's outside sums follow the model
        B_TRY(launch_tc_table(dm, const_cast<float *>(b->desc[i].tctab), b->stream));
    {
        // a slot with launches of its own carries the model in their
        // arguments: capture the slice again
        auto in = [i](const std::vector<int> &v) {
            return std::find(v.begin(), v.end(), i) != v.end();
        };
        const bool own_launch = in(b->tc.big) || in(b->tc.win) || in(b->tc.winw) ||
                                in(b->small.big) || in(b->small.bin);
        if (b->graph && own_launch) {
            B_TRY(cudaStreamSynchronize(b->stream));
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
    }
    B_TRY(cudaMemcpyAsync(&b->d_slots[i], &b->desc[i], sizeof(SlotDesc), cudaMemcpyHostToDevice,
                          b->stream));
    {
        pcad_status st2 = res_set_retable(b->res, b->desc[i], i, b->stream);
        if (st2 == PCAD_OK)
            st2 = small_set_retable(b->small, b->desc[i], i, b->stream);
        if (st2 != PCAD_OK)
            return st2;
    }
    B_TRY(cudaStreamSynchronize(b->stream));   // the host copies must outlive the transfers
    b->jobs[i].model = *m;
    return PCAD_OK;
}

pcad_status pcad_batch_reset(pcad_batch *b)
{
    if (!b)
        return set_error(PCAD_EINVAL, "batch is NULL");
    return batch_reset_state(b);
}

pcad_status pcad_batch_sync(pcad_batch *b)
{
    if (!b)
        return set_error(PCAD_EINVAL, "batch is NULL");
    return batch_check_err(b);
}

pcad_status pcad_batch_set_tiling(pcad_batch *b, int tile_rows, int order)
{
    if (!b)
        return set_error(PCAD_EINVAL, "batch is NULL");
    if (tile_rows < 4 || tile_rows > 64 || tile_rows % 4 != 0 || order < 0 || order > kOrderWave)
        return set_error(PCAD_EINVAL, "tile_rows a multiple of 4 in [4, 64], order 0..2");
    return batch_set_items(b, tile_rows, order, b->slice);
}

pcad_status pcad_batch_slice(pcad_batch *b, int sweeps, int *current)
{
    if (!b)
        return set_error(PCAD_EINVAL, "batch is NULL");
    if (sweeps != 0 && sweeps != 8 && sweeps != 16 && sweeps != 32)
        return set_error(PCAD_EINVAL, "sweeps per slice must be 8, 16 or 32 (0: keep)");
    if (sweeps != 0 && sweeps != b->slice) {
        pcad_status st = batch_set_items(b, b->rows, b->lpt, sweeps);
        if (st != PCAD_OK)
            return st;
    }
    if (current)
        *current = b->slice;
    return PCAD_OK;
}

pcad_status pcad_batch_read_sample(pcad_batch *b, int i, uint8_t *host_out, int out_pitch)
{
    if (!b || !host_out || i < 0 || i >= b->n)
        return set_error(PCAD_EINVAL, "bad batch read");
    const SlotDesc &d = b->desc[i];
    if (out_pitch < d.W)
        return set_error(PCAD_EINVAL, "out_pitch < W");
    B_TRY(cudaMemcpy2DAsync(host_out, out_pitch, d.x[b->t & 1], d.pitch, d.W, d.H,
                            cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    return PCAD_OK;
}

pcad_status pcad_batch_read_mean(pcad_batch *b, int i, float *host_out)
{
    if (!b || !host_out || i < 0 || i >= b->n)
        return set_error(PCAD_EINVAL, "bad batch read");
    const SlotDesc &d = b->desc[i];
    const uint64_t n_acc = b->t > (uint64_t)d.burn_in ? b->t - d.burn_in : 0;
    if (n_acc == 0)
        return set_error(PCAD_ESTATE, "no sweep accumulated yet");
    const long cnt = (long)d.H * d.W;
    B_TRY(launch_mean(d.acc, (float)n_acc, b->d_plane, cnt, b->stream));
    B_TRY(cudaMemcpyAsync(host_out, b->d_plane, cnt * sizeof(float), cudaMemcpyDeviceToHost,
                          b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    return PCAD_OK;
}

pcad_status pcad_batch_info(pcad_batch *b, uint64_t *t, int *tile_rows, int *lpt_order,
                            int *grid, float *tune_ms, uint64_t *fp64_draws)
{
    if (!b)
        return set_error(PCAD_EINVAL, "batch is NULL");
    if (t)
        *t = b->t;
    if (tile_rows)
        *tile_rows = b->rows;
    if (lpt_order)
        *lpt_order = b->lpt;
    if (grid)
        *grid = b->grid;
    if (tune_ms)
        *tune_ms = b->tune_ms;
    if (fp64_draws) {
        std::vector<unsigned long long> v(b->n);
        B_TRY(cudaMemcpyAsync(v.data(), b->d_fp64, b->n * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, b->stream));
        B_TRY(cudaStreamSynchronize(b->stream));
        uint64_t s = 0;
        for (auto x : v)
            s += x;
        *fp64_draws = s;
    }
    return PCAD_OK;
}

void pcad_batch_destroy(pcad_batch *b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    if (b->graph)
        cudaGraphExecDestroy(b->graph);
    if (b->d_items)
        cudaFreeAsync(b->d_items, b->stream);
    if (b->wb.mem)
        cudaFreeAsync(b->wb.mem, b->stream);
    tc_set_free(b->tc, b->stream);
    small_set_free(b->small, b->stream);
    res_set_free(b->res, b->stream);
    cudaFreeAsync(b->block, b->stream);
    cudaStreamSynchronize(b->stream);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------ server

namespace {

struct Request {
    uint64_t id = 0;
    pcad_job job{};
    std::vector<uint8_t> g;      // host copy of the observation (pitch W)
    int nsweeps = 0;
    int state = 0;               // 0 pending, 1 admitted (slot and memory held), 2 done
    bool running = false;        // admitted and in the current slice's run set
    int slot = -1;
    uint64_t t = 0;              // sweeps done (host mirror)
    size_t bytes = 0;
    void *mem = nullptr;
    double t_submit = 0.0;       // seconds (steady clock)
    double unit_cost = 0.0;      // estimated seconds per site-update
    std::vector<uint8_t> sample;
    std::vector<float> mean;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Estimated GB300 seconds per site-update of a model, for the scheduling
// order only (results never depend on it): the tensor-core sweep at
// L >= 192 (1.07e10 site-updates/s), else the CUDA-core kernels, whose time
// grows with L (measured 1.1e11 at L = 2, 4.9e10 at L = 16).
double unit_cost(const pcad_model &m)
{
    const int T = m.pair == PCAD_PAIR_POTTS ? 1 : m.pair_T;
    if (m.L >= kTcAutoLabels && T <= kTcMaxT && m.inertia_norm == 0)
        return 9.3e-11;
    return 7.4e-12 + 8.1e-13 * m.L;
}

}  // namespace

struct pcad_server {
    int max_slots = 0;
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    void *ctl = nullptr;          // descriptors, counters, grab
    SlotDesc *d_slots = nullptr;
    uint32_t *d_t = nullptr, *d_budget = nullptr;
    unsigned long long *d_fp64 = nullptr;
    int *d_grab = nullptr;
    WaveBuf wb;                   // wavefront work list of the admitted requests
    TcSet tc;                     // requests on the tensor-core sweep
    SmallSet small;               // large small-label requests, launched one at a time
    bool items_dirty = true;
    int grid = 0;
    int n_active = 0;              // admitted requests (both kinds of launch)
    int *d_err = nullptr;          // bounded-wait flag of the wavefront kernels
    int *h_err = nullptr;          // pinned: the flag after each of the last two slices
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool in_flight = false;        // the previous slice may still be running
    size_t max_active_sites = 0;   // FIFO: admission cap on the admitted requests' sites (0: none)
                                   // SRPT: run-set size in sites (0: two waves of tiles)
    size_t active_sites = 0;
    int policy = PCAD_SERVE_SRPT;
    double aging = 0.2;            // SRPT: priority seconds gained per second waited
    std::vector<SlotDesc> desc;
    std::vector<uint64_t> slot_req;   // 0 = free
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    uint64_t slices = 0;
};

namespace {

int free_slot(const pcad_server *sv)
{
    for (int i = 0; i < sv->max_slots; ++i)
        if (sv->slot_req[i] == 0)
            return i;
    return -1;
}

// Give request rq (pending, taken off the queue by the caller) slot `slot`
// and its device memory, copy its observation and initialise its state.
pcad_status admit_one(pcad_server *sv, Request &rq, int slot)
{
    cudaError_t e = cudaMallocAsync(&rq.mem, rq.bytes, sv->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PCAD_ENOMEM, cudaGetErrorString(e));
    }
    const int pitch = (rq.job.W + 15) / 16 * 16;
    SlotMem sm = job_layout(rq.job, pitch, 0);
    pcad_job j = rq.job;
    j.g_host = rq.g.data();
    j.g_pitch = rq.job.W;
    SlotDesc d{};
    pcad_status st = init_slot(j, (char *)rq.mem, sm, pitch, sv->d_t + slot,
                               sv->d_budget + slot, sv->d_fp64 + slot, sv->stream, d);
    if (st != PCAD_OK)
        return st;
    const uint32_t zero = 0, bud = (uint32_t)rq.nsweeps;
    const unsigned long long z64 = 0;
    B_TRY(cudaMemcpyAsync(sv->d_t + slot, &zero, 4, cudaMemcpyHostToDevice, sv->stream));
    B_TRY(cudaMemcpyAsync(sv->d_budget + slot, &bud, 4, cudaMemcpyHostToDevice, sv->stream));
    B_TRY(cudaMemcpyAsync(sv->d_fp64 + slot, &z64, 8, cudaMemcpyHostToDevice, sv->stream));
    B_TRY(cudaMemcpyAsync(sv->d_slots + slot, &d, sizeof(d), cudaMemcpyHostToDevice,
                          sv->stream));
    sv->desc[slot] = d;
    sv->slot_req[slot] = rq.id;
    sv->used += rq.bytes;
    sv->active_sites += (size_t)rq.job.H * rq.job.W;
    rq.slot = slot;
    rq.state = 1;
    rq.running = true;
    rq.t = 0;
    sv->items_dirty = true;
    return PCAD_OK;
}

// First come, first served: admit from the head of the queue while a slot,
// the HBM budget and the admission cap allow; every admitted request runs.
pcad_status server_admit_fifo(pcad_server *sv)
{
    while (!sv->pending.empty()) {
        Request &rq = sv->reqs[sv->pending.front()];
        const int slot = free_slot(sv);
        const size_t sites = (size_t)rq.job.H * rq.job.W;
        if (slot < 0 || sv->used + rq.bytes > sv->budget)
            break;   // wait for slots or memory
        if (sv->max_active_sites && sv->active_sites > 0 &&
            sv->active_sites + sites > sv->max_active_sites)
            break;   // enough work admitted: the GPU is full, the next one waits
        sv->pending.pop_front();
        pcad_status st = admit_one(sv, rq, slot);
        if (st != PCAD_OK) {
            sv->pending.push_front(rq.id);
            return st;
        }
    }
    return PCAD_OK;
}

// Shortest remaining work first, with aging: every step orders the queued
// and admitted requests by estimated remaining GPU time (sites x sweeps
// left x unit cost) minus `aging` x time waited since submission, and runs
// the shortest ones until the run set holds the fill target of sites (at
// least one request), admitting queued ones as slots and the HBM budget
// allow.  Admitted requests outside the run set keep their state on the
// device and pause (their descriptor is marked inactive, so the slice's
// launches and the counter advance skip them).  Under overload this
// finishes short requests first instead of sharing the GPU among all of
// them; aging bounds how long a long request can be passed over.
pcad_status server_schedule_srpt(pcad_server *sv)
{
    const double now = now_s();
    std::vector<std::pair<double, uint64_t>> order;
    order.reserve(sv->reqs.size());
    for (auto &kv : sv->reqs) {
        const Request &rq = kv.second;
        if (rq.state == 2)
            continue;
        const double left = (double)rq.job.H * rq.job.W * (double)(rq.nsweeps - rq.t);
        order.emplace_back(left * rq.unit_cost - sv->aging * (now - rq.t_submit), rq.id);
    }
    std::sort(order.begin(), order.end());
    const size_t fill = sv->max_active_sites
                            ? sv->max_active_sites
                            : (size_t)2 * (size_t)std::max(sv->grid, 1) * 128;
    // without an explicit target, also at least kMinSliceSeconds of estimated
    // work per slice, so the host's per-slice cost stays small against it
    const double min_time = sv->max_active_sites ? 0.0 : kMinSliceSeconds;
    size_t run_sites = 0;
    double run_time = 0.0;    // estimated seconds per sweep of the run set
    std::vector<uint64_t> run;
    for (const auto &pr : order) {
        if (!run.empty() && run_sites >= fill && run_time * kSlice >= min_time)
            break;
        Request &rq = sv->reqs[pr.second];
        if (rq.state == 0) {
            const int slot = free_slot(sv);
            if (slot < 0 || sv->used + rq.bytes > sv->budget)
                continue;   // no room now: a shorter one may still fit
            auto it = std::find(sv->pending.begin(), sv->pending.end(), rq.id);
            if (it != sv->pending.end())
                sv->pending.erase(it);
            pcad_status st = admit_one(sv, rq, slot);
            if (st != PCAD_OK) {
                sv->pending.push_front(rq.id);
                return st;
            }
        }
        run.push_back(rq.id);
        run_sites += (size_t)rq.job.H * rq.job.W;
        run_time += (double)rq.job.H * rq.job.W * rq.unit_cost;
    }
    // pause or resume the admitted requests
    std::vector<char> in_run(sv->max_slots, 0);
    for (uint64_t id : run)
        in_run[sv->reqs[id].slot] = 1;
    for (int i = 0; i < sv->max_slots; ++i) {
        if (sv->slot_req[i] == 0)
            continue;
        Request &rq = sv->reqs[sv->slot_req[i]];
        const bool want = in_run[i] != 0;
        if (want == rq.running && sv->desc[i].active == (want ? 1 : 0))
            continue;
        rq.running = want;
        sv->desc[i].active = want ? 1 : 0;
        B_TRY(cudaMemcpyAsync(sv->d_slots + i, &sv->desc[i], sizeof(SlotDesc),
                              cudaMemcpyHostToDevice, sv->stream));
        sv->items_dirty = true;
    }
    return PCAD_OK;
}

pcad_status server_items(pcad_server *sv)
{
    std::vector<int> all, active;   // the run set, then those not on the tensor-core sweep
    for (int i = 0; i < sv->max_slots; ++i)
        if (sv->slot_req[i] != 0 && sv->reqs[sv->slot_req[i]].running)
            all.push_back(i);
    // requests with a tensor-core table run on the batched tensor-core sweep
    std::vector<int> others;
    pcad_status st = tc_set_build(sv->tc, sv->desc, all, others, sv->stream);
    if (st == PCAD_OK)
        st = small_set_build(sv->small, sv->desc, others, active, sv->stream);
    if (st != PCAD_OK)
        return st;
    long tiles4 = 0;
    for (int i : active)
        tiles4 += (long)((sv->desc[i].W + 31) / 32) * ((sv->desc[i].H + 3) / 4);
    const int rows = tiles4 >= (long)kServeTallTiles * sv->grid ? 8 : 4;
    st = wave_upload(sv->wb, sv->desc, active, rows, sv->stream);
    if (st != PCAD_OK)
        return st;
    sv->n_active = (int)all.size();
    sv->items_dirty = false;
    return PCAD_OK;
}

// Wait for slice `s` (its event) and report a bounded-wait timeout of it.
pcad_status server_wait_slice(pcad_server *sv, uint64_t s)
{
    B_TRY(cudaEventSynchronize(sv->ev[s & 1]));
    if (sv->h_err[s & 1] != 0)
        return set_error(PCAD_ETIMEOUT, "wavefront wait for a neighbour tile gave up");
    return PCAD_OK;
}

}  // namespace

extern "C" {

pcad_status pcad_server_create(int max_slots, size_t hbm_budget_bytes, void *cuda_stream,
                               pcad_server **out)
{
    if (!out)
        return set_error(PCAD_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 65536 || hbm_budget_bytes == 0)
        return set_error(PCAD_EINVAL, "max_slots in [1, 65536] and a non-zero budget");
    pcad_server *sv = new pcad_server();
    sv->max_slots = max_slots;
    sv->budget = hbm_budget_bytes;
    sv->stream = (cudaStream_t)cuda_stream;
    const size_t bytes = al(max_slots * sizeof(SlotDesc)) +
                         al(max_slots * (2 * sizeof(uint32_t) + sizeof(unsigned long long))) +
                         al(kSlice * sizeof(int)) + al(sizeof(int));
    cudaError_t e = cudaMallocAsync(&sv->ctl, bytes, sv->stream);
    if (e != cudaSuccess) {
        delete sv;
        cudaGetLastError();
        return set_error(PCAD_ENOMEM, cudaGetErrorString(e));
    }
    char *p = (char *)sv->ctl;
    sv->d_slots = (SlotDesc *)p;
    p += al(max_slots * sizeof(SlotDesc));
    sv->d_fp64 = (unsigned long long *)p;
    sv->d_t = (uint32_t *)(sv->d_fp64 + max_slots);
    sv->d_budget = sv->d_t + max_slots;
    p += al(max_slots * (2 * sizeof(uint32_t) + sizeof(unsigned long long)));
    sv->d_grab = (int *)p;
    p += al(kSlice * sizeof(int));
    sv->d_err = (int *)p;
    e = cudaMemsetAsync(sv->ctl, 0, bytes, sv->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(sv->stream);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&sv->h_err, 2 * sizeof(int));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&sv->ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (int k = 0; k < 2; ++k)
            if (sv->ev[k])
                cudaEventDestroy(sv->ev[k]);
        if (sv->h_err)
            cudaFreeHost(sv->h_err);
        cudaFreeAsync(sv->ctl, sv->stream);
        cudaStreamSynchronize(sv->stream);
        delete sv;
        return set_error(PCAD_ECUDA, cudaGetErrorString(e));
    }
    sv->h_err[0] = sv->h_err[1] = 0;
    sv->desc.assign(max_slots, SlotDesc{});
    sv->slot_req.assign(max_slots, 0);
    sv->grid = wave_grid();
    *out = sv;
    return PCAD_OK;
}

pcad_status pcad_server_set_limits(pcad_server *sv, size_t max_active_sites)
{
    if (!sv)
        return set_error(PCAD_EINVAL, "server is NULL");
    sv->max_active_sites = max_active_sites;
    return PCAD_OK;
}

pcad_status pcad_server_set_policy(pcad_server *sv, int policy, double aging)
{
    if (!sv)
        return set_error(PCAD_EINVAL, "server is NULL");
    if (policy != PCAD_SERVE_FIFO && policy != PCAD_SERVE_SRPT)
        return set_error(PCAD_EINVAL, "policy must be PCAD_SERVE_FIFO or PCAD_SERVE_SRPT");
    if (!(aging >= 0.0 && aging <= 1e6))
        return set_error(PCAD_EINVAL, "aging must lie in [0, 1e6]");
    if (policy == PCAD_SERVE_FIFO && sv->policy != PCAD_SERVE_FIFO) {
        // every admitted request runs again under FIFO
        for (int i = 0; i < sv->max_slots; ++i) {
            if (sv->slot_req[i] == 0 || sv->desc[i].active)
                continue;
            sv->reqs[sv->slot_req[i]].running = true;
            sv->desc[i].active = 1;
            B_TRY(cudaMemcpyAsync(sv->d_slots + i, &sv->desc[i], sizeof(SlotDesc),
                                  cudaMemcpyHostToDevice, sv->stream));
            sv->items_dirty = true;
        }
    }
    sv->policy = policy;
    sv->aging = aging;
    return PCAD_OK;
}

pcad_status pcad_server_submit(pcad_server *sv, const pcad_job *job, int nsweeps, uint64_t *id)
{
    if (!sv || !job || !id)
        return set_error(PCAD_EINVAL, "NULL argument");
    if (nsweeps < 1)
        return set_error(PCAD_EINVAL, "nsweeps must be >= 1");
    pcad_status st = check_job(*job);
    if (st != PCAD_OK)
        return st;
    const uint64_t acc = nsweeps > job->burn_in ? (uint64_t)(nsweeps - job->burn_in) : 0;
    if ((uint64_t)(job->model.L - 1) * acc >= (1ull << 24))
        return set_error(PCAD_EINVAL, "accumulator would leave the exact FP32 range");
    Request rq;
    rq.id = sv->next_id++;
    rq.job = *job;
    rq.job.g_host = nullptr;
    rq.nsweeps = nsweeps;
    rq.bytes = slot_bytes(*job);
    rq.t_submit = now_s();
    rq.unit_cost = unit_cost(job->model);
    if (rq.bytes > sv->budget)
        return set_error(PCAD_ENOMEM, "request larger than the whole HBM budget");
    rq.g.resize((size_t)job->H * job->W);
    for (int r = 0; r < job->H; ++r)
        memcpy(rq.g.data() + (size_t)r * job->W, job->g_host + (size_t)r * job->g_pitch, job->W);
    *id = rq.id;
    sv->pending.push_back(rq.id);
    sv->reqs.emplace(rq.id, std::move(rq));
    return PCAD_OK;
}

pcad_status pcad_server_step(pcad_server *sv, int slice_sweeps, int *n_active, int *n_pending,
                             int *n_finished)
{
    if (!sv || slice_sweeps < 1 || slice_sweeps > kSlice)
        return set_error(PCAD_EINVAL, "slice_sweeps must be in [1, 16]");
    pcad_status st =
        sv->policy == PCAD_SERVE_FIFO ? server_admit_fifo(sv) : server_schedule_srpt(sv);
    if (st != PCAD_OK)
        return st;
    if (sv->items_dirty) {
        st = server_items(sv);
        if (st != PCAD_OK)
            return st;
    }
    int finished = 0, active = 0;
    if (sv->n_active > 0) {
        // one wavefront launch per kind runs the slice for every admitted request
        st = tc_set_issue(sv->tc, sv->desc, sv->d_slots, sv->d_t, sv->d_budget, slice_sweeps,
                          sv->d_grab, sv->d_err, sv->stream);
        if (st == PCAD_OK)
            st = small_set_issue(sv->small, sv->desc, slice_sweeps, sv->stream);
        if (st == PCAD_OK && sv->wb.n_items > 0)
            st = wave_issue(sv->wb, sv->d_slots, slice_sweeps, sv->d_grab, sv->d_err, sv->grid,
                            sv->stream);
        if (st != PCAD_OK)
            return st;
        B_TRY(launch_batch_advance(sv->d_slots, sv->max_slots, (uint32_t)slice_sweeps,
                                   sv->stream));
        const uint64_t s = sv->slices++;
        B_TRY(cudaMemcpyAsync(sv->h_err + (s & 1), sv->d_err, sizeof(int),
                              cudaMemcpyDeviceToHost, sv->stream));
        // harvest: requests whose budget this slice spends
        for (int i = 0; i < sv->max_slots; ++i) {
            if (sv->slot_req[i] == 0)
                continue;
            Request &rq = sv->reqs[sv->slot_req[i]];
            if (!rq.running) {   // paused this slice
                ++active;
                continue;
            }
            rq.t = std::min<uint64_t>(rq.t + slice_sweeps, (uint64_t)rq.nsweeps);
            if (rq.t < (uint64_t)rq.nsweeps) {
                ++active;
                continue;
            }
            const SlotDesc &d = sv->desc[i];
            rq.sample.resize((size_t)d.H * d.W);
            rq.mean.assign((size_t)d.H * d.W, 0.0f);
            B_TRY(cudaMemcpy2DAsync(rq.sample.data(), d.W, d.x[rq.t & 1], d.pitch, d.W, d.H,
                                    cudaMemcpyDeviceToHost, sv->stream));
            const uint64_t n_acc = rq.t > (uint64_t)d.burn_in ? rq.t - d.burn_in : 0;
            if (n_acc > 0) {
                B_TRY(launch_mean(d.acc, (float)n_acc, d.acc, (long)d.H * d.W, sv->stream));
                B_TRY(cudaMemcpyAsync(rq.mean.data(), d.acc, (size_t)d.H * d.W * sizeof(float),
                                      cudaMemcpyDeviceToHost, sv->stream));
            }
            SlotDesc off = d;
            off.active = 0;
            sv->desc[i] = off;
            B_TRY(cudaMemcpyAsync(sv->d_slots + i, &sv->desc[i], sizeof(SlotDesc),
                                  cudaMemcpyHostToDevice, sv->stream));
            B_TRY(cudaFreeAsync(rq.mem, sv->stream));
            rq.mem = nullptr;
            sv->used -= rq.bytes;
            sv->active_sites -= (size_t)d.H * d.W;
            sv->slot_req[i] = 0;
            rq.state = 2;
            rq.running = false;
            rq.slot = -1;
            sv->items_dirty = true;
            ++finished;
        }
        B_TRY(cudaEventRecord(sv->ev[s & 1], sv->stream));
        // a finished request's outputs must be in host memory on return;
        // otherwise only the previous slice is waited for, so the host
        // prepares the next slice while this one runs
        pcad_status ws = PCAD_OK;
        if (sv->in_flight)
            ws = server_wait_slice(sv, s - 1);
        if (ws == PCAD_OK && finished > 0)
            ws = server_wait_slice(sv, s);
        sv->in_flight = finished == 0;
        if (ws != PCAD_OK)
            return ws;
    } else if (sv->in_flight) {
        sv->in_flight = false;
        pcad_status ws = server_wait_slice(sv, sv->slices - 1);
        if (ws != PCAD_OK)
            return ws;
    }
    if (n_active)
        *n_active = active;
    if (n_pending)
        *n_pending = (int)sv->pending.size();
    if (n_finished)
        *n_finished = finished;
    return PCAD_OK;
}

pcad_status pcad_server_poll(pcad_server *sv, uint64_t id, int *state, uint8_t *sample_out,
                             float *mean_out)
{
    if (!sv || !state)
        return set_error(PCAD_EINVAL, "NULL argument");
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end())
        return set_error(PCAD_EINVAL, "unknown or already collected request");
    *state = it->second.state;
    if (it->second.state == 2) {
        if (sample_out)
            memcpy(sample_out, it->second.sample.data(), it->second.sample.size());
        if (mean_out)
            memcpy(mean_out, it->second.mean.data(), it->second.mean.size() * sizeof(float));
        if (sample_out || mean_out)
            sv->reqs.erase(it);
    }
    return PCAD_OK;
}

pcad_status pcad_server_info(pcad_server *sv, size_t *hbm_used, uint64_t *slices,
                             uint64_t *fp64_draws)
{
    if (!sv)
        return set_error(PCAD_EINVAL, "server is NULL");
    if (hbm_used)
        *hbm_used = sv->used;
    if (slices)
        *slices = sv->slices;
    if (fp64_draws) {
        std::vector<unsigned long long> v(sv->max_slots);
        B_TRY(cudaMemcpyAsync(v.data(), sv->d_fp64, v.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, sv->stream));
        B_TRY(cudaStreamSynchronize(sv->stream));
        uint64_t s = 0;
        for (auto x : v)
            s += x;
        *fp64_draws = s;
    }
    return PCAD_OK;
}

void pcad_server_destroy(pcad_server *sv)
{
    if (!sv)
        return;
    cudaStreamSynchronize(sv->stream);
    for (auto &kv : sv->reqs)
        if (kv.second.mem)
            cudaFreeAsync(kv.second.mem, sv->stream);
    if (sv->wb.mem)
        cudaFreeAsync(sv->wb.mem, sv->stream);
    tc_set_free(sv->tc, sv->stream);
    small_set_free(sv->small, sv->stream);
    cudaFreeAsync(sv->ctl, sv->stream);
    cudaStreamSynchronize(sv->stream);
    for (int k = 0; k < 2; ++k)
        cudaEventDestroy(sv->ev[k]);
    cudaFreeHost(sv->h_err);
    delete sv;
}

}  // extern "C"
