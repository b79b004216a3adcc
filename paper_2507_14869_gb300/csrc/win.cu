// Lazy-PCA sweep (Section 5.2, Eq. posterior_pca_transition_matrix) and
// checkerboard Gibbs colour phases (Section 5.1) on the CUDA cores with a
// per-site label window, truncated-linear or Potts priors with
// 9 <= L <= 256.
//
// The weights are those of the tensor-core sweep, w(s) = 2^fl(alpha (g-s)^2 +
// fl(mu Pb(s) + cb)) with the tent sum Pb(s) = sum_j max(T - |x_j - s|, 0)
// (see tc_math.cuh), so the same per-site certified margin holds.  Pb is zero
// outside the hull [x_min - T + 1, x_max + T - 1] of the present neighbours:
// there the chunk sums depend on g only and come from the model's outside
// table.  Only the hull's chunks (about 11 of 32 at L = 256, T = 30) are
// evaluated, and without tensor cores:
//
//   * Tent bytes.  For a neighbour x_j and a chunk of labels 8c .. 8c + 7,
//     the 8 tents max(T - |x_j - 8c - k|, 0) are a function of d = x_j - 8c
//     alone, zero unless -T < d < T + 7.  A 2T + 8 entry table holds them as
//     8 bytes; one 8-byte shared-memory read per neighbour and two integer
//     adds give Pb of the chunk's 8 labels, a byte each (at most
//     nbhd T <= 255, no carries).
//   * Balanced warps.  The hull size varies from site to site (one far-off
//     neighbour widens it) and a warp runs as long as its widest hull, so
//     the block sorts its 128 sites by hull size and warp w evaluates the
//     chunks of the w-th quarter.
//   * The rest is the CUDA-core draw: chunk sums in label order with Kahan
//     compensation (outside chunks from the table), the inertia correction,
//     the certified inverse-CDF selection with the chosen chunk's weights
//     recomputed exactly, FP64 re-draws of uncertain draws by the warp.
//
// One thread per site in blocks of 128 threads: 4 x 32 sites for lazy PCA
// (one Philox call per 4 sites, computed by one warp), the phase sites of
// 64 x 4 (8) cells for Gibbs.  Each form runs as one launch per sweep (per
// colour phase) or as a persistent wavefront of (sweep, tile) items with
// bounded dependency waits.
#include "tc_math.cuh"

namespace pcad {

namespace {

using namespace tcm;

constexpr int kWX = 32;
constexpr int kWY = 4;
constexpr int kWThreads = kWX * kWY;
constexpr int kWMaxChunks = 32;
constexpr int kTentMax = 2 * 33 + 8;   // entries of the tent-byte table (T <= 33)

// Entry i (d = i - T) of the tent-byte table: byte k = max(T - |d - k|, 0).
// d = x_j - 8c outside (-T, T + 7) gives all zeros: such an index is
// clamped to the last entry (2T + 7, itself zero).  Most lanes of a warp
// then read the same zero entry, which shared memory broadcasts (a table
// over every d without the clamp measured 5 % slower: more distinct
// addresses per read, more bank conflicts).
__device__ __forceinline__ uint2 tent_entry(int T, int i)
{
    const int d = i - T;
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lo |= (uint32_t)max(T - abs(d - k), 0) << (8 * k);
        hi |= (uint32_t)max(T - abs(d - 4 - k), 0) << (8 * k);
    }
    return make_uint2(lo, hi);
}

// Exact float of byte k of p (the byte placed in the mantissa of 2^23).
__device__ __forceinline__ float pb_byte(uint32_t p, int k)
{
    return __uint_as_float(__byte_perm(p, 0x4B000000u, 0x7440u | (uint32_t)k));
}

// Sum of the weights of chunk c (labels 8c .. 8c + 7) of a site with
// observation gf from its 8 tent sums (bytes of lo, hi: exact integers).
// The weights and their pairwise tree sum are window_chunk's, so the value
// equals the tensor-core sweep's for the same chunk.
template <bool LMASK>
__device__ __forceinline__ float win_chunk_sum(const DevModel &m, float mu, float gf, int c,
                                               uint32_t lo, uint32_t hi)
{
    const float dgb = __fsub_rn(gf, (float)(c * kChunk));
    const float2 a2 = make_float2(m.alpha, m.alpha), mu2 = make_float2(mu, mu),
                 cb2 = make_float2(m.cb, m.cb), mag2 = make_float2(-8388608.0f, -8388608.0f);
    const float2 dgb2 = make_float2(dgb, __fsub_rn(dgb, 1.0f));
    float2 wv[4];
#pragma unroll
    for (int k = 0; k < kChunk; k += 2) {
        const uint32_t p = k < 4 ? lo : hi;
        const float2 pb2 =
            __fadd2_rn(make_float2(pb_byte(p, k & 3), pb_byte(p, (k + 1) & 3)), mag2);
        const float2 dg = __fadd2_rn(dgb2, make_float2(-(float)k, -(float)k));
        const float2 qq = __fmul2_rn(dg, dg);
        const float2 in2 = __ffma2_rn(mu2, pb2, cb2);
        const float2 v = __ffma2_rn(a2, qq, in2);
        float w0 = ex2_ftz(v.x), w1 = ex2_ftz(v.y);
        if (LMASK && c * kChunk + k >= m.L)
            w0 = 0.0f;
        if (LMASK && c * kChunk + k + 1 >= m.L)
            w1 = 0.0f;
        wv[k >> 1] = make_float2(w0, w1);
    }
    const float2 a = __fadd2_rn(make_float2(wv[0].x, wv[2].x), make_float2(wv[0].y, wv[2].y));
    const float2 b = __fadd2_rn(make_float2(wv[1].x, wv[3].x), make_float2(wv[1].y, wv[3].y));
    const float2 t2 = __fadd2_rn(a, b);
    return __fadd_rn(t2.x, t2.y);
}

// The 8 tent sums of chunk c from neighbour labels x (bytes of lo, hi).
template <int NB>
__device__ __forceinline__ void chunk_tents(const int (&x)[NB], int c, int T, const uint2 *tent,
                                            uint32_t &lo, uint32_t &hi)
{
    const uint32_t zero_i = (uint32_t)(2 * T + 7);   // an all-zero entry
    const int off = T - kChunk * c;
    lo = hi = 0u;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const uint2 e = tent[min((uint32_t)(x[j] + off), zero_i)];
        lo += e.x;
        hi += e.y;
    }
}

// Inclusive prefix sums p[0..7] of chunk c's weights (from its tent sums lo,
// hi): the operations of chunk_prefix_exact on the same exact tent sums,
// hence the same values.
__device__ __forceinline__ void win_chunk_prefix(const DevModel &m, float mu, float gf, int c,
                                                 uint32_t lo, uint32_t hi, float (&p)[kChunk])
{
    const float dgb = __fsub_rn(gf, (float)(c * kChunk));
    const float2 a2 = make_float2(m.alpha, m.alpha), mu2 = make_float2(mu, mu),
                 cb2 = make_float2(m.cb, m.cb), mag2 = make_float2(-8388608.0f, -8388608.0f);
    const float2 dgb2 = make_float2(dgb, __fsub_rn(dgb, 1.0f));
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < kChunk; k += 2) {
        const uint32_t pw = k < 4 ? lo : hi;
        const float2 pb2 =
            __fadd2_rn(make_float2(pb_byte(pw, k & 3), pb_byte(pw, (k + 1) & 3)), mag2);
        const float2 dg = __fadd2_rn(dgb2, make_float2(-(float)k, -(float)k));
        const float2 qq = __fmul2_rn(dg, dg);
        const float2 in2 = __ffma2_rn(mu2, pb2, cb2);
        const float2 v = __ffma2_rn(a2, qq, in2);
        float w0 = ex2_ftz(v.x), w1 = ex2_ftz(v.y);
        if (c * kChunk + k >= m.L)
            w0 = 0.0f;
        if (c * kChunk + k + 1 >= m.L)
            w1 = 0.0f;
        S = __fadd_rn(S, w0);
        p[k] = S;
        S = __fadd_rn(S, w1);
        p[k + 1] = S;
    }
}

// Shared memory of a windowed draw block (128 threads).
template <int NB>
struct __align__(16) WinShared {
    float G[kWMaxChunks * kWThreads];   // [chunk][thread]: chunk sums, then prefix sums
    float F[kTabF];                     // outside-chunk sums
    uint2 tent[kTentMax];               // tent bytes
    int rec[NB + 1][kWThreads];         // per site: neighbour labels; g | clo << 9 | cnt << 16
    int bins[kWMaxChunks + 1];          // hull sizes 0..32: counts, then offsets
    uint8_t perm[kWThreads];            // sites in increasing hull size
};

// Tables into shared memory (the caller's barrier follows).
template <int NB>
__device__ __forceinline__ void win_setup(WinShared<NB> &sh, int T, const float *ftab, int tid)
{
    for (int i = tid; i < kTabF / 4; i += kWThreads)
        reinterpret_cast<float4 *>(sh.F)[i] = __ldg(reinterpret_cast<const float4 *>(ftab) + i);
    for (int i = tid; i < 2 * T + 8; i += kWThreads)
        sh.tent[i] = tent_entry(T, i);
    if (tid <= kWMaxChunks)
        sh.bins[tid] = 0;
}

// The draw of every site of the block (thread tid: site inputs `in`, valid
// or not).  Every thread of the block calls it (block barriers inside).
// Returns the label (0 for an invalid site); uncertain FP32 draws are
// re-drawn in FP64 by the warp, counted in *fp64.
template <int NB, bool LMASK>
__device__ __forceinline__ int win_draw(WinShared<NB> &sh, const DevModel &m, const SiteIn<NB> &in,
                                        bool valid, int tid, unsigned long long *fp64)
{
    const int lane = tid & 31, wp = tid >> 5;
    const int T = m.T;
    const float mu = -m.gam;
    const int nc = (m.L + kChunk - 1) / kChunk;
    const float gf = (float)in.g;
    // the hull's chunks: where some present neighbour's tent is nonzero
    int xmin = kMissingLabelI, xmax = -1;
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (in.xni[j] < kMissingLabelI) {
            xmin = min(xmin, in.xni[j]);
            xmax = max(xmax, in.xni[j]);
        }
    int clo = 0, cnt = 0;
    if (valid && xmax >= 0) {
        clo = max(xmin - T + 1, 0) >> 3;
        cnt = min((xmax + T - 1) >> 3, nc - 1) - clo + 1;
    }
    // The block's sites sorted by hull size (a counting sort): thread i
    // evaluates the chunks of the i-th smallest hull and writes them into that
    // site's column, so a warp's longest hull is close to its other lanes'.
    // (Dealing (site, chunk) tasks out over a warp with shuffles measured
    // slower: they cost more than the imbalance they remove.)
    for (int j = 0; j < NB; ++j)
        sh.rec[j][tid] = in.xni[j];
    sh.rec[NB][tid] = in.g | (clo << 9) | (cnt << 16);
    const int rank = atomicAdd(&sh.bins[cnt], 1);
    __syncthreads();
    if (wp == 0) {   // exclusive offsets of the bins 0..32
        const int b = sh.bins[lane];
        int inc = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o)
                inc += v;
        }
        __syncwarp();
        sh.bins[lane] = inc - b;
        if (lane == 31)
            sh.bins[32] = inc;
    }
    __syncthreads();
    sh.perm[sh.bins[cnt] + rank] = (uint8_t)tid;
    __syncthreads();
    {
        const int sid = sh.perm[tid];
        int sx[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j)
            sx[j] = sh.rec[j][sid];
        const int pk = sh.rec[NB][sid];
        const int sclo = (pk >> 9) & 127, scnt = pk >> 16;
        const float sgf = (float)(pk & 511);
        const int maxcnt = __reduce_max_sync(0xFFFFFFFFu, scnt);
#pragma unroll 1
        for (int k = 0; k < maxcnt; ++k) {
            if (k < scnt) {
                const int cc = sclo + k;
                uint32_t lo, hi;
                chunk_tents<NB>(sx, cc, T, sh.tent, lo, hi);
                sh.G[cc * kWThreads + sid] = win_chunk_sum<LMASK>(m, mu, sgf, cc, lo, hi);
            }
        }
    }
    __syncthreads();
    float *Gcol = sh.G + tid;

    // chunk prefix sums in label order (Kahan), outside chunks from the table
    float G = 0.0f, comp = 0.0f;
    const int chi = clo + cnt - 1;
#pragma unroll 4
    for (int cc = 0; cc < nc; ++cc) {
        const float S = (cc >= clo && cc <= chi) ? Gcol[cc * kWThreads]
                                                 : tab_sum<LMASK>(sh.F, in.g, cc, nc);
        const float y = __fsub_rn(S, comp);
        const float tt = __fadd_rn(G, y);
        comp = __fsub_rn(__fsub_rn(tt, G), y);
        G = tt;
        Gcol[cc * kWThreads] = G;
    }
    int s = 0;
    bool certain = true;
    if (valid) {
        float xn[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j)
            xn[j] = (float)in.xni[j];
        float delta = 0.0f;
        if (m.em1 != 0.0f) {
            const float xif = (float)in.xi;
            delta = __fmul_rn(label_wb(m, mu, tent_sum<NB>(xn, m.Tf, xif), __fsub_rn(gf, xif)),
                              m.em1);
        }
        s = cdf_select(m, site_margin(m, G, delta), [&](int cc) { return Gcol[cc * kWThreads]; },
                       nc, G, delta, in.xi, in.ub, certain, [&](int cs, float (&pp)[kChunk]) {
                           uint32_t lo, hi;
                           chunk_tents<NB>(in.xni, cs, T, sh.tent, lo, hi);
                           win_chunk_prefix(m, mu, gf, cs, lo, hi, pp);
                       });
    }
    return warp_redraw_fp64<NB>(m, valid && !certain, in, s, fp64);
}

// One lazy-PCA sweep: a.xin -> a.xout, accumulate after burn-in.  ftab: the
// model's outside-chunk table (tc_table_floats floats, launch_tc_table).
// Warp wp takes the block's columns 8 wp .. 8 wp + 7 over its 4 rows.
// Planes: a.xin -> a.xout, or (x0 != nullptr) x0 / x1 holding the states of
// even / odd sweep indices; budget (optional): a sweep with index >= *budget
// is skipped (a chain of a batch or of the server).
template <int NB, bool LMASK>
__global__ void __launch_bounds__(kWThreads, 8) pca_win_kernel(const SweepArgs a,
                                                               const float *ftab, uint8_t *x0,
                                                               uint8_t *x1, const uint32_t *budget)
{
    const uint32_t t = sweep_index(a);
    if (budget && t >= *budget)
        return;   // the whole launch, before any barrier
    const uint8_t *xin = x0 ? ((t & 1u) ? x1 : x0) : a.xin;
    uint8_t *xout = x0 ? ((t & 1u) ? x0 : x1) : a.xout;
    __shared__ WinShared<NB> sh;
    __shared__ __align__(16) uint32_t U_s[kWY * kWX];
    const int lane = (int)threadIdx.x, wp = (int)threadIdx.y;
    const int tid = wp * kWX + lane;
    const int lr = lane >> 3, lc = 8 * wp + (lane & 7);
    const int c = (int)blockIdx.x * kWX + lc;
    const int r = (int)blockIdx.y * kWY + lr;
    win_setup(sh, a.m.T, ftab, tid);
    if (wp == 0)
        block_uniforms(a, (int)blockIdx.y * kWY, (int)blockIdx.x * kWX, t, U_s);
    __syncthreads();
    const bool valid = r < a.H && c < a.W;
    SiteIn<NB> in{};
    if (valid) {
        load_site<NB, false, false>(a, xin, r, c, kTagPCA, t, in);
        in.ub = U_s[lr * kWX + lc];
    }
    const int s = win_draw<NB, LMASK>(sh, a.m, in, valid, tid, a.fp64_draws);
    if (valid) {
        xout[(size_t)r * a.pitch + c] = (uint8_t)s;
        if (accumulate_after(a, t)) {
            float *p = a.acc + (size_t)r * a.W + c;
            *p = *p + (float)s;
        }
    }
}

// Wavefront form for images of few tiles: the nsweeps sweeps of a block in
// one persistent launch.  Items (sweep k, tile j) of 4 x 32 sites are taken
// in increasing order from an atomic counter; item (k, j) waits until the
// 3 x 3 tiles around j have finished sweep k - 1 (done[] counts finished
// sweeps per tile, observed with acquire loads, each wait bounded; a wait
// that runs out sets *err and no block takes a further item).  Every item an
// item depends on has a smaller index and was taken by a resident block (the
// grid is the resident capacity), so the waits end.  Labels and sums written
// by other blocks in the launch are read through L2.  Plane of sweep k of
// the launch: x0 for even k, x1 for odd, or (par_from_t) by the parity of
// the sweep index t; budget (optional): items of sweeps t >= *budget are
// skipped (nothing waited for, read, written or published).
template <int NB, bool LMASK>
__global__ void __launch_bounds__(kWThreads, 8)
    pca_winw_kernel(const SweepArgs a, const float *ftab, uint8_t *x0, uint8_t *x1, int nsweeps,
                    int tiles_x, int tiles_y, unsigned int *done, unsigned int *grab, int *err,
                    int par_from_t, const uint32_t *budget)
{
    __shared__ WinShared<NB> sh;
    __shared__ __align__(16) uint32_t U_s[kWY * kWX];
    __shared__ unsigned int s_next;
    const int lane = (int)threadIdx.x, wp = (int)threadIdx.y;
    const int tid = wp * kWX + lane;
    const int lr = lane >> 3, lc = 8 * wp + (lane & 7);
    const unsigned int ntiles = (unsigned int)(tiles_x * tiles_y);
    const unsigned int total = ntiles * (unsigned int)nsweeps;
    const uint32_t t0 = sweep_index(a);
    const long long limit = wait_limit(a.wait_ns);
    win_setup(sh, a.m.T, ftab, tid);
    if (tid == 0)
        s_next = atomicAdd(grab, 1u);
    __syncthreads();
    unsigned int item = s_next;
    while (item < total) {
        const int k = (int)(item / ntiles);
        const int j = (int)(item - (unsigned int)k * ntiles);
        const int ty = j / tiles_x;
        const int tx = j - ty * tiles_x;
        const uint32_t t = t0 + (uint32_t)k;
        const bool run = budget == nullptr || t < *budget;   // the same for the whole block
        __syncthreads();   // s_next read; the previous item's draw is complete
        if (tid <= kWMaxChunks)
            sh.bins[tid] = 0;
        if (wp == 0) {
            // lane 31 takes the following item (none once a wait of the
            // launch gave up); lanes 0-8 wait for the 3 x 3 tiles around j
            if (lane == 31)
                s_next = ld_flag(err) ? total : atomicAdd(grab, 1u);
            bool ok = true;
            if (run && k > 0 && lane < 9) {
                const int yy = ty + lane / 3 - 1;
                const int xx = tx + lane % 3 - 1;
                if (yy >= 0 && yy < tiles_y && xx >= 0 && xx < tiles_x) {
                    const unsigned int *d = done + (size_t)yy * tiles_x + xx;
                    ok = wait_ge(d, (unsigned int)k, ld_acquire_u32(d), err, limit);
                }
            }
            if (!ok)
                atomicExch(err, 1);
            __syncwarp();
        } else if (wp == 1 && run) {
            block_uniforms(a, ty * kWY, tx * kWX, t, U_s);
        }
        __syncthreads();
        if (run) {
            const uint32_t ph = par_from_t ? (t & 1u) : (uint32_t)(k & 1);
            const uint8_t *xin = ph ? x1 : x0;
            uint8_t *xout = ph ? x0 : x1;
            const int r = ty * kWY + lr, c = tx * kWX + lc;
            const bool valid = r < a.H && c < a.W;
            SiteIn<NB> in{};
            if (valid) {
                load_site<NB, true, false>(a, xin, r, c, kTagPCA, t, in);
                in.ub = U_s[lr * kWX + lc];
            }
            const int s = win_draw<NB, LMASK>(sh, a.m, in, valid, tid, a.fp64_draws);
            if (valid) {
                xout[(size_t)r * a.pitch + c] = (uint8_t)s;
                if (accumulate_after(a, t)) {
                    float *p = a.acc + (size_t)r * a.W + c;
                    *p = __ldcg(p) + (float)s;
                }
            }
        }
        __syncthreads();
        // a skipped item publishes nothing: only later, also skipped, items of
        // the chain could depend on it, and an early count would let a
        // neighbour's item of an earlier sweep pass its wait too soon
        if (run && tid == 0 && j != a.stall_tile - 1) {
            __threadfence();   // the tile's labels and sums before its counter
            atomicExch(done + j, (unsigned int)(k + 1));
        }
        item = s_next;
    }
}

// Checkerboard Gibbs colour phase q in place on a.xin (Section 5.1): thread
// (x, y) owns a cell, two columns of a row (4 neighbours, colours (r + c)
// mod 2) or a 2 x 2 block (8 neighbours, colours (r mod 2, c mod 2)), and
// draws its site of colour q with the windowed draw; after the last phase
// (a.last_phase) it accumulates the whole cell.  A block covers 64 columns
// and 4 (8) rows; its phase sites' uniforms come from 64 Philox calls.
template <int NB, bool LMASK>
__global__ void __launch_bounds__(kWThreads, 8) gibbs_win_kernel(const SweepArgs a, int q,
                                                                 const float *ftab)
{
    __shared__ WinShared<NB> sh;
    __shared__ __align__(16) uint32_t U_s[kWY * 2 * kWX];   // 4 site rows x 64 columns
    const int lane = (int)threadIdx.x, wp = (int)threadIdx.y;
    const int tid = wp * kWX + lane;
    const int cx = (int)blockIdx.x * kWX + lane, cy = (int)blockIdx.y * kWY + wp;
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
    uint8_t *x = const_cast<uint8_t *>(a.xin);
    win_setup(sh, a.m.T, ftab, tid);
    const uint32_t t = sweep_index(a);
    if (wp < 2) {   // warp w, lane l: site row (32 w + l) / 16, columns 4 ((32 w + l) % 16) ..
        const int i = wp * 32 + lane;
        const int ri = i >> 4;
        const int row = NB == 4 ? (int)blockIdx.y * kWY + ri
                                : 2 * ((int)blockIdx.y * kWY + ri) + (q >> 1);
        uint32_t o0, o1, o2, o3;
        philox4x32_10((uint32_t)(16 * (int)blockIdx.x + (i & 15)), (uint32_t)(row + a.row_off), t,
                      (kTagGibbs << 24) | (a.chain & 0xFFFFFFu), (uint32_t)(a.seed & 0xFFFFFFFFull),
                      (uint32_t)(a.seed >> 32), o0, o1, o2, o3);
        reinterpret_cast<uint4 *>(U_s)[i] = make_uint4(o0 >> 8, o1 >> 8, o2 >> 8, o3 >> 8);
    }
    __syncthreads();
    const bool cell = r0 < a.H && c0 < a.W;
    const bool valid = cell && r < a.H && c < a.W;
    SiteIn<NB> in{};
    if (valid) {
        load_site<NB, false, false>(a, x, r, c, kTagGibbs, t, in);
        in.ub = U_s[wp * 2 * kWX + (c - 2 * kWX * (int)blockIdx.x)];
    }
    const int s = win_draw<NB, LMASK>(sh, a.m, in, valid, tid, a.fp64_draws);
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

// Wavefront form of the windowed Gibbs sweep: items (phase k, tile j) over
// the tiles of gibbs_win_kernel's blocks (64 columns x 4 or 8 rows), phase k
// being colour k mod (nbhd / 2) of sweep k / (nbhd / 2), in place.  Item
// (k, j) waits until the 3 x 3 tiles around j have finished phase k - 1:
// then the labels it reads are final and no neighbour still reads the ones
// it overwrites.  Waits bounded as pca_winw_kernel's; labels read through L2.
template <int NB, bool LMASK>
__global__ void __launch_bounds__(kWThreads, 8)
    gibbs_winw_kernel(const SweepArgs a, const float *ftab, uint8_t *x, int nphases, int tiles_x,
                      int tiles_y, unsigned int *done, unsigned int *grab, int *err)
{
    constexpr int kCol = NB == 4 ? 2 : 4;
    __shared__ WinShared<NB> sh;
    __shared__ __align__(16) uint32_t U_s[kWY * 2 * kWX];   // 4 site rows x 64 columns
    __shared__ unsigned int s_next;
    const int lane = (int)threadIdx.x, wp = (int)threadIdx.y;
    const int tid = wp * kWX + lane;
    const unsigned int ntiles = (unsigned int)(tiles_x * tiles_y);
    const unsigned int total = ntiles * (unsigned int)nphases;
    const uint32_t t0 = sweep_index(a);
    const long long limit = wait_limit(a.wait_ns);
    win_setup(sh, a.m.T, ftab, tid);
    if (tid == 0)
        s_next = atomicAdd(grab, 1u);
    __syncthreads();
    unsigned int item = s_next;
    while (item < total) {
        const int k = (int)(item / ntiles);
        const int j = (int)(item - (unsigned int)k * ntiles);
        const int ty = j / tiles_x;
        const int tx = j - ty * tiles_x;
        const int q = k % kCol;
        const uint32_t t = t0 + (uint32_t)(k / kCol);
        __syncthreads();   // s_next read; the previous item's draw is complete
        if (tid <= kWMaxChunks)
            sh.bins[tid] = 0;
        if (wp == 0) {
            if (lane == 31)
                s_next = ld_flag(err) ? total : atomicAdd(grab, 1u);
            bool ok = true;
            if (k > 0 && lane < 9) {
                const int yy = ty + lane / 3 - 1;
                const int xx = tx + lane % 3 - 1;
                if (yy >= 0 && yy < tiles_y && xx >= 0 && xx < tiles_x) {
                    const unsigned int *d = done + (size_t)yy * tiles_x + xx;
                    ok = wait_ge(d, (unsigned int)k, ld_acquire_u32(d), err, limit);
                }
            }
            if (!ok)
                atomicExch(err, 1);
            __syncwarp();
        } else if (wp == 1 || wp == 2) {   // 64 Philox calls: site rows of the phase
            const int i = (wp - 1) * 32 + lane;
            const int ri = i >> 4;
            const int row = NB == 4 ? ty * kWY + ri : 2 * (ty * kWY + ri) + (q >> 1);
            uint32_t o0, o1, o2, o3;
            philox4x32_10((uint32_t)(16 * tx + (i & 15)), (uint32_t)(row + a.row_off), t,
                          (kTagGibbs << 24) | (a.chain & 0xFFFFFFu),
                          (uint32_t)(a.seed & 0xFFFFFFFFull), (uint32_t)(a.seed >> 32), o0, o1,
                          o2, o3);
            reinterpret_cast<uint4 *>(U_s)[i] = make_uint4(o0 >> 8, o1 >> 8, o2 >> 8, o3 >> 8);
        }
        __syncthreads();
        const int cx = tx * kWX + lane, cy = ty * kWY + wp;
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
        SiteIn<NB> in{};
        if (valid) {
            load_site<NB, true, false>(a, x, r, c, kTagGibbs, t, in);
            in.ub = U_s[wp * 2 * kWX + (c - 2 * kWX * tx)];
        }
        const int s = win_draw<NB, LMASK>(sh, a.m, in, valid, tid, a.fp64_draws);
        if (valid)
            x[(size_t)r * a.pitch + c] = (uint8_t)s;
        if (cell && q == kCol - 1 && accumulate_after(a, t)) {
            const int nr = NB == 4 ? 1 : 2;
#pragma unroll
            for (int dr = 0; dr < nr; ++dr)
#pragma unroll
                for (int dc = 0; dc < 2; ++dc) {
                    const int rr = r0 + dr, cc = c0 + dc;
                    if (rr < a.H && cc < a.W) {
                        float *p = a.acc + (size_t)rr * a.W + cc;
                        const int v = (rr == r && cc == c) ? s : (int)__ldcg(x + (size_t)rr * a.pitch + cc);
                        *p = __ldcg(p) + (float)v;
                    }
                }
        }
        __syncthreads();
        if (tid == 0 && j != a.stall_tile - 1) {
            __threadfence();   // the tile's labels and sums before its counter
            atomicExch(done + j, (unsigned int)(k + 1));
        }
        item = s_next;
    }
}

template <int NB, bool LMASK>
cudaError_t launch_gibbs_win_t(const SweepArgs &a, int q, const float *ftab, cudaStream_t st)
{
    const dim3 block(kWX, kWY);
    const int rows = NB == 4 ? kWY : 2 * kWY;
    const dim3 grid((a.W + 2 * kWX - 1) / (2 * kWX), (a.H + rows - 1) / rows);
    if (grid.y > 65535u)
        return cudaErrorInvalidValue;
    gibbs_win_kernel<NB, LMASK><<<grid, block, 0, st>>>(a, q, ftab);
    return cudaGetLastError();
}

template <int NB, bool LMASK>
cudaError_t launch_win_t(const SweepArgs &a, const float *ftab, uint8_t *x0, uint8_t *x1,
                         const uint32_t *budget, cudaStream_t st)
{
    const dim3 block(kWX, kWY);
    const dim3 grid((a.W + kWX - 1) / kWX, (a.H + kWY - 1) / kWY);
    if (grid.y > 65535u)
        return cudaErrorInvalidValue;
    pca_win_kernel<NB, LMASK><<<grid, block, 0, st>>>(a, ftab, x0, x1, budget);
    return cudaGetLastError();
}

template <int NB, bool LMASK>
cudaError_t launch_winw_t(const SweepArgs &a, const float *ftab, uint8_t *x0, uint8_t *x1, int n,
                          unsigned int *done, unsigned int *grab, int *err, int par_from_t,
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
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pca_winw_kernel<NB, LMASK>,
                                                          kWThreads, 0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = nb > 0 ? nb : 1;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (a.W + kWX - 1) / kWX;
    const int tiles_y = (a.H + kWY - 1) / kWY;
    const long long items = (long long)tiles_x * tiles_y * n;
    if (items <= 0)
        return cudaSuccess;
    if (items >= (1ll << 32))
        return cudaErrorInvalidValue;
    // at most the resident capacity: every block that takes an item runs
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(items < cap ? items : cap);
    pca_winw_kernel<NB, LMASK><<<grid, dim3(kWX, kWY), 0, st>>>(
        a, ftab, x0, x1, n, tiles_x, tiles_y, done, grab, err, par_from_t, budget);
    return cudaGetLastError();
}

template <int NB, bool LMASK>
cudaError_t launch_gibbs_winw_t(const SweepArgs &a, const float *ftab, uint8_t *x, int nsweeps,
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
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gibbs_winw_kernel<NB, LMASK>,
                                                          kWThreads, 0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = nb > 0 ? nb : 1;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int rows = NB == 4 ? kWY : 2 * kWY;
    const int tiles_x = (a.W + 2 * kWX - 1) / (2 * kWX);
    const int tiles_y = (a.H + rows - 1) / rows;
    const int nphases = nsweeps * (NB == 4 ? 2 : 4);
    const long long items = (long long)tiles_x * tiles_y * nphases;
    if (items <= 0)
        return cudaSuccess;
    if (items >= (1ll << 32))
        return cudaErrorInvalidValue;
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(items < cap ? items : cap);
    gibbs_winw_kernel<NB, LMASK><<<grid, dim3(kWX, kWY), 0, st>>>(a, ftab, x, nphases, tiles_x,
                                                                  tiles_y, done, grab, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gibbs_winw(const SweepArgs &a, const float *ftab, uint8_t *x, int nsweeps,
                              unsigned int *done, unsigned int *grab, int *err, cudaStream_t st)
{
    if (!pca_win_eligible(a.m) || ftab == nullptr || nsweeps < 0)
        return cudaErrorInvalidValue;
    if (a.H <= 0 || a.W <= 0 || nsweeps == 0)
        return cudaSuccess;
    const bool lmask = (a.m.L % kChunk) != 0;
    if (a.m.nbhd == 8)
        return lmask ? launch_gibbs_winw_t<8, true>(a, ftab, x, nsweeps, done, grab, err, st)
                     : launch_gibbs_winw_t<8, false>(a, ftab, x, nsweeps, done, grab, err, st);
    return lmask ? launch_gibbs_winw_t<4, true>(a, ftab, x, nsweeps, done, grab, err, st)
                 : launch_gibbs_winw_t<4, false>(a, ftab, x, nsweeps, done, grab, err, st);
}

cudaError_t launch_pca_winw(const SweepArgs &a, const float *ftab, uint8_t *x0, uint8_t *x1,
                            int nsweeps, unsigned int *done, unsigned int *grab, int *err,
                            cudaStream_t st, const uint32_t *budget, bool par_from_t)
{
    if (!pca_win_eligible(a.m) || ftab == nullptr || nsweeps < 0)
        return cudaErrorInvalidValue;
    if (a.H <= 0 || a.W <= 0 || nsweeps == 0)
        return cudaSuccess;
    const bool lmask = (a.m.L % kChunk) != 0;
    const int par = par_from_t ? 1 : 0;
    if (a.m.nbhd == 8)
        return lmask ? launch_winw_t<8, true>(a, ftab, x0, x1, nsweeps, done, grab, err, par,
                                              budget, st)
                     : launch_winw_t<8, false>(a, ftab, x0, x1, nsweeps, done, grab, err, par,
                                               budget, st);
    return lmask ? launch_winw_t<4, true>(a, ftab, x0, x1, nsweeps, done, grab, err, par, budget,
                                          st)
                 : launch_winw_t<4, false>(a, ftab, x0, x1, nsweeps, done, grab, err, par,
                                           budget, st);
}

cudaError_t launch_gibbs_win(const SweepArgs &a, int q, const float *ftab, cudaStream_t st)
{
    if (!pca_win_eligible(a.m) || ftab == nullptr || q < 0 || q >= (a.m.nbhd == 8 ? 4 : 2))
        return cudaErrorInvalidValue;
    if (a.H <= 0 || a.W <= 0)
        return cudaSuccess;
    const bool lmask = (a.m.L % kChunk) != 0;
    if (a.m.nbhd == 8)
        return lmask ? launch_gibbs_win_t<8, true>(a, q, ftab, st)
                     : launch_gibbs_win_t<8, false>(a, q, ftab, st);
    return lmask ? launch_gibbs_win_t<4, true>(a, q, ftab, st)
                 : launch_gibbs_win_t<4, false>(a, q, ftab, st);
}

bool pca_win_eligible(const DevModel &m)
{
    return m.L >= kWinMinLabels && m.L <= 256 && m.T >= 1 && m.T <= kTcMaxT && m.norm == 0 &&
           (m.nbhd == 4 || m.nbhd == 8) && m.nbhd * m.T <= 255;
}

cudaError_t launch_pca_win(const SweepArgs &a, const float *ftab, cudaStream_t st, uint8_t *x0,
                           uint8_t *x1, const uint32_t *budget)
{
    if (!pca_win_eligible(a.m) || ftab == nullptr || (x0 == nullptr) != (x1 == nullptr))
        return cudaErrorInvalidValue;
    if (a.H <= 0 || a.W <= 0)
        return cudaSuccess;
    const bool lmask = (a.m.L % kChunk) != 0;
    if (a.m.nbhd == 8)
        return lmask ? launch_win_t<8, true>(a, ftab, x0, x1, budget, st)
                     : launch_win_t<8, false>(a, ftab, x0, x1, budget, st);
    return lmask ? launch_win_t<4, true>(a, ftab, x0, x1, budget, st)
                 : launch_win_t<4, false>(a, ftab, x0, x1, budget, st);
}

}  // namespace pcad
