// Whole chains of small two-label images in one CTA
// (lazy PCA, Section 5.2; checkerboard Gibbs, Section 5.1).
//
// A 64 x 64 binary chain does 4096 site-updates per sweep: one launch per
// sweep costs more than the sweep.  Here one CTA of 1024 threads holds the
// whole state in shared memory and runs every sweep of a run in one launch,
// with one block barrier per sweep (PCA) or colour phase (Gibbs).
//
// The draw.  With two labels the conditional law of site i depends on the
// site only through its configuration (x_i, g_i, n1, nm): n1 neighbours at
// label 1, nm neighbours outside the image (the rest at label 0).  The prior
// sums P(0) = n1 + nm T and P(1) = n0 + nm T are small integers, exact in
// FP32 in any order.  For one configuration the FP32 draw of the other
// kernels picks label 1 exactly when fl(fl(u 2^-24) Z) >= C0, a monotone
// test in the 24-bit uniform numerator u; its certified margin leaves one
// contiguous band [A, B) of u uncertain, where the FP64 re-draw decides,
// again by a monotone test (label 1 iff u >= D).  The whole draw therefore
// is "label 1 iff u >= max(A, min(D, B))", and the FP64 re-draw count is
// the number of draws with u in [A, B).  A set-up kernel finds A, B and D
// for every configuration by bisection over u, calling the very FP32 draw
// and FP64 re-draw functions the other kernels use, so the labels and the
// re-draw count are theirs draw for draw.
//
// The sweep.  Labels live in shared memory as bytes in padded rows (four
// zero bytes left and right of each row, a zero row above and below), so a
// thread reads the 4-site word of its quad and the words around it and
// counts the label-1 neighbours of its four sites with byte-wise integer
// adds (no carries: a count is at most 8).  A per-site base byte holds
// (g_i, nm) in the table's index.  One Philox call gives the quad's four
// uniforms of the sweep.  Posterior-mean counts accumulate in packed 16-bit
// registers and reach global memory at the end of the launch.
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kResThreads = 1024;
constexpr int kResMaxQuadsPerThread = 4;
constexpr int kResMaxSmem = 200 * 1024;

// Table entries: configuration index e = 2 (b + n1) + x_i with the base
// b = (g (NB + 1) + nm) (NB + 1).
template <int NB>
constexpr int btab_entries()
{
    return 4 * (NB + 1) * (NB + 1);
}
constexpr int kBtabStride = 4 * 9 * 9;   // entries per table in a batch's table array

__device__ unsigned long long g_btab_redraws;   // re-draw counter of the bisection (unused)

// One warp per configuration: A (first u with label 1 or an uncertain FP32
// draw), B (first u with a certain label 1), D (first u whose FP64 draw is
// label 1).  Entry {max(A, min(D, B)), A, B - A, 0}; impossible
// configurations (n1 + nm > NB) get zeros.
template <int NB>
__global__ void __launch_bounds__(256) btab_kernel(const DevModel m, uint4 *out)
{
    constexpr int NE = btab_entries<NB>();
    const int e = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    const int lane = (int)(threadIdx.x & 31u);
    if (e >= NE)
        return;   // whole warps
    const int xi = e & 1, v = e >> 1;
    const int n1 = v % (NB + 1), nm = (v / (NB + 1)) % (NB + 1), g = v / ((NB + 1) * (NB + 1));
    if (n1 + nm > NB) {
        if (lane == 0)
            out[e] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    SiteIn<NB> in{};
    in.g = g;
    in.xi = xi;
#pragma unroll
    for (int j = 0; j < NB; ++j)
        in.xni[j] = j < n1 ? 1 : (j < n1 + nm ? kMissingLabelI : 0);
    uint32_t bound[2];
#pragma unroll 1
    for (int which = 0; which < 2; ++which) {
        uint32_t lo = 0u, hi = 1u << 24;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            in.ub = mid;
            bool certain = true;
            const int s = draw_binary<NB>(m, in, certain);
            const bool hit = which == 0 ? (s == 1 || !certain) : (s == 1 && certain);
            if (hit)
                hi = mid;
            else
                lo = mid + 1u;
        }
        bound[which] = lo;
    }
    uint32_t lo = 0u, hi = 1u << 24;
    while (lo < hi) {   // warp-uniform: every lane holds the same bounds
        const uint32_t mid = (lo + hi) >> 1;
        in.ub = mid;
        int s = warp_redraw_fp64<NB>(m, lane == 0, in, 0, &g_btab_redraws);
        s = __shfl_sync(0xFFFFFFFFu, s, 0);
        if (s == 1)
            hi = mid;
        else
            lo = mid + 1u;
    }
    const uint32_t A = bound[0], B = bound[1], D = lo;
    if (lane == 0)
        out[e] = make_uint4(max(A, min(D, B)), A, B - A, 0u);
}

// Padded label plane: H + 2 rows of Wq + 8 bytes (Wq = W rounded up to 4).
inline int res_plane_bytes(int H, int W)
{
    return (H + 2) * (((W + 3) & ~3) + 8);
}

// Shared memory of a launch: table, one (Gibbs) or two (PCA) planes, base bytes.
inline int res_smem_bytes(int nb, bool gibbs, int H, int W)
{
    const int ne = 4 * (nb + 1) * (nb + 1);
    return ne * 16 + (gibbs ? 1 : 2) * res_plane_bytes(H, W) + H * ((W + 3) & ~3);
}

// Label-1 neighbour counts of the 4 sites of the word at index o (one per
// byte), from the padded plane X with pw words per row; M gets the word.
template <int NB>
__device__ __forceinline__ uint32_t quad_counts(const uint32_t *X, int o, int pw, uint32_t &M)
{
    M = X[o];
    const uint32_t U = X[o - pw], D = X[o + pw];
    uint32_t S = U + D + ((M << 8) | (X[o - 1] >> 24)) + ((M >> 8) | (X[o + 1] << 24));
    if (NB == 8)
        S += ((U << 8) | (X[o - pw - 1] >> 24)) + ((U >> 8) | (X[o - pw + 1] << 24)) +
             ((D << 8) | (X[o + pw - 1] >> 24)) + ((D >> 8) | (X[o + pw + 1] << 24));
    return S;
}

// New labels of the bytes of `act` (a byte mask) of one quad: S holds base +
// count per byte, M the current labels, u the uniforms.  Returns the labels
// as bytes (other bytes 0); adds the draws the FP64 re-draw decides to nre.
__device__ __forceinline__ uint32_t quad_draw(const uint4 *tab, uint32_t S, uint32_t M,
                                              const uint32_t (&u)[4], uint32_t act, uint32_t &nre)
{
    uint32_t out = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((act >> (8 * j)) & 1u) {
            const uint32_t key = ((S >> (8 * j)) & 0xFFu) * 2u + ((M >> (8 * j)) & 1u);
            const uint4 e = tab[key];
            out |= (u[j] >= e.x ? 1u : 0u) << (8 * j);
            nre += (u[j] - e.y) < e.z ? 1u : 0u;
        }
    }
    return out;
}

__device__ __forceinline__ void quad_uniforms(const SweepArgs &a, uint32_t tag, uint32_t t,
                                              int r, int c4, uint32_t (&u)[4])
{
    uint32_t o0, o1, o2, o3;
    philox4x32_10((uint32_t)c4, (uint32_t)(r + a.row_off), t, (tag << 24) | (a.chain & 0xFFFFFFu),
                  (uint32_t)(a.seed & 0xFFFFFFFFull), (uint32_t)(a.seed >> 32), o0, o1, o2, o3);
    u[0] = o0 >> 8;
    u[1] = o1 >> 8;
    u[2] = o2 >> 8;
    u[3] = o3 >> 8;
}

// Gibbs colour phase ph of a quad in row r: the bytes whose site has colour
// ph ((r + c) mod 2 for 4 neighbours, (r mod 2, c mod 2) for 8).
template <int NB>
__device__ __forceinline__ uint32_t phase_mask(int r, int ph)
{
    if (NB == 4)
        return ((r ^ ph) & 1) == 0 ? 0x00FF00FFu : 0xFF00FF00u;
    if ((r & 1) != (ph >> 1))
        return 0u;
    return (ph & 1) ? 0xFF00FF00u : 0x00FF00FFu;
}

// One CTA runs nsweeps sweeps of one chain from plane xg_in with the
// threshold table btab; the final labels go to xg_out (pitch a.pitch), the
// posterior-mean counts are added to a.acc and the re-draw count to
// a.fp64_draws.  Thread i takes the quads i, i + 1024, ... (QPT at most), a
// quad being 4 adjacent sites of a row.
template <int NB, bool GIBBS, int QPT>
__device__ __forceinline__ void resident_run(const SweepArgs &a, const uint4 *btab,
                                             const uint8_t *xg_in, uint8_t *xg_out, int nsweeps)
{
    extern __shared__ __align__(16) uint8_t sm[];
    constexpr int NE = btab_entries<NB>();
    const int tid = (int)threadIdx.x;
    const int H = a.H, W = a.W;
    const int Wq = (W + 3) & ~3, P = Wq + 8, pw = P >> 2;
    const int plane = (H + 2) * P;
    const int nplanes = GIBBS ? 1 : 2;
    uint4 *tab = reinterpret_cast<uint4 *>(sm);
    uint8_t *const pl0 = sm + NE * 16;
    uint8_t *const pl1 = pl0 + (GIBBS ? 0 : plane);
    uint8_t *const bs = pl0 + nplanes * plane;
    {
        uint32_t *z = reinterpret_cast<uint32_t *>(pl0);
        const int nz = (nplanes * plane + H * Wq) >> 2;
        for (int i = tid; i < nz; i += kResThreads)
            z[i] = 0u;   // borders, row padding and the base bytes of padding sites stay 0
        for (int i = tid; i < NE; i += kResThreads)
            tab[i] = btab[i];
    }
    __syncthreads();
    for (int i = tid; i < H * W; i += kResThreads) {
        const int r = i / W, c = i - (i / W) * W;
        const int gv = a.g[(size_t)r * a.pitch + c];
        pl0[(r + 1) * P + 4 + c] = xg_in[(size_t)r * a.pitch + c];
        int nm = (r == 0) + (r == H - 1) + (c == 0) + (c == W - 1);
        if (NB == 8)
            nm += (r == 0 || c == 0) + (r == 0 || c == W - 1) + (r == H - 1 || c == 0) +
                  (r == H - 1 || c == W - 1);
        bs[r * Wq + c] = (uint8_t)((gv * (NB + 1) + nm) * (NB + 1));
    }
    __syncthreads();

    const int qrow = Wq >> 2, nq = H * qrow;
    int qo[QPT], qr[QPT], qc[QPT];
    uint32_t qb[QPT], qm[QPT], clo[QPT], chi[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = tid + i * kResThreads;
        qo[i] = -1;
        qr[i] = qc[i] = 0;
        qb[i] = qm[i] = clo[i] = chi[i] = 0u;
        if (q < nq) {
            qr[i] = q / qrow;
            qc[i] = q - qr[i] * qrow;
            qo[i] = (qr[i] + 1) * pw + 1 + qc[i];
            qb[i] = reinterpret_cast<const uint32_t *>(bs)[q];
            const int nv = min(4, W - 4 * qc[i]);
            qm[i] = nv >= 4 ? 0xFFFFFFFFu : (1u << (8 * nv)) - 1u;
        }
    }
    const uint32_t t0 = sweep_index(a);
    const uint32_t tag = GIBBS ? kTagGibbs : kTagPCA;
    uint32_t nre = 0u;
    int cur = 0, nacc = 0;
    // add the counts of the 16-bit lanes to the accumulator and clear them
    auto flush = [&]() {
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            if (qo[i] < 0)
                continue;
            const uint32_t cnt[4] = {clo[i] & 0xFFFFu, chi[i] & 0xFFFFu, clo[i] >> 16,
                                     chi[i] >> 16};
            float *accq = a.acc + (size_t)qr[i] * W + 4 * qc[i];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (((qm[i] >> (8 * j)) & 1u) && cnt[j] != 0u)
                    accq[j] += (float)cnt[j];
            clo[i] = chi[i] = 0u;
        }
    };
    for (int k = 0; k < nsweeps; ++k) {
        const uint32_t t = t0 + (uint32_t)k;
        const bool acc_now = accumulate_after(a, t);
        uint32_t *X = reinterpret_cast<uint32_t *>(cur ? pl1 : pl0);
        if (!GIBBS) {
            uint32_t *Y = reinterpret_cast<uint32_t *>(cur ? pl0 : pl1);
#pragma unroll
            for (int i = 0; i < QPT; ++i) {
                if (qo[i] < 0)
                    continue;
                uint32_t u[4];
                quad_uniforms(a, tag, t, qr[i], qc[i], u);
                uint32_t M;
                const uint32_t S = quad_counts<NB>(X, qo[i], pw, M) + qb[i];
                const uint32_t nw = quad_draw(tab, S, M, u, qm[i], nre);
                Y[qo[i]] = nw;
                if (acc_now) {
                    clo[i] += nw & 0x00FF00FFu;
                    chi[i] += (nw >> 8) & 0x00FF00FFu;
                }
            }
            __syncthreads();
            cur ^= 1;
        } else {
            constexpr int kColours = NB == 4 ? 2 : 4;
            uint32_t u[QPT][4];
#pragma unroll
            for (int i = 0; i < QPT; ++i)
                if (qo[i] >= 0)
                    quad_uniforms(a, tag, t, qr[i], qc[i], u[i]);
#pragma unroll 1
            for (int ph = 0; ph < kColours; ++ph) {
#pragma unroll
                for (int i = 0; i < QPT; ++i) {
                    const uint32_t act = qo[i] < 0 ? 0u : phase_mask<NB>(qr[i], ph) & qm[i];
                    if (act == 0u)
                        continue;
                    uint32_t M;
                    const uint32_t S = quad_counts<NB>(X, qo[i], pw, M) + qb[i];
                    const uint32_t nw = quad_draw(tab, S, M, u[i], act, nre);
                    X[qo[i]] = (M & ~act) | nw;
                }
                __syncthreads();
            }
            if (acc_now) {
#pragma unroll
                for (int i = 0; i < QPT; ++i) {
                    if (qo[i] < 0)
                        continue;
                    const uint32_t w = X[qo[i]];
                    clo[i] += w & 0x00FF00FFu;
                    chi[i] += (w >> 8) & 0x00FF00FFu;
                }
            }
        }
        if (acc_now && ++nacc == 0xFFFF) {   // a 16-bit lane is full
            flush();
            nacc = 0;
        }
    }
    flush();
    const uint8_t *fin = cur ? pl1 : pl0;
    for (int i = tid; i < H * W; i += kResThreads) {
        const int r = i / W, c = i - (i / W) * W;
        xg_out[(size_t)r * a.pitch + c] = fin[(r + 1) * P + 4 + c];
    }
    const uint32_t warp_re = __reduce_add_sync(0xFFFFFFFFu, nre);
    if ((tid & 31) == 0 && warp_re != 0u)
        atomicAdd(a.fp64_draws, (unsigned long long)warp_re);
}

template <int NB, bool GIBBS, int QPT>
__global__ void __launch_bounds__(kResThreads, 1)
    resident_kernel(const SweepArgs a, const uint8_t *xg_in, uint8_t *xg_out, int nsweeps)
{
    resident_run<NB, GIBBS, QPT>(a, a.m.btab, xg_in, xg_out, nsweeps);
}

// Batched chains: CTA b runs chain idx[b] (a PCA slot) with the table
// tabs + b * kBtabStride, for the sweeps t0 .. t0 + n - 1 below the slot's
// budget (t0 its device sweep counter); the planes follow the counter.
template <int NB>
__global__ void __launch_bounds__(kResThreads, 1)
    resident_batch_kernel(const SlotDesc *slots, const int *idx, const uint4 *tabs, int n)
{
    const SlotDesc &d = slots[idx[blockIdx.x]];
    if (!d.active)
        return;
    const uint32_t t0 = *d.tdev, bud = *d.budget;
    const int nb = bud > t0 ? (int)min((uint32_t)n, bud - t0) : 0;
    if (nb == 0)
        return;
    SweepArgs a;
    slot_args(d, t0, a);
    a.sweep_base = d.tdev;
    a.sweep_off = 0u;
    a.last_phase = 0;
    resident_run<NB, false, kResMaxQuadsPerThread>(a, tabs + (size_t)blockIdx.x * kBtabStride,
                                                   d.x[t0 & 1u], d.x[(t0 + (uint32_t)nb) & 1u],
                                                   nb);
}

template <int NB, bool GIBBS, int QPT>
cudaError_t launch_res_t(const SweepArgs &a, const uint8_t *x_in, uint8_t *x_out, int n,
                         cudaStream_t st)
{
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64)
        return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(resident_kernel<NB, GIBBS, QPT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kResMaxSmem);
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    const int smem = res_smem_bytes(NB, GIBBS, a.H, a.W);
    resident_kernel<NB, GIBBS, QPT><<<1, kResThreads, smem, st>>>(a, x_in, x_out, n);
    return cudaGetLastError();
}

template <int NB, bool GIBBS>
cudaError_t launch_res_q(const SweepArgs &a, const uint8_t *x_in, uint8_t *x_out, int n,
                         cudaStream_t st)
{
    const int nq = a.H * (((a.W + 3) & ~3) >> 2);
    if (nq <= kResThreads)
        return launch_res_t<NB, GIBBS, 1>(a, x_in, x_out, n, st);
    if (nq <= 2 * kResThreads)
        return launch_res_t<NB, GIBBS, 2>(a, x_in, x_out, n, st);
    return launch_res_t<NB, GIBBS, kResMaxQuadsPerThread>(a, x_in, x_out, n, st);
}

// ------------------------------------------------------- large images
// Two labels on images too large for one CTA: one launch per sweep, the
// same threshold table (a table read and a compare per site), persistent
// blocks of 256 threads over tiles of 16 rows x 128 columns.  A block stages
// its tile's label words with a one-word halo in shared memory (words
// outside the image and bytes beyond W read as zero: a missing neighbour
// counts as no label-1 neighbour, and its absence enters through nm), and
// each thread takes two quads: neighbour counts by byte-wise adds, the base
// (g (NB + 1) + nm) (NB + 1) from the observation word (g < 2, checked at
// chain creation), one Philox call, four table reads, one 32-bit label
// store and one float4 accumulator update.  The next tile's label words are
// loaded into registers during the draws, and a tile's observation words
// and accumulator sums before them.
constexpr int kBinThreads = 256;
constexpr int kBinRows = 16;
constexpr int kBinQW = 32;                 // quads (4-site words) per tile row
constexpr int kBinPW = kBinQW + 2;         // staged words per row
constexpr int kBinWords = (kBinRows + 2) * kBinPW;

// Planes: a.xin -> a.xout, or (x0 != nullptr) x0 / x1 holding the states of
// even / odd sweep indices; budget (optional): a sweep with index >= *budget
// is skipped (a chain of a batch or of the server).
template <int NB>
__global__ void __launch_bounds__(kBinThreads)
    pca_binary_kernel(const SweepArgs a, int tiles_x, int ntiles, int acc_vec, uint8_t *x0,
                      uint8_t *x1, const uint32_t *budget)
{
    constexpr int NE = btab_entries<NB>();
    __shared__ uint4 tab[NE];
    __shared__ uint32_t X[kBinWords];
    const int tid = (int)threadIdx.x;
    const uint32_t t = sweep_index(a);
    if (budget && t >= *budget)
        return;   // the whole launch, before any barrier
    const uint8_t *xin = x0 ? ((t & 1u) ? x1 : x0) : a.xin;
    uint8_t *xout = x0 ? ((t & 1u) ? x0 : x1) : a.xout;
    for (int i = tid; i < NE; i += kBinThreads)
        tab[i] = a.m.btab[i];
    const bool acc_on = accumulate_after(a, t);
    const int H = a.H, W = a.W, pitch = a.pitch;
    const int Wq = (W + 3) >> 2;
    uint32_t nre = 0u;
    constexpr int kSlots = (kBinWords + kBinThreads - 1) / kBinThreads;
    // the label words of a tile into registers (issued early, stored later)
    auto stage_load = [&](int tile, uint32_t (&pw)[kSlots]) {
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int r0 = ty * kBinRows, q0 = tx * kBinQW;
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            const int i = tid + sl * kBinThreads;
            pw[sl] = 0u;
            if (i < kBinWords) {
                const int lr = i / kBinPW, lw = i - lr * kBinPW;
                const int gr = r0 - 1 + lr, gq = q0 - 1 + lw;
                if (gr >= 0 && gr < H && gq >= 0 && gq < Wq) {
                    uint32_t w = *reinterpret_cast<const uint32_t *>(xin + (size_t)gr * pitch + 4 * gq);
                    const int nv = W - 4 * gq;
                    if (nv < 4)
                        w &= (1u << (8 * nv)) - 1u;
                    pw[sl] = w;
                }
            }
        }
    };
    uint32_t pw[kSlots];
    int tile = (int)blockIdx.x;
    if (tile < ntiles)
        stage_load(tile, pw);
    for (; tile < ntiles; tile += (int)gridDim.x) {
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int r0 = ty * kBinRows, q0 = tx * kBinQW;
        __syncthreads();   // the table is in place; the last tile's words are read
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            const int i = tid + sl * kBinThreads;
            if (i < kBinWords)
                X[i] = pw[sl];
        }
        __syncthreads();
        if (tile + (int)gridDim.x < ntiles)
            stage_load(tile + (int)gridDim.x, pw);   // in flight during the draws
        constexpr int kQ = kBinRows * kBinQW / kBinThreads;
        uint32_t Gw[kQ];
        float4 A4[kQ];
#pragma unroll
        for (int qi = 0; qi < kQ; ++qi) {   // the quads' observations and sums, issued first
            const int k = tid + qi * kBinThreads;
            const int lr = k / kBinQW, lq = k - lr * kBinQW;
            const int gr = r0 + lr, gq = q0 + lq;
            Gw[qi] = 0u;
            A4[qi] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (gr < H && gq < Wq) {
                Gw[qi] = *reinterpret_cast<const uint32_t *>(a.g + (size_t)gr * pitch + 4 * gq);
                if (acc_on && acc_vec && 4 * gq + 4 <= W)
                    A4[qi] = *reinterpret_cast<const float4 *>(a.acc + (size_t)gr * W + 4 * gq);
            }
        }
#pragma unroll
        for (int qi = 0; qi < kQ; ++qi) {
            const int k = tid + qi * kBinThreads;
            const int lr = k / kBinQW, lq = k - lr * kBinQW;
            const int gr = r0 + lr, gq = q0 + lq;
            if (gr >= H || gq >= Wq)
                continue;
            const int nv = min(4, W - 4 * gq);
            const uint32_t act = nv >= 4 ? 0xFFFFFFFFu : (1u << (8 * nv)) - 1u;
            uint32_t M;
            uint32_t S = quad_counts<NB>(X, (lr + 1) * kBinPW + 1 + lq, kBinPW, M);
            S += (Gw[qi] & act & 0x01010101u) * (uint32_t)((NB + 1) * (NB + 1));
            if (gr == 0 || gr == H - 1 || gq == 0 || 4 * gq + 4 >= W) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = 4 * gq + j;
                    int nm = (gr == 0) + (gr == H - 1) + (c == 0) + (c == W - 1);
                    if (NB == 8)
                        nm += (gr == 0 || c == 0) + (gr == 0 || c == W - 1) +
                              (gr == H - 1 || c == 0) + (gr == H - 1 || c == W - 1);
                    S += (uint32_t)(nm * (NB + 1)) << (8 * j);
                }
            }
            uint32_t u[4];
            quad_uniforms(a, kTagPCA, t, gr, gq, u);
            const uint32_t nw = quad_draw(tab, S, M, u, act, nre);
            uint8_t *out = xout + (size_t)gr * pitch + 4 * gq;
            float *acc = a.acc + (size_t)gr * W + 4 * gq;
            if (nv >= 4) {
                *reinterpret_cast<uint32_t *>(out) = nw;
                if (acc_on) {
                    const float l0 = (float)(nw & 0xFFu), l1 = (float)((nw >> 8) & 0xFFu),
                                l2 = (float)((nw >> 16) & 0xFFu), l3 = (float)(nw >> 24);
                    if (acc_vec) {
                        const float4 v = A4[qi];
                        *reinterpret_cast<float4 *>(acc) =
                            make_float4(v.x + l0, v.y + l1, v.z + l2, v.w + l3);
                    } else {
                        acc[0] += l0;
                        acc[1] += l1;
                        acc[2] += l2;
                        acc[3] += l3;
                    }
                }
            } else {
                for (int j = 0; j < nv; ++j) {
                    const uint32_t sl = (nw >> (8 * j)) & 0xFFu;
                    out[j] = (uint8_t)sl;
                    if (acc_on)
                        acc[j] += (float)sl;
                }
            }
        }
    }
    const uint32_t warp_re = __reduce_add_sync(0xFFFFFFFFu, nre);
    if ((tid & 31) == 0 && warp_re != 0u)
        atomicAdd(a.fp64_draws, (unsigned long long)warp_re);
}

template <int NB>
cudaError_t launch_binary_t(const SweepArgs &a, uint8_t *x0, uint8_t *x1, const uint32_t *budget,
                            cudaStream_t st)
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
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pca_binary_kernel<NB>, kBinThreads,
                                                          0);
        if (e != cudaSuccess)
            return e;
        per_sm[dev] = n > 0 ? n : 1;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int Wq = (a.W + 3) >> 2;
    const int tiles_x = (Wq + kBinQW - 1) / kBinQW;
    const long long ntiles = (long long)tiles_x * ((a.H + kBinRows - 1) / kBinRows);
    if (ntiles <= 0)
        return cudaSuccess;
    if (ntiles >= (1ll << 31))
        return cudaErrorInvalidValue;
    const long long cap = (long long)per_sm[dev] * sms;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    const int acc_vec = (a.W % 4 == 0 && (reinterpret_cast<uintptr_t>(a.acc) & 15u) == 0) ? 1 : 0;
    pca_binary_kernel<NB><<<grid, kBinThreads, 0, st>>>(a, tiles_x, (int)ntiles, acc_vec, x0, x1,
                                                        budget);
    return cudaGetLastError();
}

}  // namespace

int btab_bytes()
{
    return kBtabStride * 16;
}

cudaError_t launch_btab(const DevModel &m, uint4 *out, cudaStream_t st)
{
    if (m.L != 2 || (m.nbhd != 4 && m.nbhd != 8))
        return cudaErrorInvalidValue;
    const int ne = m.nbhd == 8 ? btab_entries<8>() : btab_entries<4>();
    const int grid = (ne + 7) / 8;   // 8 warps per block, one per configuration
    if (m.nbhd == 8)
        btab_kernel<8><<<grid, 256, 0, st>>>(m, out);
    else
        btab_kernel<4><<<grid, 256, 0, st>>>(m, out);
    return cudaGetLastError();
}

bool resident_fits(int L, int nbhd, int H, int W)
{
    if (L != 2 || (nbhd != 4 && nbhd != 8))
        return false;
    if ((long long)H * (((W + 3) & ~3) >> 2) > (long long)kResMaxQuadsPerThread * kResThreads)
        return false;
    return res_smem_bytes(nbhd, false, H, W) <= kResMaxSmem;
}

int resident_smem_bytes(int nbhd, int H, int W)
{
    return res_smem_bytes(nbhd, false, H, W);
}

cudaError_t launch_resident_batch(const SlotDesc *slots, const int *idx, const uint4 *tabs,
                                  int count, int nbhd, int n, int smem, cudaStream_t st)
{
    if (count <= 0 || n <= 0)
        return cudaSuccess;
    if ((nbhd != 4 && nbhd != 8) || smem > kResMaxSmem)
        return cudaErrorInvalidValue;
    static bool attr_set[2][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64)
        return cudaErrorInvalidDevice;
    const int k = nbhd == 8 ? 1 : 0;
    if (!attr_set[k][dev]) {
        e = nbhd == 8 ? cudaFuncSetAttribute(resident_batch_kernel<8>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kResMaxSmem)
                      : cudaFuncSetAttribute(resident_batch_kernel<4>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kResMaxSmem);
        if (e != cudaSuccess)
            return e;
        attr_set[k][dev] = true;
    }
    if (nbhd == 8)
        resident_batch_kernel<8><<<count, kResThreads, smem, st>>>(slots, idx, tabs, n);
    else
        resident_batch_kernel<4><<<count, kResThreads, smem, st>>>(slots, idx, tabs, n);
    return cudaGetLastError();
}

bool resident_eligible(const DevModel &m, int H, int W)
{
    if (m.L != 2 || m.norm != 0 || (m.nbhd != 4 && m.nbhd != 8) || m.btab == nullptr)
        return false;
    if ((long long)H * (((W + 3) & ~3) >> 2) > (long long)kResMaxQuadsPerThread * kResThreads)
        return false;
    return res_smem_bytes(m.nbhd, false, H, W) <= kResMaxSmem;
}

cudaError_t launch_resident(const SweepArgs &a, const uint8_t *x_in, uint8_t *x_out, int nsweeps,
                            bool gibbs, cudaStream_t st)
{
    if (!resident_eligible(a.m, a.H, a.W) || nsweeps < 0)
        return cudaErrorInvalidValue;
    if (nsweeps == 0)
        return cudaSuccess;
    if (a.m.nbhd == 8)
        return gibbs ? launch_res_q<8, true>(a, x_in, x_out, nsweeps, st)
                     : launch_res_q<8, false>(a, x_in, x_out, nsweeps, st);
    return gibbs ? launch_res_q<4, true>(a, x_in, x_out, nsweeps, st)
                 : launch_res_q<4, false>(a, x_in, x_out, nsweeps, st);
}

bool binary_eligible(const DevModel &m)
{
    return m.L == 2 && m.norm == 0 && (m.nbhd == 4 || m.nbhd == 8) && m.btab != nullptr;
}

cudaError_t launch_pca_binary(const SweepArgs &a, cudaStream_t st, uint8_t *x0, uint8_t *x1,
                              const uint32_t *budget)
{
    if (!binary_eligible(a.m))
        return cudaErrorInvalidValue;
    // word loads and stores of the planes
    const uintptr_t planes = x0 ? (reinterpret_cast<uintptr_t>(x0) | reinterpret_cast<uintptr_t>(x1))
                                : (reinterpret_cast<uintptr_t>(a.xin) |
                                   reinterpret_cast<uintptr_t>(a.xout));
    if ((a.pitch & 3) != 0 || ((planes | reinterpret_cast<uintptr_t>(a.g)) & 3u) != 0)
        return cudaErrorMisalignedAddress;
    return a.m.nbhd == 8 ? launch_binary_t<8>(a, x0, x1, budget, st)
                         : launch_binary_t<4>(a, x0, x1, budget, st);
}

}  // namespace pcad
