// Sweep kernels: lazy PCA (Section 5.2) and checkerboard Gibbs (Section 5.1).
//
// One thread per site.  The site's labels, its neighbours' labels and its
// observation are read straight from global memory (each byte is reused by
// up to 9 threads through L1); the per-label work (energy, exponential, CDF)
// dominates for L >= 16.  The data-factor table lives in shared memory, as
// do the per-thread chunk prefix sums of the two-pass CDF.
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 4;
constexpr int kThreads = kBX * kBY;
constexpr int kTable = 511;

// Neighbour order: up, down, left, right, then the four diagonals.
template <int NB>
__device__ __forceinline__ void load_neighbours(const uint8_t *__restrict__ x, int pitch, int H,
                                                int W, int r, int c, float (&xn)[NB],
                                                int (&xni)[NB])
{
    constexpr int dr[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
    constexpr int dc[8] = {0, 0, -1, 1, -1, 1, -1, 1};
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int rr = r + dr[j];
        const int cc = c + dc[j];
        const bool in = rr >= 0 && rr < H && cc >= 0 && cc < W;
        const int v = in ? (int)x[(size_t)rr * pitch + cc] : kMissingLabelI;
        xni[j] = v;
        xn[j] = (float)v;
    }
}

__device__ __forceinline__ void load_table(float *ta_s, const float *ta32, int tid)
{
    for (int i = tid; i < kTable; i += kThreads)
        ta_s[i] = ta32[i];
}

template <int NC, int NB>
__device__ __forceinline__ int update_site(const SweepArgs &a, const uint8_t *x, const float *ta_s,
                                           float *Gcol, int r, int c, uint32_t tag, uint32_t t)
{
    float xn[NB];
    int xni[NB];
    load_neighbours<NB>(x, a.pitch, a.H, a.W, r, c, xn, xni);
    const size_t idx = (size_t)r * a.pitch + c;
    const int xi = x[idx];
    const int g = a.g[idx];
    const uint32_t ub = site_u24(a.seed, a.chain, tag, t, (uint32_t)r, (uint32_t)c);
    const float u = (float)ub * (1.0f / 16777216.0f);
    bool certain;
    int s = draw_fp32<NC, NB>(a.m, ta_s, Gcol, kThreads, g, xi, xn, u, certain);
    if (!certain) {
        s = draw_fp64<NB>(a.m, g, xi, xni, (double)ub * (1.0 / 16777216.0));
        atomicAdd(a.fp64_draws, 1ull);
    }
    return s;
}

template <int NC, int NB>
__global__ void __launch_bounds__(kThreads) pca_direct_kernel(const SweepArgs a)
{
    __shared__ float ta_s[kTable];
    __shared__ float G_s[NC * kThreads];
    const int tid = threadIdx.y * kBX + threadIdx.x;
    load_table(ta_s, a.m.ta32, tid);
    __syncthreads();
    const int c = blockIdx.x * kBX + threadIdx.x;
    const int r = blockIdx.y * kBY + threadIdx.y;
    if (r >= a.H || c >= a.W)
        return;
    const uint32_t t = sweep_index(a);
    const int s = update_site<NC, NB>(a, a.xin, ta_s, G_s + tid, r, c, kTagPCA, t);
    a.xout[(size_t)r * a.pitch + c] = (uint8_t)s;
    if (accumulate_after(a, t))
        a.acc[(size_t)r * a.W + c] += (float)s;
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
    __shared__ float ta_s[kTable];
    __shared__ float G_s[NC * kThreads];
    const int tid = threadIdx.y * kBX + threadIdx.x;
    load_table(ta_s, a.m.ta32, tid);
    __syncthreads();
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
    if (r0 >= a.H || c0 >= a.W)
        return;
    const uint32_t t = sweep_index(a);
    if (r < a.H && c < a.W) {
        const int s = update_site<NC, NB>(a, x, ta_s, G_s + tid, r, c, kTagGibbs, t);
        x[(size_t)r * a.pitch + c] = (uint8_t)s;
    }
    if (a.last_phase && accumulate_after(a, t)) {
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

template <int NC, int NB>
cudaError_t launch_pca_t(const SweepArgs &a, cudaStream_t st)
{
    dim3 block(kBX, kBY);
    dim3 grid((a.W + kBX - 1) / kBX, (a.H + kBY - 1) / kBY);
    pca_direct_kernel<NC, NB><<<grid, block, 0, st>>>(a);
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

cudaError_t launch_pca_sweep(const SweepArgs &a, cudaStream_t st)
{
    return a.m.nbhd == 8 ? dispatch_pca<8>(a, st) : dispatch_pca<4>(a, st);
}

cudaError_t launch_gibbs_phase(const SweepArgs &a, int q, cudaStream_t st)
{
    return a.m.nbhd == 8 ? dispatch_gibbs<8>(a, q, st) : dispatch_gibbs<4>(a, q, st);
}

}  // namespace pcad
