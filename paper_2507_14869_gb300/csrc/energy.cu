// Posterior energy of a labelling and minimum-energy tracking.
//
//   H(x) = sum over unordered neighbour pairs <ij> of V(x_i, x_j) + sum_i U(g_i, x_i)
//
// is the energy of the posterior Gibbs measure pi_post ~ exp(-H) (Section 4,
// Eq. mrf_gauss_noise_posterior_distribution) with the per-edge pair weight
// of the single-site conditional (Eq. gibbs_sampler_elementary_step).  Each
// term is a model coefficient times an integer count:
//   pair sum: Potts -> pairs with equal labels (V = -c_P each),
//             truncated linear -> sum of min(|x_i - x_j|, T) (V = c_T each);
//   data sum: Gaussian -> sum of (g_i - x_i)^2 (U = that / (2 sigma^2)),
//             flip -> sites with x_i != g_i (U = -ln p there, -ln(1 - p) elsewhere);
//             none (prior only) -> 0.
// The sums are reduced exactly in 64-bit integers; H is combined from them
// in FP64 by one thread.  Pairs are counted once: right and down neighbours
// (and the two lower diagonals for the 8-neighbourhood), free boundary.
#include "pcad_internal.h"

namespace pcad {

namespace {

constexpr int kEThreads = 256;

__global__ void __launch_bounds__(kEThreads) energy_sums_kernel(const uint8_t *__restrict__ x,
                                                                const uint8_t *__restrict__ g,
                                                                int H, int W, int pitch,
                                                                EnergyCoef k,
                                                                unsigned long long *sums)
{
    uint32_t pair = 0, data = 0;   // per thread: <= 4 x 255 and <= 65025 per site
    const long n = (long)H * W;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / W);
        const int c = (int)(i - (long)r * W);
        const int xi = x[(size_t)r * pitch + c];
        const int gi = g[(size_t)r * pitch + c];
        const int dr[4] = {0, 1, 1, 1};
        const int dc[4] = {1, 0, 1, -1};
        const int npairs = k.nbhd == 8 ? 4 : 2;
        for (int e = 0; e < npairs; ++e) {
            const int rr = r + dr[e], cc = c + dc[e];
            if (rr < H && cc >= 0 && cc < W) {
                const int xj = x[(size_t)rr * pitch + cc];
                pair += k.potts ? (xi == xj ? 1u : 0u) : (uint32_t)min(abs(xi - xj), k.T);
            }
        }
        if (!k.none)
            data += k.gauss ? (uint32_t)((gi - xi) * (gi - xi)) : (gi != xi ? 1u : 0u);
    }
    // block reduction in 64 bits, one atomic per block and sum
    unsigned long long p64 = pair, d64 = data;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p64 += __shfl_down_sync(0xFFFFFFFFu, p64, o);
        d64 += __shfl_down_sync(0xFFFFFFFFu, d64, o);
    }
    __shared__ unsigned long long sp[kEThreads / 32], sd[kEThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sp[warp] = p64;
        sd[warp] = d64;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long P = 0, D = 0;
        for (int w = 0; w < kEThreads / 32; ++w) {
            P += sp[w];
            D += sd[w];
        }
        atomicAdd(&sums[0], P);
        atomicAdd(&sums[1], D);
    }
}

// H from the sums (the same operation order as the host-side description in
// EnergyCoef), then optionally: record it, compare with the running
// minimum, flag a new minimum.  Zeroes the sums for the next reduction.
__global__ void energy_finish_kernel(unsigned long long *sums, EnergyCoef k, double *out,
                                     EnergyTrack tr, const uint32_t *tdev, uint32_t sweep_off)
{
    const double pair = (double)sums[0];
    const double data = (double)sums[1];
    double e = __dmul_rn(k.pair_c, pair);
    if (k.gauss)
        e = __dadd_rn(e, __ddiv_rn(data, k.two_s2));
    else if (!k.none)
        e = __dadd_rn(e, __dadd_rn(__dmul_rn(k.lf_same, __dsub_rn((double)k.n_sites, data)),
                                   __dmul_rn(k.lf_diff, data)));
    if (out) {   // H and the two sums (exact in FP64: both are < 2^53)
        out[0] = e;
        out[1] = pair;
        out[2] = data;
    }
    if (tr.trace) {
        const unsigned int n = *tr.n;
        if (n < (unsigned int)tr.cap) {
            tr.trace[n] = e;
            *tr.n = n + 1;
        }
        const bool lower = e < *tr.best;
        if (lower) {
            *tr.best = e;
            *tr.best_sweep = (unsigned long long)(*tdev + sweep_off) + 1ull;
        }
        *tr.flag = lower ? 1 : 0;
    }
    sums[0] = 0;
    sums[1] = 0;
}

__global__ void copy_if_kernel(const uint8_t *__restrict__ x, uint8_t *__restrict__ xb, int H,
                               int W, int pitch, const int *flag)
{
    if (*flag == 0)
        return;
    const long n = (long)H * W;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / W);
        const int c = (int)(i - (long)r * W);
        xb[(size_t)r * pitch + c] = x[(size_t)r * pitch + c];
    }
}

int reduce_grid(long n)
{
    const long blocks = (n + kEThreads - 1) / kEThreads;
    return (int)(blocks < 1024 ? (blocks < 1 ? 1 : blocks) : 1024);
}

}  // namespace

EnergyCoef energy_coef(const pcad_model &m, long n_sites)
{
    EnergyCoef k{};
    k.potts = m.pair == PCAD_PAIR_POTTS;
    k.T = m.pair == PCAD_PAIR_POTTS ? 1 : m.pair_T;
    k.gauss = m.noise == PCAD_NOISE_GAUSS;
    k.none = m.noise == PCAD_NOISE_NONE;
    k.nbhd = m.nbhd;
    k.pair_c = (k.potts ? -1.0 : 1.0) * (double)m.pair_coef;
    k.two_s2 = 2.0 * (double)m.sigma * (double)m.sigma;
    if (m.noise == PCAD_NOISE_FLIP) {
        const double p = (double)m.flip_p;
        k.lf_same = -std::log1p(-p);
        k.lf_diff = -std::log(p);
    }
    k.n_sites = (unsigned long long)n_sites;
    return k;
}

cudaError_t launch_energy(const uint8_t *x, const uint8_t *g, int H, int W, int pitch,
                          const EnergyCoef &k, unsigned long long *sums, double *out,
                          const EnergyTrack &tr, const uint32_t *tdev, uint32_t sweep_off,
                          cudaStream_t s)
{
    const long n = (long)H * W;
    energy_sums_kernel<<<reduce_grid(n), kEThreads, 0, s>>>(x, g, H, W, pitch, k, sums);
    energy_finish_kernel<<<1, 1, 0, s>>>(sums, k, out, tr, tdev, sweep_off);
    if (tr.trace)
        copy_if_kernel<<<reduce_grid(n), kEThreads, 0, s>>>(x, tr.xb, H, W, pitch, tr.flag);
    return cudaGetLastError();
}

}  // namespace pcad
