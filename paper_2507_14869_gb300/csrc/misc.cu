// Read-back kernels: posterior mean, label planes, label validation, and the
// image-quality metrics of Section 6 (PSNR, SSIM) in FP64.
#include "pcad_internal.h"

namespace pcad {

namespace {

__global__ void mean_kernel(const float *acc, float n, float *mean, long count)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count)
        mean[i] = acc[i] / n;
}

__global__ void labels_to_float_kernel(const uint8_t *x, int pitch, int H, int W, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c < W && r < H)
        out[(size_t)r * W + c] = (float)x[(size_t)r * pitch + c];
}

__global__ void check_labels_kernel(const uint8_t *x, int pitch, int H, int W, int L, int *bad)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c < W && r < H && (int)x[(size_t)r * pitch + c] >= L)
        atomicAdd(bad, 1);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// scratch[0] += sum of squared luminance errors; int max label at scratch[7]
__global__ void psnr_kernel(const float *est, const uint8_t *clean, long n, double inv,
                            double *scratch)
{
    double se = 0.0;
    int mx = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const double d = (double)est[i] * inv - (double)clean[i] * inv;
        se += d * d;
        mx = max(mx, (int)clean[i]);
    }
    se = warp_sum(se);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&scratch[0], se);
        atomicMax(reinterpret_cast<int *>(&scratch[7]), mx);
    }
}

// Gaussian window 11x11, sigma 1.5, normalised to sum 1 (filled by the host).
__constant__ double c_win[121];

// One thread per window position; scratch[1] += SSIM at that position.
__global__ void ssim_window_kernel(const float *est, const uint8_t *clean, int H, int W,
                                   double inv, double *scratch)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    double v = 0.0;
    if (j < W - 10 && i < H - 10) {
        double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
        for (int a = 0; a < 11; ++a) {
            for (int b = 0; b < 11; ++b) {
                const double w = c_win[a * 11 + b];
                const size_t k = (size_t)(i + a) * W + (j + b);
                const double x = (double)clean[k] * inv;
                const double y = (double)est[k] * inv;
                mx += w * x;
                my += w * y;
                sxx += w * x * x;
                syy += w * y * y;
                sxy += w * x * y;
            }
        }
        sxx -= mx * mx;
        syy -= my * my;
        sxy -= mx * my;
        const double c1 = 1e-4, c2 = 9e-4;
        v = ((2.0 * mx * my + c1) * (2.0 * sxy + c2)) /
            ((mx * mx + my * my + c1) * (sxx + syy + c2));
    }
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(&scratch[1], v);
}

// Single-window (printed) form for images smaller than the window: two-pass
// unbiased sample statistics.
__global__ void ssim_global_kernel(const float *est, const uint8_t *clean, long n, double inv,
                                   double *scratch)
{
    if (blockIdx.x != 0 || threadIdx.x != 0)
        return;
    double sx = 0, sy = 0;
    for (long i = 0; i < n; ++i) {
        sx += (double)clean[i] * inv;
        sy += (double)est[i] * inv;
    }
    const double mx = sx / (double)n, my = sy / (double)n;
    double vx = 0, vy = 0, cxy = 0;
    for (long i = 0; i < n; ++i) {
        const double dx = (double)clean[i] * inv - mx;
        const double dy = (double)est[i] * inv - my;
        vx += dx * dx;
        vy += dy * dy;
        cxy += dx * dy;
    }
    vx /= (double)(n - 1);
    vy /= (double)(n - 1);
    cxy /= (double)(n - 1);
    const double c1 = 1e-4, c2 = 9e-4;
    scratch[1] = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
}

__global__ void metrics_finish_kernel(const double *scratch, long n, long npos, double inv,
                                      double *out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0)
        return;
    const double mse = scratch[0] / (double)n;
    const int mxl = *reinterpret_cast<const int *>(&scratch[7]);
    const double peak = (double)mxl * inv;
    out[0] = mse == 0.0 ? (double)INFINITY : 20.0 * log10(peak / sqrt(mse));
    out[1] = npos > 0 ? scratch[1] / (double)npos : scratch[1];
}

bool g_win_ready = false;

}  // namespace

cudaError_t launch_mean(const float *acc, float n, float *mean, long count, cudaStream_t s)
{
    const int bs = 256;
    const long nb = (count + bs - 1) / bs;
    if (nb > 0)
        mean_kernel<<<(unsigned)nb, bs, 0, s>>>(acc, n, mean, count);
    return cudaGetLastError();
}

cudaError_t launch_labels_to_float(const uint8_t *x, int pitch, int H, int W, float *out,
                                   cudaStream_t s)
{
    dim3 grid((W + 255) / 256, H);
    labels_to_float_kernel<<<grid, 256, 0, s>>>(x, pitch, H, W, out);
    return cudaGetLastError();
}

cudaError_t launch_check_labels(const uint8_t *x, int pitch, int H, int W, int L, int *bad,
                                cudaStream_t s)
{
    dim3 grid((W + 255) / 256, H);
    check_labels_kernel<<<grid, 256, 0, s>>>(x, pitch, H, W, L, bad);
    return cudaGetLastError();
}

cudaError_t launch_metrics(const float *est, const uint8_t *clean, int H, int W, int L,
                           double *scratch, double *out, cudaStream_t s)
{
    cudaError_t e;
    if (!g_win_ready) {
        double w[121], g1[11], tot = 0.0;
        for (int a = 0; a < 11; ++a) {
            const double d = (double)a - 5.0;
            g1[a] = exp(-(d * d) / (2.0 * 1.5 * 1.5));
        }
        for (int a = 0; a < 11; ++a)
            for (int b = 0; b < 11; ++b) {
                w[a * 11 + b] = g1[a] * g1[b];
                tot += w[a * 11 + b];
            }
        for (int k = 0; k < 121; ++k)
            w[k] /= tot;
        e = cudaMemcpyToSymbol(c_win, w, sizeof(w));
        if (e != cudaSuccess)
            return e;
        g_win_ready = true;
    }
    e = cudaMemsetAsync(scratch, 0, 8 * sizeof(double), s);
    if (e != cudaSuccess)
        return e;
    const long n = (long)H * W;
    const double inv = 1.0 / (double)(L - 1);
    psnr_kernel<<<256, 256, 0, s>>>(est, clean, n, inv, scratch);
    long npos = 0;
    if (H >= 11 && W >= 11) {
        dim3 grid((W - 10 + 255) / 256, H - 10);
        ssim_window_kernel<<<grid, 256, 0, s>>>(est, clean, H, W, inv, scratch);
        npos = (long)(H - 10) * (W - 10);
    } else {
        ssim_global_kernel<<<1, 32, 0, s>>>(est, clean, n, inv, scratch);
    }
    metrics_finish_kernel<<<1, 32, 0, s>>>(scratch, n, npos, inv, out);
    return cudaGetLastError();
}

}  // namespace pcad
