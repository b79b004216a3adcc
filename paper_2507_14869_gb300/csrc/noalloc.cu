// pcad_pca_run_noalloc: the lazy-PCA chain without any device allocation.
//
// Some callers cannot allocate device memory on their own: an application
// whose framework already reserved the GPU's memory in its own pool, or a
// latency-bound loop that must never call cudaMalloc / cudaFree (they can
// synchronise the whole device and take milliseconds).  This entry point
// runs the same sweep kernels as pcad_chain_run with the caller's input and
// output buffers only.  The one extra label plane the synchronous update
// needs, the model tables and the counters live in a fixed-size array in the
// library's own device memory (`g_noalloc_scratch`, 8 MiB, held by every GPU
// that loads the library until the process exits).
//
// Every call reuses that array: two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it.  Each call
// re-initialises everything it reads (tables, counters, the accumulator in
// the caller's mean buffer) before its sweeps start.
//
// The host needs the array's device address: the first call on a device,
// with that device current, looks it up with cudaGetSymbolAddress and keeps
// it together with the device's current context (the array's host-side
// name is only a stand-in, not a device pointer).  If that context is later
// replaced (cudaDeviceReset, or a primary context released and created
// again, which reloads the module) the next call sees a different context
// and looks the address up again.  Make the first call on a device before
// any CUDA stream capture.
//
// The model tables reach the device as a kernel parameter, not by a copy
// from host memory, so no call reads host memory after it returns.
#include <cstring>
#include <mutex>
#include <vector>

#include "pcad_internal.h"

namespace {

constexpr size_t kScratchBytes = 8u << 20;             // 8 MiB
constexpr size_t kOffCounters = 0;                      // u32 sweep base, u64 FP64 re-draws
constexpr size_t kOffTa64 = 256;                        // 511 doubles
constexpr size_t kOffPr64 = kOffTa64 + 4096;            // up to 2041 doubles
constexpr int kPrMax = 2041;                            // nbhd * T + 1 with T <= 255
constexpr size_t kOffPlane = 32768;                     // the second label plane
constexpr size_t kPlaneMax = kScratchBytes - kOffPlane; // 8,355,840 bytes

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The FP64 tables of one call, passed by value (20 KB of kernel parameters).
struct NoallocTables {
    double ta64[511];
    double pr64[kPrMax];
    int npr;
};

__global__ void noalloc_tables_kernel(const __grid_constant__ NoallocTables t, double *ta,
                                      double *pr)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 511 + t.npr;
         i += gridDim.x * blockDim.x) {
        if (i < 511)
            ta[i] = t.ta64[i];
        else
            pr[i - 511] = t.pr64[i - 511];
    }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// The calling thread's current context (nullptr if it cannot be read).
CUcontext current_context()
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS)
        return nullptr;
    return c;
}

pcad_status scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return pcad::set_error(PCAD_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return pcad::set_error(PCAD_EINVAL, "device ordinal beyond 63");
    const CUcontext ctx = current_context();   // nullptr before the thread's first CUDA work
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // binds the device's context
        if (e != cudaSuccess || !p)
            return pcad::set_error(PCAD_ECUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                : "symbol address is NULL");
        g_scratch_addr[dev] = (unsigned char *)p;
        g_scratch_ctx[dev] = current_context();
    }
    *out = g_scratch_addr[dev];
    return PCAD_OK;
}

// [a, a + na) and [b, b + nb) share a byte.
bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

#define NA_TRY(call)                                                    \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess)                                          \
            return pcad::set_error(PCAD_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" pcad_status pcad_pca_run_noalloc(const uint8_t *g_dev, int H, int W, int pitch,
                                            const pcad_model *m, uint64_t seed,
                                            uint32_t chain_id, int nsweeps, int burn_in,
                                            uint8_t *sample_dev, float *mean_dev,
                                            void *cuda_stream)
{
    using namespace pcad;
    if (!g_dev || !sample_dev || !mean_dev)
        return set_error(PCAD_EINVAL, "g_dev, sample_dev and mean_dev must be device buffers");
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || pitch < W)
        return set_error(PCAD_EINVAL, "image size or pitch outside the limits");
    if ((size_t)pitch * (size_t)H > kPlaneMax)
        return set_error(PCAD_EINVAL, "pitch * H exceeds the 8,355,840-byte scratch plane");
    if (nsweeps < 0 || burn_in < 0)
        return set_error(PCAD_EINVAL, "nsweeps and burn_in must be >= 0");
    if (chain_id >= (1u << 24))
        return set_error(PCAD_EINVAL, "chain id must be < 2^24");
    pcad_status st = check_model(m);
    if (st != PCAD_OK)
        return st;
    if (m->sampler != PCAD_SAMPLER_PCA)
        return set_error(PCAD_EINVAL, "the allocation-free entry point runs the PCA sampler");
    if (m->inertia_norm != 0 && m->L > 2 && m->inertia > 0.0f)
        return set_error(PCAD_EINVAL, "the allocation-free entry point runs the L0 inertia price");
    const size_t plane_bytes = (size_t)pitch * (size_t)(H - 1) + (size_t)W;
    const size_t mean_bytes = (size_t)H * (size_t)W * sizeof(float);
    if (overlap(g_dev, plane_bytes, sample_dev, plane_bytes) ||
        overlap(g_dev, plane_bytes, mean_dev, mean_bytes) ||
        overlap(sample_dev, plane_bytes, mean_dev, mean_bytes))
        return set_error(PCAD_EINVAL, "g_dev, sample_dev and mean_dev must not overlap");
    const uint64_t n_acc = nsweeps > burn_in ? (uint64_t)(nsweeps - burn_in) : 0;
    if ((uint64_t)(m->L - 1) * n_acc >= (1ull << 24))
        return set_error(PCAD_EINVAL, "accumulator would leave the exact FP32 range");

    NoallocTables tabs{};
    std::vector<double> pr64;
    DevModel dm{};
    model_tables(*m, tabs.ta64, pr64, dm);
    if (pr64.size() > (size_t)kPrMax)
        return set_error(PCAD_EINVAL, "prior table exceeds its scratch slot");
    std::memcpy(tabs.pr64, pr64.data(), pr64.size() * sizeof(double));
    tabs.npr = (int)pr64.size();

    unsigned char *scr = nullptr;
    st = scratch_address(&scr);
    if (st != PCAD_OK)
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t *tdev = (uint32_t *)(scr + kOffCounters);
    unsigned long long *fp64 = (unsigned long long *)(scr + kOffCounters + 8);
    dm.ta64 = (const double *)(scr + kOffTa64);
    dm.pr64 = (const double *)(scr + kOffPr64);
    uint8_t *planes[2] = {sample_dev, (uint8_t *)(scr + kOffPlane)};

    NA_TRY(cudaMemsetAsync(scr + kOffCounters, 0, 16, s));
    noalloc_tables_kernel<<<4, 256, 0, s>>>(tabs, (double *)(scr + kOffTa64),
                                           (double *)(scr + kOffPr64));
    NA_TRY(cudaGetLastError());
    NA_TRY(cudaMemsetAsync(mean_dev, 0, (size_t)H * W * sizeof(float), s));
    NA_TRY(cudaMemcpy2DAsync(sample_dev, pitch, g_dev, pitch, W, H, cudaMemcpyDeviceToDevice, s));

    SweepArgs a{};
    a.g = g_dev;
    a.acc = mean_dev;
    a.fp64_draws = fp64;
    a.sweep_base = tdev;
    a.seed = seed;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.chain = chain_id;
    a.burn_in = burn_in;
    a.m = dm;
    int cur = 0;
    for (int k = 0; k < nsweeps; ++k) {
        a.sweep_off = (uint32_t)k;
        a.xin = planes[cur];
        a.xout = planes[cur ^ 1];
        NA_TRY(launch_pca_sweep(a, s));
        cur ^= 1;
    }
    if (cur != 0)
        NA_TRY(cudaMemcpy2DAsync(sample_dev, pitch, planes[1], pitch, W, H,
                                 cudaMemcpyDeviceToDevice, s));
    if (n_acc > 0)
        NA_TRY(launch_mean(mean_dev, (float)n_acc, mean_dev, (long)H * W, s));
    return PCAD_OK;
}
