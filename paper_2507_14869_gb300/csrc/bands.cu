// Row-band decomposition of one image over several chains (and devices).
//
// The lazy PCA draws every site from the previous configuration only
// (Section 3, Eq. general_pca_definition; the synchronous update of Section
// 5.2), so after k sweeps a site's label depends only on the sites within k
// rows of it.  An H x W image is split into nbands bands of whole rows: band
// b owns rows [o_b, o_{b+1}), o_b = floor(b H / nbands), and runs an ordinary
// chain on the rows [o_b - h, o_{b+1} + h) clipped to the image, h = `halo`.
// That chain treats the ends of its buffer as a free boundary, which is wrong
// only for the halo rows: after k <= h sweeps the error has moved k rows in,
// so the owned rows are exact.  Every block of h sweeps therefore ends with
// one exchange step: each band copies, from its neighbours' planes, the
// owned rows its halos mirror (device to device; a peer copy when the bands
// live on different GPUs).  Philox rows are global (each band chain has a row
// offset), so every owned row -- labels at every sweep, hence also its
// posterior-mean accumulator -- equals the whole-image chain's bit for bit.
//
// Ordering per block, all stream-ordered: every band runs its h sweeps and
// records `done`; each band waits for its neighbours' `done`, copies their
// rows into its halos and records `copied`; each band then waits for its
// neighbours' `copied` before its next block, so no band overwrites a plane
// a neighbour is still reading.
#include <algorithm>
#include <vector>

#include "pcad_internal.h"

using namespace pcad;

struct pcad_bands {
    int n = 0, H = 0, W = 0, halo = 0;
    std::vector<pcad_chain *> ch;
    std::vector<int> own0, own1, buf0, buf1, dev;
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> done, copied;
    uint64_t t = 0;
};

namespace {

constexpr int kMaxBands = 64;
constexpr int kMaxHalo = 64;

#define BD_TRY(call)                                                    \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess)                                          \
            return set_error(PCAD_ECUDA, cudaGetErrorString(e_));       \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int saved = 0;
    bool ok = false;
    DeviceGuard() { ok = cudaGetDevice(&saved) == cudaSuccess; }
    ~DeviceGuard()
    {
        if (ok)
            cudaSetDevice(saved);
    }
};

void free_bands(pcad_bands *b)
{
    for (int i = 0; i < (int)b->ch.size(); ++i) {
        if (!b->dev.empty())
            cudaSetDevice(b->dev[i]);
        if (b->ch[i])
            pcad_chain_destroy(b->ch[i]);
        if (i < (int)b->done.size() && b->done[i])
            cudaEventDestroy(b->done[i]);
        if (i < (int)b->copied.size() && b->copied[i])
            cudaEventDestroy(b->copied[i]);
        if (i < (int)b->st.size() && b->st[i])
            cudaStreamDestroy(b->st[i]);
    }
    delete b;
}

// Copy global rows [r0, r1) of band `from`'s current state into band `to`'s
// plane (both hold those rows), on band `to`'s stream.
pcad_status copy_rows(pcad_bands *b, int from, int to, int r0, int r1)
{
    if (r1 <= r0)
        return PCAD_OK;
    const uint8_t *src = chain_state(b->ch[from]) + (size_t)(r0 - b->buf0[from]) *
                                                        chain_pitch(b->ch[from]);
    uint8_t *dst = chain_state(b->ch[to]) + (size_t)(r0 - b->buf0[to]) * chain_pitch(b->ch[to]);
    BD_TRY(cudaMemcpy2DAsync(dst, chain_pitch(b->ch[to]), src, chain_pitch(b->ch[from]), b->W,
                             r1 - r0, cudaMemcpyDefault, b->st[to]));
    return PCAD_OK;
}

}  // namespace

extern "C" {

pcad_status pcad_bands_create(const uint8_t *g_host, int H, int W, int g_pitch,
                              const pcad_model *m, uint64_t seed, uint32_t chain_id, int burn_in,
                              int nbands, int halo, const int *devices, pcad_bands **out)
{
    if (!out)
        return set_error(PCAD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g_host || !m)
        return set_error(PCAD_EINVAL, "NULL argument");
    if (H < 1 || W < 1 || g_pitch < W)
        return set_error(PCAD_EINVAL, "image size or pitch outside the limits");
    if (nbands < 1 || nbands > kMaxBands || halo < 1 || halo > kMaxHalo)
        return set_error(PCAD_EINVAL, "nbands must lie in [1, 64] and halo in [1, 64]");
    if (nbands > 1 && H / nbands < halo)
        return set_error(PCAD_EINVAL, "every band must own at least `halo` rows");
    if (m->sampler != PCAD_SAMPLER_PCA)
        return set_error(PCAD_EINVAL, "row bands run the lazy PCA sampler");
    DeviceGuard guard;
    if (!guard.ok)
        return set_error(PCAD_ECUDA, "no current device");
    pcad_bands *b = new pcad_bands();
    b->n = nbands;
    b->H = H;
    b->W = W;
    b->halo = halo;
    b->ch.assign(nbands, nullptr);
    b->st.assign(nbands, nullptr);
    b->done.assign(nbands, nullptr);
    b->copied.assign(nbands, nullptr);
    for (int i = 0; i < nbands; ++i) {
        b->own0.push_back((int)((long long)i * H / nbands));
        b->own1.push_back((int)((long long)(i + 1) * H / nbands));
        b->buf0.push_back(std::max(0, b->own0[i] - halo));
        b->buf1.push_back(std::min(H, b->own1[i] + halo));
        b->dev.push_back(devices ? devices[i] : guard.saved);
    }
    for (int i = 0; i < nbands; ++i) {
        cudaError_t e = cudaSetDevice(b->dev[i]);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->copied[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            free_bands(b);
            return set_error(PCAD_ECUDA, cudaGetErrorString(e));
        }
        // neighbours on other devices read this one's plane directly when they can
        for (int j : {i - 1, i + 1}) {
            if (j < 0 || j >= nbands || b->dev[j] == b->dev[i])
                continue;
            int can = 0;
            if (cudaDeviceCanAccessPeer(&can, b->dev[i], b->dev[j]) == cudaSuccess && can)
                cudaDeviceEnablePeerAccess(b->dev[j], 0);
            cudaGetLastError();   // "already enabled" is not an error here
        }
        pcad_status s = pcad_chain_create(g_host + (size_t)b->buf0[i] * g_pitch,
                                          b->buf1[i] - b->buf0[i], W, g_pitch, m, seed, chain_id,
                                          burn_in, b->st[i], &b->ch[i]);
        if (s == PCAD_OK)
            s = pcad_chain_set_row_offset(b->ch[i], b->buf0[i]);
        if (s != PCAD_OK) {
            free_bands(b);
            return s;
        }
    }
    *out = b;
    return PCAD_OK;
}

pcad_status pcad_bands_run(pcad_bands *b, int nsweeps)
{
    if (!b)
        return set_error(PCAD_EINVAL, "bands is NULL");
    if (nsweeps < 0)
        return set_error(PCAD_EINVAL, "nsweeps < 0");
    DeviceGuard guard;
    for (int left = nsweeps; left > 0;) {
        const int k = std::min(b->halo, left);
        for (int i = 0; i < b->n; ++i) {
            BD_TRY(cudaSetDevice(b->dev[i]));
            pcad_status s = pcad_chain_run(b->ch[i], k);
            if (s != PCAD_OK)
                return s;
            BD_TRY(cudaEventRecord(b->done[i], b->st[i]));
        }
        if (b->n > 1) {
            // the exchange step: halos from the neighbours' owned rows
            for (int i = 0; i < b->n; ++i) {
                BD_TRY(cudaSetDevice(b->dev[i]));
                if (i > 0) {
                    BD_TRY(cudaStreamWaitEvent(b->st[i], b->done[i - 1], 0));
                    pcad_status s = copy_rows(b, i - 1, i, b->buf0[i], b->own0[i]);
                    if (s != PCAD_OK)
                        return s;
                }
                if (i + 1 < b->n) {
                    BD_TRY(cudaStreamWaitEvent(b->st[i], b->done[i + 1], 0));
                    pcad_status s = copy_rows(b, i + 1, i, b->own1[i], b->buf1[i]);
                    if (s != PCAD_OK)
                        return s;
                }
                BD_TRY(cudaEventRecord(b->copied[i], b->st[i]));
            }
            // no band overwrites its plane while a neighbour still reads it
            for (int i = 0; i < b->n; ++i) {
                BD_TRY(cudaSetDevice(b->dev[i]));
                if (i > 0)
                    BD_TRY(cudaStreamWaitEvent(b->st[i], b->copied[i - 1], 0));
                if (i + 1 < b->n)
                    BD_TRY(cudaStreamWaitEvent(b->st[i], b->copied[i + 1], 0));
            }
        }
        left -= k;
    }
    b->t += (uint64_t)nsweeps;
    return PCAD_OK;
}

pcad_status pcad_bands_sync(pcad_bands *b)
{
    if (!b)
        return set_error(PCAD_EINVAL, "bands is NULL");
    DeviceGuard guard;
    pcad_status first = PCAD_OK;
    for (int i = 0; i < b->n; ++i) {
        BD_TRY(cudaSetDevice(b->dev[i]));
        const pcad_status s = pcad_chain_sync(b->ch[i]);
        if (first == PCAD_OK)
            first = s;
    }
    return first;
}

pcad_status pcad_bands_read_sample(pcad_bands *b, uint8_t *host_out, int out_pitch)
{
    if (!b || !host_out)
        return set_error(PCAD_EINVAL, "NULL argument");
    if (out_pitch < b->W)
        return set_error(PCAD_EINVAL, "out_pitch < W");
    DeviceGuard guard;
    std::vector<uint8_t> tmp;
    for (int i = 0; i < b->n; ++i) {
        BD_TRY(cudaSetDevice(b->dev[i]));
        tmp.resize((size_t)(b->buf1[i] - b->buf0[i]) * b->W);
        pcad_status s = pcad_chain_read_sample(b->ch[i], tmp.data(), b->W);
        if (s != PCAD_OK)
            return s;
        for (int r = b->own0[i]; r < b->own1[i]; ++r)
            std::copy_n(tmp.data() + (size_t)(r - b->buf0[i]) * b->W, b->W,
                        host_out + (size_t)r * out_pitch);
    }
    return PCAD_OK;
}

pcad_status pcad_bands_read_mean(pcad_bands *b, float *host_out)
{
    if (!b || !host_out)
        return set_error(PCAD_EINVAL, "NULL argument");
    DeviceGuard guard;
    std::vector<float> tmp;
    for (int i = 0; i < b->n; ++i) {
        BD_TRY(cudaSetDevice(b->dev[i]));
        tmp.resize((size_t)(b->buf1[i] - b->buf0[i]) * b->W);
        pcad_status s = pcad_chain_read_mean(b->ch[i], tmp.data());
        if (s != PCAD_OK)
            return s;
        for (int r = b->own0[i]; r < b->own1[i]; ++r)
            std::copy_n(tmp.data() + (size_t)(r - b->buf0[i]) * b->W, b->W,
                        host_out + (size_t)r * b->W);
    }
    return PCAD_OK;
}

pcad_status pcad_bands_info(const pcad_bands *b, int band, int *own_row0, int *own_row1,
                            int *buf_row0, int *buf_row1, uint64_t *t)
{
    if (!b || band < 0 || band >= b->n)
        return set_error(PCAD_EINVAL, "no such band");
    if (own_row0)
        *own_row0 = b->own0[band];
    if (own_row1)
        *own_row1 = b->own1[band];
    if (buf_row0)
        *buf_row0 = b->buf0[band];
    if (buf_row1)
        *buf_row1 = b->buf1[band];
    if (t)
        *t = b->t;
    return PCAD_OK;
}

void pcad_bands_destroy(pcad_bands *b)
{
    if (!b)
        return;
    DeviceGuard guard;
    free_bands(b);
}

}  // extern "C"
