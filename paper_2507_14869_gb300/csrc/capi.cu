// C ABI and chain runtime (see include/pcaden.h for the contract).
//
// A chain owns, in one stream-ordered device allocation: two label planes
// (ping-pong for the synchronous PCA update; Gibbs updates one in place),
// the observation, the FP32 accumulator, the model tables, the device sweep
// counter and the FP64-redraw counter.  Sweeps are issued in blocks of
// kGraphSweeps captured once per chain into a CUDA graph: every kernel reads
// its sweep index as *counter + offset and the block ends with a one-thread
// kernel that advances the counter, so one instantiated graph replays any
// block (the ping-pong parity returns to 0 after an even number of sweeps).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pcaden.h"
#include "pcad_internal.h"

using namespace pcad;

namespace {

thread_local std::string g_err;
constexpr int kGraphSweeps = 32;    // sweeps per captured block (even)
constexpr int kTable = 511;

pcad_status fail(pcad_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(PCAD_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                            \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

pcad_status validate_model(const pcad_model *m)
{
    if (!m)
        return fail(PCAD_EINVAL, "model is NULL");
    if (m->L < 2 || m->L > 256)
        return fail(PCAD_EINVAL, "L=%d outside [2, 256]", m->L);
    if (m->nbhd != 4 && m->nbhd != 8)
        return fail(PCAD_EINVAL, "nbhd=%d must be 4 or 8", m->nbhd);
    if (m->pair != PCAD_PAIR_POTTS && m->pair != PCAD_PAIR_TRUNC_LINEAR)
        return fail(PCAD_EINVAL, "unknown pair potential %d", m->pair);
    if (m->noise != PCAD_NOISE_GAUSS && m->noise != PCAD_NOISE_FLIP &&
        m->noise != PCAD_NOISE_NONE)
        return fail(PCAD_EINVAL, "unknown noise model %d", m->noise);
    if (m->sampler != PCAD_SAMPLER_PCA && m->sampler != PCAD_SAMPLER_GIBBS_CB)
        return fail(PCAD_EINVAL, "unknown sampler %d", m->sampler);
    if (!std::isfinite(m->pair_coef))
        return fail(PCAD_EINVAL, "pair_coef not finite");
    const int T = m->pair == PCAD_PAIR_POTTS ? 1 : m->pair_T;
    if (m->pair == PCAD_PAIR_TRUNC_LINEAR && (m->pair_T < 0 || m->pair_T > 255))
        return fail(PCAD_EINVAL, "pair_T=%d outside [0, 255]", m->pair_T);
    if (std::fabs((double)m->pair_coef) * m->nbhd * T > 40.0)
        return fail(PCAD_EINVAL, "prior range |pair_coef|*nbhd*T = %g exceeds 40",
                    std::fabs((double)m->pair_coef) * m->nbhd * T);
    if (m->noise == PCAD_NOISE_GAUSS) {
        if (!(m->sigma > 0.0f) || !std::isfinite(m->sigma))
            return fail(PCAD_EINVAL, "sigma must be positive and finite");
    } else if (m->noise == PCAD_NOISE_FLIP) {
        if (m->L != 2)
            return fail(PCAD_EINVAL, "flip noise needs L=2");
        if (!(m->flip_p > 0.0f && m->flip_p < 1.0f))
            return fail(PCAD_EINVAL, "flip_p must be in (0, 1)");
        const double p = m->flip_p;
        if (std::fabs(std::log((1.0 - p) / p)) > 40.0)
            return fail(PCAD_EINVAL, "|ln((1-p)/p)| exceeds 40");
    }
    if (!(m->inertia >= 0.0f && m->inertia <= 40.0f))
        return fail(PCAD_EINVAL, "inertia must be in [0, 40]");
    if (m->inertia_norm < 0 || m->inertia_norm > 2)
        return fail(PCAD_EINVAL, "inertia_norm=%d must be 0, 1 or 2", m->inertia_norm);
    return PCAD_OK;
}

// Host copy of the model tables and the FP32 error bound.
struct ModelTables {
    double ta64[kTable];
    std::vector<double> pr64;
    double in64[256];   // Lp inertia price factors (norm 1, 2)
    DevModel dm;  // table pointers filled once uploaded
};

void build_tables(const pcad_model &m, ModelTables &t)
{
    const int T = m.pair == PCAD_PAIR_POTTS ? 1 : m.pair_T;
    const int pmax = m.nbhd * T;
    const double c = (double)m.pair_coef;
    for (int d = -255; d <= 255; ++d) {
        double v;
        if (m.noise == PCAD_NOISE_GAUSS) {
            const double s = (double)m.sigma;
            const double a = 1.0 / (2.0 * s * s);
            v = std::exp(-(a * (double)(d * d)));
        } else if (m.noise == PCAD_NOISE_FLIP) {
            const double p = (double)m.flip_p;
            v = d == 0 ? 1.0 : (std::abs(d) == 1 ? p / (1.0 - p) : 0.0);
        } else {
            v = 1.0;   // no likelihood
        }
        t.ta64[d + 255] = v;
    }
    t.pr64.assign(pmax + 1, 0.0);
    for (int P = 0; P <= pmax; ++P)
        t.pr64[P] = std::exp(-(c * (double)P));
    const double lam = m.sampler == PCAD_SAMPLER_PCA ? (double)m.inertia : 0.0;
    const double log2e = 1.4426950408889634074;
    DevModel &d = t.dm;
    d.L = m.L;
    d.nbhd = m.nbhd;
    d.T = T;
    d.pmax = pmax;
    d.gam = (float)(-c * log2e);
    if (m.noise == PCAD_NOISE_GAUSS) {
        const double s = (double)m.sigma;
        d.alpha = (float)(-log2e / (2.0 * s * s));
    } else if (m.noise == PCAD_NOISE_FLIP) {
        const double p = (double)m.flip_p;
        d.alpha = (float)(-log2e * std::log((1.0 - p) / p));
    } else {
        d.alpha = 0.0f;
    }
    d.Tf = (float)T;
    // Lp prices only for the PCA sampler (Gibbs has no inertia)
    // (for L = 2, (|s - x_i| / 1)^p = 1{s != x_i}: the L0 price exactly)
    const int norm = (lam > 0.0 && m.L > 2) ? m.inertia_norm : 0;
    d.norm = norm;
    d.em1 = norm == 0 ? (float)std::expm1(lam) : 0.0f;
    d.el64 = std::exp(lam);
    d.kappa = norm == 0 ? 0.0f
                        : (float)(-lam * log2e / std::pow((double)(m.L - 1), (double)norm));
    for (int dd = 0; dd < 256; ++dd) {
        const double q = (double)dd / (double)(m.L - 1);
        t.in64[dd] = norm == 0 ? 1.0 : std::exp(-lam * (norm == 1 ? q : q * q));
    }
    // Rigorous bound on |C_k/Z (FP32) - F_k (exact)|.  Exponent v = alpha Q +
    // gam P: |dv| <= u (2|gam P| + |alpha Q| + |v|) from the two rounded
    // coefficients and the two roundings.  The CDF error from the weights is
    // sum_s p_s theta_s, theta_s <= ln2 |dv_s| + e_ex2; with |gam P| <=
    // |gam| pmax, |alpha Q| <= |v| + |gam| pmax and E_p|v| <= |v_max| + log2 L
    // <= |gam| pmax + log2 L (entropy bound), the weight part is at most
    // u ln2 (5 |gam| pmax + 2 log2 L) + e_ex2, doubled for the inertia
    // correction.  Summation: 8 in-chunk additions, Kahan across chunks
    // (2u), the pass-2 prefix (8), 3 combining roundings: 21u.  The ratio
    // doubles both; 1.5x slack.  e_ex2: ex2.approx.ftz within 2 ulp.
    const double u = 5.9604644775390625e-08;
    const double A = std::fabs((double)d.gam) * pmax;
    const double e_w = u * 0.6931471805599453 * (5.0 * A + 2.0 * std::log2((double)m.L)) +
                       4.0 * u;
    const double gsum = 21.0 * u;
    d.eta = (float)(1.5 * 2.0 * (2.0 * e_w + gsum) + 8.0 * u);
    if (norm != 0) {
        // Lp price: v' = alpha Q + gam P + kappa R + c, R = |s - x_i|^p, the
        // per-site shift c = |kappa| |g - x_i|^p in [0, I], I = lambda log2(e)
        // (so v'(g) >= -A and v' <= I: no overflow, no flushed mass), FFMA
        // chain kappa R + c -> + gam P -> + alpha Q.  |dv'| <= u (2|v'| + 3A +
        // 4I) and E_p|v'| <= max(A, I) + log2 L, so the weight part is at most
        // u ln2 (5A + 6I + 2 log2 L) + e_ex2 (7I taken for the rounding of c).
        const double I = lam * 1.4426950408889634074;
        const double e_wn = u * 0.6931471805599453 *
                                (5.0 * A + 7.0 * I + 2.0 * std::log2((double)m.L)) +
                            4.0 * u;
        d.eta = (float)(1.5 * 2.0 * (2.0 * e_wn + gsum) + 8.0 * u);
    }
    // Per-site margin (the tensor-core sweep; the CUDA-core sweeps' weights
    // 2^fl(alpha q + fl(gam P)) with gam <= 0 satisfy the same |dv| <= 3u |v|
    // with cb = 0 and R = P, and take it too).  Tensor-core window labels take
    // v = fl(alpha q + fl(mu Pb + cb)) (q = (g - s)^2 and the tent sum Pb
    // exact integers, mu = -gam), outside labels (Pb = 0) v = fl(alpha q + cb),
    // with cb = -fl(mu nbhd T) for mu > 0 (else 0), the same float for every
    // label: up to one common shift K, v is alpha q - |mu| R with R =
    // nbhd T - Pb (mu > 0) or Pb (mu <= 0), both terms <= 0, so |alpha q| +
    // |mu| R = |v| and the roundings give |dv| <= u (|alpha q| + 2 |mu| R +
    // |v|) <= 3u |v|.  The common shift 2^K scales every weight alike and
    // leaves all ratios unchanged.  Mixture p~ of the L labels and the
    // inertia atom (weight (e^lambda - 1) w_xi, delta = fl(w_xi em1), 2u
    // more): a relative weight error theta_a moves every CDF value by at
    // most sum_a p~_a |theta_a| (not twice: F~ - F = ((1 - F) a - F (b - a))
    // / (1 + b) with a, b - a the errors below and above k), and with
    // log-weights v_a <= 0 (v of the atom: v_xi + J, J = log2(e^lambda - 1))
    // E|v| = H(p~) - log2 Z + rho J <= log2(L + 1) - log2 Z + rho J+ (Z the
    // exact total, rho = delta / Z the atom's mass).  So
    //   E_w <= 3u ln2 (log2(L + 1) - log2 Z + rho J+) + e_ex2 + 2u rho.
    // Summation: chunk sums (7 roundings), Kahan prefix (2u), pass-2 prefix
    // (7), the joins with Gprev and delta (2): C_k within 11u, Z within 10u,
    // their ratio within 21u; t = fl(u Z) one more u.  eta = 1.5 (E_w +
    // 22u), 1.5 the slack for second-order terms, the FP32 evaluation of
    // eta and of the margin comparison, and log2 Z from lg2.approx of the
    // computed Z (within 2^-22 absolute; the computed Z is within 1e-4 of
    // 2^K Z, |K| <= u |mu| nbhd T) with 1/64 added.  Per site:
    //   eta = kb1 (hb - lg2(Z)) + kb0 + kbr delta / Z.
    {
        const double mu_f = -(double)d.gam;
        d.cb = mu_f > 0.0 ? (float)(-mu_f * (double)pmax) : 0.0f;
        const double ln2 = 0.6931471805599453;
        const double J = lam > 0.0 ? std::log2(std::expm1(lam)) : 0.0;
        d.hb = (float)(std::log2((double)m.L + 1.0) + 1.0 / 64.0);
        d.kb1 = (float)(1.5 * 3.0 * u * ln2);
        d.kb0 = (float)(1.5 * (4.0 + 22.0) * u);
        d.kbr = (float)(1.01 * 1.5 * (3.0 * u * ln2 * std::fmax(J, 0.0) + 2.0 * u));
    }
    d.ta64 = nullptr;
    d.pr64 = nullptr;
}

}  // namespace

struct pcad_chain {
    int H = 0, W = 0, pitch = 0;
    pcad_model model{};
    uint64_t seed = 0;
    uint32_t chain_id = 0;
    int burn_in = 0;
    uint64_t t = 0;      // host mirror of the device sweep counter
    uint64_t n_acc = 0;
    int cur = 0;         // PCA: plane holding the current state
    cudaStream_t stream = nullptr;
    void *block = nullptr;   // single device allocation
    uint8_t *x[2] = {nullptr, nullptr};
    uint8_t *g = nullptr;
    float *acc = nullptr;
    float *fplane = nullptr;      // H*W floats for read-back / metrics
    uint8_t *clean = nullptr;     // H*W bytes for metrics input
    uint32_t *tdev = nullptr;
    unsigned long long *fp64 = nullptr;
    double *mscratch = nullptr;   // 8 scratch + 2 results
    double *ta64 = nullptr, *pr64 = nullptr, *in64 = nullptr;
    uint32_t *ptab = nullptr;     // small-L sweep: pair prior table
    uint4 *btab = nullptr;        // two-label draw thresholds (L = 2)
    float *ftab = nullptr;        // outside-chunk sums of the windowed sweeps
    DevModel dm{};
    cudaGraphExec_t graph = nullptr;
    int tb_k = 0;                 // sweeps per temporally blocked launch (0: one per launch)
    int kernel = PCAD_KERNEL_AUTO;  // kernel of unblocked PCA sweeps
    bool maps_ready = false;
    CUtensorMap xmap[2];          // TMA descriptors of the two label planes
    CUtensorMap gmap;             // and of the observation
    int *err = nullptr;           // bounded-wait timeout flag (device)
    long long wait_ns = 0;        // limit of each bounded device wait (0: the default, 1 s)
    int row_off = 0;              // global row of local row 0 (a band of a larger image)
    int stall_tile = 0;           // test aid: wavefront tile stall_tile - 1 never publishes
    unsigned long long *esums = nullptr;   // energy reduction sums (device, 2 x u64)
    EnergyCoef ecoef{};
    EnergyTrack track{};          // minimum-energy tracking (trace == nullptr: off)
    unsigned int *wave = nullptr; // wavefront kernel: per-tile counters + work counter
    int wave_tiles = 0;
    int sms = 0;                  // multiprocessors of the chain's device
    void *track_block = nullptr;
};

namespace {

SweepArgs make_args(const pcad_chain *ch)
{
    SweepArgs a{};
    a.g = ch->g;
    a.acc = ch->acc;
    a.fp64_draws = ch->fp64;
    a.sweep_base = ch->tdev;
    a.seed = ch->seed;
    a.H = ch->H;
    a.W = ch->W;
    a.pitch = ch->pitch;
    a.chain = ch->chain_id;
    a.burn_in = ch->burn_in;
    a.wait_ns = ch->wait_ns;
    a.stall_tile = ch->stall_tile;
    a.row_off = ch->row_off;
    a.m = ch->dm;
    return a;
}

// The windowed sweeps AUTO takes (0: none, 1: one launch per sweep or
// Gibbs colour phase, 2: the wavefront), for the models the windowed sweeps
// accept with L >= 32, either neighbourhood, without energy tracking, by
// image size in blocks of 4 x 32 sites per multiprocessor: per-sweep (per-phase) launches from 100 blocks
// per SM, the wavefront from 8; 8-neighbourhood Gibbs the wavefront from 3.
// Measured on GB300 at L = 256, lazy PCA (site-updates/s; per-sweep /
// wavefront / tensor-core):
// 8192^2 1.63e10 / - / 1.07e10; 2048^2 1.70e10 / 1.63e10 / 1.14e10; 1024^2
// 1.51e10 / 1.58e10 / 1.11e10; 768^2 1.38e10 / 1.54e10 / 1.10e10; 512^2
// 1.11e10 / 1.45e10 / 1.08e10; 256^2 0.54e10 / 0.59e10 / 0.63e10.  At 2048^2
// and L = 64, 96 (T = 8), 128, 160 the per-sweep windowed sweep ran 2.67e10,
// 3.08e10, 2.24e10, 1.96e10 against 2.25e10, 1.49e10, 1.43e10, 0.80e10 for
// the per-sweep CUDA-core kernel; at 2048^2 (512^2: the wavefronts) L = 33
// Potts 3.09e10 (2.57e10) against 2.19e10 (1.85e10) with 8 neighbours, L = 48
// 3.22e10 (2.78e10) against 2.19e10 (1.87e10), L = 63 2.35e10 (2.10e10)
// against 2.16e10 (1.83e10), but L = 24 3.65e10 against 3.96e10: AUTO takes
// the windowed sweeps from L = 32.  Gibbs, 4 neighbours (per-phase /
// wavefront / tensor-core phases): 2048^2 1.68e10 / 1.61e10 / 1.11e10,
// 1024^2 1.39e10 / 1.55e10 / 1.09e10, 512^2 0.89e10 / 1.04e10 / 1.01e10,
// 256^2 0.32e10 / 0.33e10 / 0.34e10; 8 neighbours (per-phase / wavefront /
// CUDA-core phases): 2048^2 1.47e10 / 1.56e10 / 0.64e10, 256^2 0.17e10 /
// 0.19e10 / 0.15e10.
int win_auto_mode(const pcad_chain *ch)
{
    if (ch->tb_k > 0 || ch->track.trace || ch->kernel != PCAD_KERNEL_AUTO || ch->sms <= 0)
        return 0;
    if (!pca_win_eligible(ch->dm) || ch->model.L < kWinAutoMinLabels)
        return 0;
    // launch grids: (W / 32) x (H / 4) blocks (Gibbs: H / 8 for 8
    // neighbours); the second dimension is at most 65535
    if ((ch->H + 3) / 4 > 65535)
        return 0;
    const long long blocks = (long long)((ch->W + 31) / 32) * ((ch->H + 3) / 4);
    if (ch->model.sampler != PCAD_SAMPLER_PCA && ch->model.nbhd == 8)
        return blocks >= 3LL * ch->sms ? 2 : 0;   // no tensor-core Gibbs form to compare
    if (blocks >= 100LL * ch->sms)
        return 1;
    return blocks >= 8LL * ch->sms ? 2 : 0;
}

bool win_auto(const pcad_chain *ch)
{
    return win_auto_mode(ch) == 1;
}

// Unblocked PCA sweeps, and 4-neighbourhood checkerboard Gibbs sweeps, on the
// tensor-core kernel: on request, or with AUTO for the models pca_tc_auto
// accepts when every sweep's state is not needed (energy tracking would force
// one launch per sweep).
bool uses_tc(const pcad_chain *ch)
{
    if (!pca_tc_eligible(ch->dm))
        return false;
    if (ch->model.sampler == PCAD_SAMPLER_PCA ? ch->tb_k > 0 : ch->model.nbhd != 4)
        return false;
    if (ch->kernel == PCAD_KERNEL_TENSOR)
        return true;
    return ch->kernel == PCAD_KERNEL_AUTO && pca_tc_auto(ch->dm) && !ch->track.trace &&
           win_auto_mode(ch) == 0;
}

// Whole runs of sweeps of small two-label images in one single-CTA launch
// (state in shared memory): on request, or with AUTO for every image it
// accepts, without energy tracking or temporal blocking.
bool uses_resident(const pcad_chain *ch)
{
    if (ch->tb_k > 0 || ch->track.trace || !resident_eligible(ch->dm, ch->H, ch->W))
        return false;
    return ch->kernel == PCAD_KERNEL_RESIDENT || ch->kernel == PCAD_KERNEL_AUTO;
}

bool uses_wave(const pcad_chain *ch);

// Unblocked sweeps (PCA or Gibbs) on the CUDA-core windowed kernels: on
// request, or with AUTO where win_auto takes them.
bool uses_win(const pcad_chain *ch)
{
    if (win_auto(ch))
        return true;
    return ch->tb_k == 0 &&
           (ch->kernel == PCAD_KERNEL_WINDOW || ch->kernel == PCAD_KERNEL_WINDOW_WAVE) &&
           pca_win_eligible(ch->dm);
}

// Sweeps of the windowed kernels as one wavefront launch per block of sweeps
// (lazy PCA, or Gibbs colour phases): on request, without energy tracking (which needs every sweep's
// state: then one windowed launch per sweep), or with AUTO where
// win_auto_mode takes it.
bool uses_winw(const pcad_chain *ch)
{
    if (win_auto_mode(ch) == 2)
        return true;
    return ch->tb_k == 0 && !ch->track.trace && ch->kernel == PCAD_KERNEL_WINDOW_WAVE &&
           pca_win_eligible(ch->dm);
}

// TMA descriptors of the two label planes and the observation (once).
bool ensure_maps(pcad_chain *ch)
{
    if (!ch->maps_ready)
        ch->maps_ready = encode_plane_map(&ch->xmap[0], ch->x[0], ch->H, ch->W, ch->pitch) &&
                         encode_plane_map(&ch->xmap[1], ch->x[1], ch->H, ch->W, ch->pitch) &&
                         encode_plane_map(&ch->gmap, ch->g, ch->H, ch->W, ch->pitch);
    return ch->maps_ready;
}

// Unblocked PCA sweeps on the small-label kernel: on request, or with AUTO
// for the models it accepts (3 <= L <= 16, c >= 0, L0 price) unless the
// wavefront kernel is chosen (L = 16 at 1/2 to 3 waves of 4 x 32 tiles,
// where the small-label kernel's 16 x 32 tiles leave SMs idle).  Measured on
// GB300 at L = 16: 1.05e11 site-updates/s at 8192^2 (TMA tiles) and 6.9e10
// at 1024^2 against 4.9e10 and 4.1e10 for the general per-sweep kernel;
// 3.2e10 at 512^2 against 3.7e10 for the wavefront kernel.
bool uses_small(const pcad_chain *ch)
{
    if (ch->model.sampler != PCAD_SAMPLER_PCA || ch->tb_k > 0 || !pca_small_eligible(ch->dm))
        return false;
    return ch->kernel == PCAD_KERNEL_SMALL || (ch->kernel == PCAD_KERNEL_AUTO && !uses_wave(ch));
}

// The small-label kernel's launch form for large images: persistent blocks
// over TMA-loaded 64 x 46 tiles, the next tile's box in flight during the
// draw (launch_pca_small_tma), from kSmallTmaMinSites sites.  Measured on
// GB300 at L = 16 (site-updates/s, TMA tiles / persistent 16 x 32 tiles):
// 8192^2 1.049e11 / 0.954e11, 4096^2 1.015e11 / 0.953e11, 3072^2
// 0.997e11 / 0.959e11, 2048^2 0.931e11 / 0.926e11, 1024^2 0.588e11 /
// 0.691e11; 8 neighbours at 4096^2: L = 5 10.9e10 / 10.4e10, L = 16
// 9.5e10 / 9.1e10.
bool small_tma(const pcad_chain *ch)
{
    return ch->maps_ready && (long long)ch->H * ch->W >= kSmallTmaMinSites && uses_small(ch);
}

// Unblocked two-label PCA sweeps, one launch per sweep with the threshold
// table of the resident kernel (a table read and a compare per site): on
// request, or with AUTO for images of kBinaryAutoMinSites sites and more
// (smaller images run whole runs on the resident kernel, or the per-sweep
// CUDA-core kernel).
bool uses_binary(const pcad_chain *ch)
{
    if (ch->model.sampler != PCAD_SAMPLER_PCA || ch->tb_k > 0 || !binary_eligible(ch->dm))
        return false;
    if (ch->kernel == PCAD_KERNEL_BINARY)
        return true;
    return ch->kernel == PCAD_KERNEL_AUTO && !uses_resident(ch) &&
           (long long)ch->H * ch->W >= kBinaryAutoMinSites;
}

// Unblocked PCA sweeps as wavefront launches (L0 price, no per-sweep energy).
// AUTO takes them where the measured GB300 sweep favoured them: L >= 16 and
// between 1/2 and 3 waves of the per-sweep kernel (10 resident 4 x 32 tiles
// per SM): there the per-sweep tail wave costs up to 25 %; with fewer tiles
// or cheaper labels the wavefront's single work counter limits it.
bool uses_wave(const pcad_chain *ch)
{
    if (ch->model.sampler != PCAD_SAMPLER_PCA || ch->dm.norm != 0 || ch->tb_k > 0 ||
        ch->track.trace)
        return false;
    if (ch->kernel == PCAD_KERNEL_WAVE)
        return true;
    if (ch->kernel != PCAD_KERNEL_AUTO || ch->model.L < 16 || ch->sms <= 0 ||
        win_auto_mode(ch) != 0)
        return false;
    const long slots = 10L * ch->sms;
    return 2L * ch->wave_tiles >= slots && ch->wave_tiles <= 3L * slots;
}

// Issue sweeps [*counter + off0, *counter + off0 + n) without advancing the counter.
pcad_status issue_sweeps(pcad_chain *ch, int off0, int n, int &cur, cudaStream_t st)
{
    SweepArgs a = make_args(ch);
    if (uses_resident(ch) && n > 0) {
        // all n sweeps in one single-CTA launch; PCA ends in the other plane
        // when n is odd, Gibbs in place
        a.sweep_off = (uint32_t)off0;
        const bool gibbs = ch->model.sampler != PCAD_SAMPLER_PCA;
        const int out = gibbs ? cur : cur ^ (n & 1);
        CUDA_TRY(launch_resident(a, ch->x[cur], ch->x[out], n, gibbs, st));
        cur = out;
        return PCAD_OK;
    }
    if (uses_tc(ch) && n > 0) {
        // tensor-core wavefront: all n sweeps in one launch, or one launch
        // per sweep when every sweep's state is needed (energy tracking)
        const int per = ch->track.trace ? 1 : n;
        for (int k = 0; k < n; k += per) {
            a.sweep_off = (uint32_t)(off0 + k);
            CUDA_TRY(cudaMemsetAsync(ch->wave, 0,
                                     (size_t)(ch->wave_tiles + 1) * sizeof(unsigned int), st));
            if (ch->model.sampler == PCAD_SAMPLER_PCA) {
                CUDA_TRY(launch_pca_tc(a, ch->x[cur], ch->x[cur ^ 1], per, ch->wave,
                                       ch->wave + ch->wave_tiles, ch->err, st));
                if (per & 1)
                    cur ^= 1;
            } else {   // checkerboard Gibbs, in place
                CUDA_TRY(launch_gibbs_tc(a, ch->x[cur], per, ch->wave, ch->wave + ch->wave_tiles,
                                         ch->err, st));
            }
            if (ch->track.trace)
                CUDA_TRY(launch_energy(ch->x[cur], ch->g, ch->H, ch->W, ch->pitch, ch->ecoef,
                                       ch->esums, nullptr, ch->track, ch->tdev, a.sweep_off, st));
        }
        return PCAD_OK;
    }
    if (uses_winw(ch) && n > 0) {
        a.sweep_off = (uint32_t)off0;
        CUDA_TRY(cudaMemsetAsync(ch->wave, 0, (size_t)(ch->wave_tiles + 1) * sizeof(unsigned int),
                                 st));
        if (ch->model.sampler == PCAD_SAMPLER_PCA) {
            CUDA_TRY(launch_pca_winw(a, ch->ftab, ch->x[cur], ch->x[cur ^ 1], n, ch->wave,
                                     ch->wave + ch->wave_tiles, ch->err, st));
            if (n & 1)
                cur ^= 1;
        } else {   // colour phases in place
            CUDA_TRY(launch_gibbs_winw(a, ch->ftab, ch->x[cur], n, ch->wave,
                                       ch->wave + ch->wave_tiles, ch->err, st));
        }
        return PCAD_OK;
    }
    if (uses_wave(ch) && n > 0) {
        // one persistent launch for all n sweeps: counters zeroed first
        a.sweep_off = (uint32_t)off0;
        CUDA_TRY(cudaMemsetAsync(ch->wave, 0, (size_t)(ch->wave_tiles + 1) * sizeof(unsigned int),
                                 st));
        CUDA_TRY(launch_pca_wave(a, ch->x[cur], ch->x[cur ^ 1], n, ch->wave,
                                 ch->wave + ch->wave_tiles, ch->err, st));
        if (n & 1)
            cur ^= 1;
        return PCAD_OK;
    }
    const int ncol = ch->model.nbhd == 4 ? 2 : 4;
    int done = 0;
    if (ch->model.sampler == PCAD_SAMPLER_PCA && ch->tb_k > 0) {
        // temporally blocked: tb_k sweeps per launch, always into the other plane
        for (; done + ch->tb_k <= n; done += ch->tb_k) {
            a.sweep_off = (uint32_t)(off0 + done);
            a.xin = ch->x[cur];
            a.xout = ch->x[cur ^ 1];
            CUDA_TRY(launch_pca_tb(ch->xmap[cur], ch->gmap, a, ch->tb_k, ch->err, st));
            cur ^= 1;
        }
    }
    for (int k = done; k < n; ++k) {
        a.sweep_off = (uint32_t)(off0 + k);
        if (ch->model.sampler == PCAD_SAMPLER_PCA) {
            a.xin = ch->x[cur];
            a.xout = ch->x[cur ^ 1];
            if (small_tma(ch))
                CUDA_TRY(launch_pca_small_tma(ch->xmap[cur], ch->gmap, a, ch->err, st));
            else if (uses_small(ch))
                // chains check g < L at creation: the data term from a table
                CUDA_TRY(launch_pca_small(a, st, nullptr, nullptr, nullptr, true));
            else if (uses_binary(ch))
                CUDA_TRY(launch_pca_binary(a, st));
            else if (uses_win(ch))
                CUDA_TRY(launch_pca_win(a, ch->ftab, st));
            else
                CUDA_TRY(launch_pca_sweep(a, st));
            cur ^= 1;
            if (ch->track.trace)
                CUDA_TRY(launch_energy(ch->x[cur], ch->g, ch->H, ch->W, ch->pitch, ch->ecoef,
                                       ch->esums, nullptr, ch->track, ch->tdev, a.sweep_off, st));
        } else {
            a.xin = ch->x[cur];
            a.xout = nullptr;
            const bool win = uses_win(ch);
            for (int q = 0; q < ncol; ++q) {
                a.last_phase = q == ncol - 1;
                if (win)
                    CUDA_TRY(launch_gibbs_win(a, q, ch->ftab, st));
                else
                    CUDA_TRY(launch_gibbs_phase(a, q, st));
            }
            if (ch->track.trace)
                CUDA_TRY(launch_energy(ch->x[cur], ch->g, ch->H, ch->W, ch->pitch, ch->ecoef,
                                       ch->esums, nullptr, ch->track, ch->tdev, a.sweep_off, st));
        }
    }
    return PCAD_OK;
}

pcad_status build_graph(pcad_chain *ch)
{
    cudaStream_t cap;
    CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    pcad_status st = PCAD_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int cur = 0;
        st = issue_sweeps(ch, 0, kGraphSweeps, cur, cap);
        cudaError_t e2 = launch_advance(ch->tdev, kGraphSweeps, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (st == PCAD_OK && e2 != cudaSuccess)
            st = fail(PCAD_ECUDA, "advance launch: %s", cudaGetErrorString(e2));
    }
    if (st == PCAD_OK && e != cudaSuccess)
        st = fail(PCAD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    if (st == PCAD_OK) {
        e = cudaGraphInstantiate(&ch->graph, graph, 0);
        if (e != cudaSuccess)
            st = fail(PCAD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    if (graph)
        cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    return st;
}

pcad_status create_common(const uint8_t *g_src, bool g_on_device, int H, int W, int g_pitch,
                          const pcad_model *m, uint64_t seed, uint32_t chain_id, int burn_in,
                          void *cuda_stream, pcad_chain **out)
{
    if (!out)
        return fail(PCAD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g_src)
        return fail(PCAD_EINVAL, "g is NULL");
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || (long long)H * W > (1LL << 31))
        return fail(PCAD_EINVAL, "image size %dx%d outside the limits", H, W);
    if (g_pitch < W)
        return fail(PCAD_EINVAL, "g_pitch %d < W %d", g_pitch, W);
    if (burn_in < 0)
        return fail(PCAD_EINVAL, "burn_in < 0");
    if (chain_id >= (1u << 24))
        return fail(PCAD_EINVAL, "chain id must be < 2^24");
    pcad_status st = validate_model(m);
    if (st != PCAD_OK)
        return st;

    ModelTables tabs;
    build_tables(*m, tabs);

    pcad_chain *ch = new pcad_chain();
    ch->H = H;
    ch->W = W;
    ch->pitch = (int)align_up((size_t)W, 16);
    ch->model = *m;
    ch->seed = seed;
    ch->chain_id = chain_id;
    ch->burn_in = burn_in;
    ch->stream = (cudaStream_t)cuda_stream;

    const size_t plane = align_up((size_t)ch->pitch * H, 256);
    const size_t fbytes = align_up((size_t)H * W * sizeof(float), 256);
    const size_t cbytes = align_up((size_t)H * W, 256);
    const size_t tbytes = align_up(kTable * sizeof(double), 256) +
                          align_up(tabs.pr64.size() * sizeof(double), 256) +
                          sizeof(tabs.in64);
    const size_t misc = 256;
    const int ntiles = wave_tiles(H, W);
    const size_t wbytes = align_up((size_t)(ntiles + 1) * sizeof(unsigned int), 256);
    const size_t pbytes = align_up((size_t)ptab_words() * sizeof(uint32_t), 256);
    const size_t bbytes = align_up((size_t)btab_bytes(), 256);
    const size_t obytes = align_up((size_t)tc_table_floats(m->L) * sizeof(float), 256);
    const size_t total =
        3 * plane + 2 * fbytes + cbytes + tbytes + wbytes + pbytes + bbytes + obytes + misc;
    cudaError_t e = cudaMallocAsync(&ch->block, total, ch->stream);
    if (e != cudaSuccess) {
        delete ch;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PCAD_ENOMEM : PCAD_ECUDA,
                    "device allocation of %zu bytes: %s", total, cudaGetErrorString(e));
    }
    char *p = (char *)ch->block;
    ch->x[0] = (uint8_t *)p; p += plane;
    ch->x[1] = (uint8_t *)p; p += plane;
    ch->g = (uint8_t *)p; p += plane;
    ch->acc = (float *)p; p += fbytes;
    ch->fplane = (float *)p; p += fbytes;
    ch->clean = (uint8_t *)p; p += cbytes;
    ch->ta64 = (double *)p; p += align_up(kTable * sizeof(double), 256);
    ch->pr64 = (double *)p; p += align_up(tabs.pr64.size() * sizeof(double), 256);
    ch->in64 = (double *)p; p += sizeof(tabs.in64);
    ch->wave = (unsigned int *)p; p += wbytes;
    ch->ptab = (uint32_t *)p; p += pbytes;
    ch->btab = (uint4 *)p; p += bbytes;
    ch->ftab = (float *)p; p += obytes;
    ch->wave_tiles = ntiles;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&ch->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    ch->tdev = (uint32_t *)p;
    ch->fp64 = (unsigned long long *)(p + 8);
    ch->mscratch = (double *)(p + 16);
    ch->esums = (unsigned long long *)(p + 96);
    ch->err = (int *)(p + 128);
    ch->ecoef = energy_coef(*m, (long)H * W);

    auto cleanup = [&](pcad_status s) {
        cudaFreeAsync(ch->block, ch->stream);
        cudaStreamSynchronize(ch->stream);
        delete ch;
        return s;
    };
    const cudaMemcpyKind gk = g_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpy2DAsync(ch->g, ch->pitch, g_src, g_pitch, W, H, gk, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(ch->x[0], ch->pitch, ch->g, ch->pitch, W, H,
                              cudaMemcpyDeviceToDevice, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ch->acc, 0, fbytes, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ch->ta64, tabs.ta64, sizeof(tabs.ta64), cudaMemcpyHostToDevice,
                            ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ch->in64, tabs.in64, sizeof(tabs.in64), cudaMemcpyHostToDevice,
                            ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ch->pr64, tabs.pr64.data(), tabs.pr64.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ch->tdev, 0, misc, ch->stream);
    if (e == cudaSuccess && m->L <= kSmallMaxLabels)
        e = launch_ptab(tabs.dm.T, ch->ptab, ch->stream);
    if (e == cudaSuccess && (pca_tc_eligible(tabs.dm) || pca_win_eligible(tabs.dm)))
        e = launch_tc_table(tabs.dm, ch->ftab, ch->stream);
    if (e == cudaSuccess && m->L == 2) {
        DevModel dm = tabs.dm;
        dm.ta64 = ch->ta64;
        dm.pr64 = ch->pr64;
        dm.in64 = ch->in64;
        e = launch_btab(dm, ch->btab, ch->stream);
    }
    if (e == cudaSuccess) {
        int *bad = (int *)(ch->mscratch);
        e = launch_check_labels(ch->g, ch->pitch, H, W, m->L, bad, ch->stream);
        int hbad = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ch->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(ch->stream);
        if (e == cudaSuccess && hbad != 0)
            return cleanup(fail(PCAD_EINVAL, "%d observed labels are >= L=%d", hbad, m->L));
    }
    if (e != cudaSuccess)
        return cleanup(fail(PCAD_ECUDA, "chain set-up: %s", cudaGetErrorString(e)));
    ch->dm = tabs.dm;
    ch->dm.ta64 = ch->ta64;
    ch->dm.pr64 = ch->pr64;
    ch->dm.in64 = ch->in64;
    ch->dm.ptab = m->L <= kSmallMaxLabels ? ch->ptab : nullptr;
    ch->dm.btab = m->L == 2 ? ch->btab : nullptr;
    // TMA descriptors of the planes for the small-label kernel's tile form
    // (large images; temporal blocking encodes them on demand otherwise)
    if (m->L <= kSmallMaxLabels && (long long)H * W >= kSmallTmaMinSites)
        ensure_maps(ch);
    *out = ch;
    return PCAD_OK;
}

bool acc_would_overflow(const pcad_chain *ch, uint64_t n)
{
    const uint64_t t1 = ch->t + n;
    const uint64_t start = ch->t > (uint64_t)ch->burn_in ? ch->t : (uint64_t)ch->burn_in;
    const uint64_t add = t1 > start ? t1 - start : 0;
    return (uint64_t)(ch->model.L - 1) * (ch->n_acc + add) >= (1ull << 24);
}

}  // namespace

extern "C" {

pcad_status pcad_chain_create(const uint8_t *g_host, int H, int W, int g_pitch,
                              const pcad_model *m, uint64_t seed, uint32_t chain_id,
                              int burn_in, void *cuda_stream, pcad_chain **out)
{
    return create_common(g_host, false, H, W, g_pitch, m, seed, chain_id, burn_in, cuda_stream,
                         out);
}

pcad_status pcad_chain_create_dev(const uint8_t *g_dev, int H, int W, int g_pitch,
                                  const pcad_model *m, uint64_t seed, uint32_t chain_id,
                                  int burn_in, void *cuda_stream, pcad_chain **out)
{
    return create_common(g_dev, true, H, W, g_pitch, m, seed, chain_id, burn_in, cuda_stream,
                         out);
}

pcad_status pcad_chain_run(pcad_chain *ch, int nsweeps)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (nsweeps < 0)
        return fail(PCAD_EINVAL, "nsweeps < 0");
    if (nsweeps == 0)
        return PCAD_OK;
    if (ch->t + (uint64_t)nsweeps > 0xFFFFFFFFull)
        return fail(PCAD_EINVAL, "sweep counter would exceed 2^32");
    if (acc_would_overflow(ch, (uint64_t)nsweeps))
        return fail(PCAD_EINVAL, "accumulator would leave the exact FP32 range");
    int left = nsweeps;
    // Whole captured blocks need the ping-pong parity at 0 (always true for
    // Gibbs); the resident kernel runs any number of sweeps in one launch.
    const bool parity_ok = ch->model.sampler != PCAD_SAMPLER_PCA || ch->cur == 0;
    if (left >= kGraphSweeps && parity_ok && !uses_resident(ch)) {
        if (!ch->graph) {
            pcad_status st = build_graph(ch);
            if (st != PCAD_OK)
                return st;
        }
        while (left >= kGraphSweeps) {
            CUDA_TRY(cudaGraphLaunch(ch->graph, ch->stream));
            left -= kGraphSweeps;
        }
    }
    if (left > 0) {
        int cur = ch->cur;
        pcad_status st = issue_sweeps(ch, 0, left, cur, ch->stream);
        if (st != PCAD_OK)
            return st;
        CUDA_TRY(launch_advance(ch->tdev, (uint32_t)left, ch->stream));
        ch->cur = cur;
    }
    const uint64_t start = ch->t > (uint64_t)ch->burn_in ? ch->t : (uint64_t)ch->burn_in;
    const uint64_t t1 = ch->t + (uint64_t)nsweeps;
    ch->n_acc += t1 > start ? t1 - start : 0;
    ch->t = t1;
    return PCAD_OK;
}

namespace {

// Empty the energy trace and forget the minimum (asynchronous).
pcad_status reset_track(pcad_chain *ch)
{
    const double inf = HUGE_VAL;
    CUDA_TRY(cudaMemsetAsync(ch->track.n, 0, sizeof(unsigned int), ch->stream));
    CUDA_TRY(cudaMemsetAsync(ch->track.flag, 0, sizeof(int), ch->stream));
    CUDA_TRY(cudaMemsetAsync(ch->track.best_sweep, 0, sizeof(unsigned long long), ch->stream));
    CUDA_TRY(cudaMemcpyAsync(ch->track.best, &inf, sizeof(double), cudaMemcpyHostToDevice,
                             ch->stream));
    return cudaStreamSynchronize(ch->stream) == cudaSuccess
               ? PCAD_OK
               : fail(PCAD_ECUDA, "energy tracking reset failed");
}

}  // namespace

pcad_status pcad_chain_reset(pcad_chain *ch)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    const size_t n = (size_t)ch->H * ch->W;
    CUDA_TRY(cudaMemcpy2DAsync(ch->x[0], ch->pitch, ch->g, ch->pitch, ch->W, ch->H,
                               cudaMemcpyDeviceToDevice, ch->stream));
    CUDA_TRY(cudaMemsetAsync(ch->acc, 0, n * sizeof(float), ch->stream));
    CUDA_TRY(cudaMemsetAsync(ch->tdev, 0, 16, ch->stream));
    CUDA_TRY(cudaMemsetAsync(ch->err, 0, sizeof(int), ch->stream));
    ch->cur = 0;
    ch->t = 0;
    ch->n_acc = 0;
    if (ch->track.trace)
        return reset_track(ch);
    return PCAD_OK;
}

pcad_status pcad_chain_sync(pcad_chain *ch)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    if (ch->tb_k > 0 || uses_tc(ch) || uses_wave(ch) || uses_winw(ch) || small_tma(ch)) {
        int e = 0;
        CUDA_TRY(cudaMemcpy(&e, ch->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e == 2)
            return fail(PCAD_ECUDA, "tensor-core sweep: shared memory not 1024-byte aligned");
        if (e)
            return fail(PCAD_ETIMEOUT, "a bounded wait of the sweep kernel (tile load, MMA "
                                       "completion or wavefront dependency) gave up");
    }
    return PCAD_OK;
}

namespace {

// set_model may change coefficients only: the state layout, the tables' sizes
// and the kernels chosen stay as they are.
bool same_structure(const pcad_model &a, const pcad_model &b)
{
    const int Ta = a.pair == PCAD_PAIR_POTTS ? 1 : a.pair_T;
    const int Tb = b.pair == PCAD_PAIR_POTTS ? 1 : b.pair_T;
    return a.L == b.L && a.nbhd == b.nbhd && a.pair == b.pair && Ta == Tb &&
           a.noise == b.noise && a.sampler == b.sampler && a.inertia_norm == b.inertia_norm;
}

}  // namespace

pcad_status pcad_chain_set_model(pcad_chain *ch, const pcad_model *m)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    pcad_status st = validate_model(m);
    if (st != PCAD_OK)
        return st;
    if (!same_structure(*m, ch->model))
        return fail(PCAD_EINVAL, "set_model changes coefficients only (L, nbhd, pair, pair_T, "
                                 "noise, sampler and inertia_norm stay)");
    ModelTables tabs;
    build_tables(*m, tabs);
    // stream-ordered: sweeps queued before use the old tables
    CUDA_TRY(cudaMemcpyAsync(ch->ta64, tabs.ta64, sizeof(tabs.ta64), cudaMemcpyHostToDevice,
                             ch->stream));
    CUDA_TRY(cudaMemcpyAsync(ch->pr64, tabs.pr64.data(), tabs.pr64.size() * sizeof(double),
                             cudaMemcpyHostToDevice, ch->stream));
    CUDA_TRY(cudaMemcpyAsync(ch->in64, tabs.in64, sizeof(tabs.in64), cudaMemcpyHostToDevice,
                             ch->stream));
    if (ch->graph) {   // captured sweeps hold the old coefficients
        CUDA_TRY(cudaStreamSynchronize(ch->stream));
        cudaGraphExecDestroy(ch->graph);
        ch->graph = nullptr;
    }
    ch->model = *m;
    ch->dm = tabs.dm;
    ch->dm.ta64 = ch->ta64;
    ch->dm.pr64 = ch->pr64;
    ch->dm.in64 = ch->in64;
    ch->dm.ptab = m->L <= kSmallMaxLabels ? ch->ptab : nullptr;   // T is unchanged
    ch->dm.btab = m->L == 2 ? ch->btab : nullptr;
    if (m->L == 2)   // stream-ordered after the new FP64 tables
        CUDA_TRY(launch_btab(ch->dm, ch->btab, ch->stream));
    if (pca_tc_eligible(ch->dm) || pca_win_eligible(ch->dm))
        CUDA_TRY(launch_tc_table(ch->dm, ch->ftab, ch->stream));
    ch->ecoef = energy_coef(*m, (long)ch->H * ch->W);
    return PCAD_OK;
}

pcad_status pcad_chain_run_schedule(pcad_chain *ch, const pcad_model *models, const int *sweeps,
                                    int nstages)
{
    if (!ch || nstages < 0 || (nstages > 0 && (!models || !sweeps)))
        return fail(PCAD_EINVAL, "bad schedule");
    for (int k = 0; k < nstages; ++k)
        if (sweeps[k] < 0)
            return fail(PCAD_EINVAL, "stage %d has a negative sweep count", k);
    for (int k = 0; k < nstages; ++k) {
        pcad_status st = pcad_chain_set_model(ch, &models[k]);
        if (st == PCAD_OK)
            st = pcad_chain_run(ch, sweeps[k]);
        if (st != PCAD_OK)
            return st;
    }
    return PCAD_OK;
}

pcad_status pcad_chain_kernel_in_use(const pcad_chain *ch, int *kind)
{
    if (!ch || !kind)
        return fail(PCAD_EINVAL, "chain or kind is NULL");
    if (uses_resident(ch))
        *kind = PCAD_KERNEL_RESIDENT;
    else if (ch->model.sampler != PCAD_SAMPLER_PCA)
        *kind = uses_tc(ch) ? PCAD_KERNEL_TENSOR
                : uses_winw(ch) ? PCAD_KERNEL_WINDOW_WAVE
                : uses_win(ch) ? PCAD_KERNEL_WINDOW : PCAD_KERNEL_CUDA_CORE;
    else if (ch->tb_k > 0)
        *kind = -ch->tb_k;
    else if (uses_tc(ch))
        *kind = PCAD_KERNEL_TENSOR;
    else if (uses_winw(ch))
        *kind = PCAD_KERNEL_WINDOW_WAVE;
    else if (uses_wave(ch))
        *kind = PCAD_KERNEL_WAVE;
    else if (uses_small(ch))
        *kind = PCAD_KERNEL_SMALL;
    else if (uses_binary(ch))
        *kind = PCAD_KERNEL_BINARY;
    else if (uses_win(ch))
        *kind = PCAD_KERNEL_WINDOW;
    else
        *kind = PCAD_KERNEL_CUDA_CORE;
    return PCAD_OK;
}

pcad_status pcad_chain_energy(pcad_chain *ch, double *energy, uint64_t *pair_sum,
                              uint64_t *data_sum)
{
    if (!ch || !energy)
        return fail(PCAD_EINVAL, "chain or energy is NULL");
    double res[3] = {0.0, 0.0, 0.0};
    CUDA_TRY(launch_energy(ch->x[ch->cur], ch->g, ch->H, ch->W, ch->pitch, ch->ecoef, ch->esums,
                           ch->mscratch, EnergyTrack{}, ch->tdev, 0, ch->stream));
    CUDA_TRY(cudaMemcpyAsync(res, ch->mscratch, sizeof(res), cudaMemcpyDeviceToHost,
                             ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    *energy = res[0];
    if (pair_sum)
        *pair_sum = (uint64_t)res[1];
    if (data_sum)
        *data_sum = (uint64_t)res[2];
    return PCAD_OK;
}

pcad_status pcad_chain_track_energy(pcad_chain *ch, int capacity)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (capacity < 0)
        return fail(PCAD_EINVAL, "capacity must be >= 0");
    if (capacity > 0 && ch->tb_k > 0)
        return fail(PCAD_ESTATE, "energy tracking needs every sweep's state: no temporal blocking");
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    if (ch->graph) {
        cudaGraphExecDestroy(ch->graph);
        ch->graph = nullptr;
    }
    if (ch->track_block) {
        CUDA_TRY(cudaFreeAsync(ch->track_block, ch->stream));
        ch->track_block = nullptr;
    }
    ch->track = EnergyTrack{};
    if (capacity == 0)
        return PCAD_OK;
    const size_t head = 64;   // best, best_sweep, n, flag
    const size_t trace = align_up((size_t)capacity * sizeof(double), 256);
    const size_t plane = (size_t)ch->pitch * ch->H;
    void *blk = nullptr;
    cudaError_t e = cudaMallocAsync(&blk, head + trace + plane, ch->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PCAD_ENOMEM : PCAD_ECUDA,
                    "energy tracking allocation: %s", cudaGetErrorString(e));
    }
    char *p = (char *)blk;
    ch->track_block = blk;
    ch->track.best = (double *)p;
    ch->track.best_sweep = (unsigned long long *)(p + 8);
    ch->track.n = (unsigned int *)(p + 16);
    ch->track.flag = (int *)(p + 20);
    ch->track.trace = (double *)(p + head);
    ch->track.cap = capacity;
    ch->track.xb = (uint8_t *)(p + head + trace);
    return reset_track(ch);
}

pcad_status pcad_chain_read_energies(pcad_chain *ch, double *host, int max, int *n)
{
    if (!ch || !n || (max > 0 && !host))
        return fail(PCAD_EINVAL, "chain, host or n is NULL");
    if (!ch->track.trace) {
        *n = 0;
        return fail(PCAD_ESTATE, "energy tracking is off");
    }
    unsigned int cnt = 0;
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    CUDA_TRY(cudaMemcpy(&cnt, ch->track.n, sizeof(cnt), cudaMemcpyDeviceToHost));
    const int k = (int)cnt < max ? (int)cnt : max;
    if (k > 0)
        CUDA_TRY(cudaMemcpy(host, ch->track.trace, (size_t)k * sizeof(double),
                            cudaMemcpyDeviceToHost));
    *n = (int)cnt;
    return PCAD_OK;
}

pcad_status pcad_chain_read_min_state(pcad_chain *ch, uint8_t *host_out, int out_pitch,
                                      double *energy, uint64_t *sweep)
{
    if (!ch || !host_out || out_pitch < ch->W)
        return fail(PCAD_EINVAL, "bad output buffer");
    if (!ch->track.trace)
        return fail(PCAD_ESTATE, "energy tracking is off");
    double best = 0.0;
    unsigned long long bs = 0;
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    CUDA_TRY(cudaMemcpy(&best, ch->track.best, sizeof(best), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&bs, ch->track.best_sweep, sizeof(bs), cudaMemcpyDeviceToHost));
    if (bs == 0)
        return fail(PCAD_ESTATE, "no sweep has been tracked yet");
    CUDA_TRY(cudaMemcpy2D(host_out, out_pitch, ch->track.xb, ch->pitch, ch->W, ch->H,
                          cudaMemcpyDeviceToHost));
    if (energy)
        *energy = best;
    if (sweep)
        *sweep = bs;
    return PCAD_OK;
}

pcad_status pcad_chain_set_kernel(pcad_chain *ch, int kind)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (kind != PCAD_KERNEL_AUTO && kind != PCAD_KERNEL_CUDA_CORE &&
        kind != PCAD_KERNEL_TENSOR && kind != PCAD_KERNEL_WAVE && kind != PCAD_KERNEL_SMALL &&
        kind != PCAD_KERNEL_RESIDENT && kind != PCAD_KERNEL_WINDOW &&
        kind != PCAD_KERNEL_WINDOW_WAVE && kind != PCAD_KERNEL_BINARY)
        return fail(PCAD_EINVAL, "kernel kind must be PCAD_KERNEL_AUTO, _CUDA_CORE, _TENSOR, "
                                 "_WAVE, _SMALL, _RESIDENT, _WINDOW, _WINDOW_WAVE or _BINARY");
    if (kind == PCAD_KERNEL_WINDOW_WAVE && !pca_win_eligible(ch->dm))
        return fail(PCAD_EINVAL, "the windowed wavefront sweep needs 9 <= L <= 256, T <= 33, "
                                 "nbhd T <= 255 and the L0 price");
    if (kind == PCAD_KERNEL_WINDOW && !pca_win_eligible(ch->dm))
        return fail(PCAD_EINVAL, "the windowed sweep needs 9 <= L <= 256, T <= 33, "
                                 "nbhd T <= 255 and the L0 inertia price");
    if (kind == PCAD_KERNEL_BINARY &&
        (ch->model.sampler != PCAD_SAMPLER_PCA || !binary_eligible(ch->dm)))
        return fail(PCAD_EINVAL, "the two-label sweep needs the PCA sampler, L = 2 and 4 or 8 "
                                 "neighbours");
    if (kind == PCAD_KERNEL_RESIDENT && !resident_eligible(ch->dm, ch->H, ch->W))
        return fail(PCAD_EINVAL, "the resident kernel needs L = 2, 4 or 8 neighbours and at most "
                                 "4096 quads of 4 sites (H * ceil(W / 4))");
    if (kind == PCAD_KERNEL_SMALL &&
        (ch->model.sampler != PCAD_SAMPLER_PCA || !pca_small_eligible(ch->dm)))
        return fail(PCAD_EINVAL, "the small-label kernel needs the PCA sampler, 3 <= L <= 16, "
                                 "pair_coef >= 0 and the L0 inertia price");
    if (kind == PCAD_KERNEL_WAVE && (ch->model.sampler != PCAD_SAMPLER_PCA || ch->dm.norm != 0))
        return fail(PCAD_EINVAL, "the wavefront kernel needs the PCA sampler and the L0 price");
    if (kind == PCAD_KERNEL_TENSOR &&
        (!pca_tc_eligible(ch->dm) ||
         (ch->model.sampler != PCAD_SAMPLER_PCA && ch->model.nbhd != 4)))
        return fail(PCAD_EINVAL, "the tensor-core sweep needs 64 <= L <= 256, T <= 33, the L0 "
                                 "inertia price and, for Gibbs, the 4-neighbourhood");
    if (kind != ch->kernel && ch->graph) {
        cudaStreamSynchronize(ch->stream);
        cudaGraphExecDestroy(ch->graph);
        ch->graph = nullptr;
    }
    ch->kernel = kind;
    return PCAD_OK;
}

namespace {

// Captured sweeps hold the launch arguments: rebuild them on next use.
void drop_graph(pcad_chain *ch)
{
    if (ch->graph) {
        cudaStreamSynchronize(ch->stream);
        cudaGraphExecDestroy(ch->graph);
        ch->graph = nullptr;
    }
}

}  // namespace

pcad_status pcad_chain_set_wait_limit(pcad_chain *ch, double seconds)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (!(seconds >= 1e-4 && seconds <= 60.0))
        return fail(PCAD_EINVAL, "wait limit must lie in [1e-4, 60] seconds");
    const long long ns = (long long)(seconds * 1e9);
    if (ns != ch->wait_ns) {
        drop_graph(ch);
        ch->wait_ns = ns;
    }
    return PCAD_OK;
}

pcad_status pcad_chain_inject_stall(pcad_chain *ch, int tile)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (tile < -1 || tile >= ch->wave_tiles)
        return fail(PCAD_EINVAL, "tile must be -1 (off) or a tile index below %d", ch->wave_tiles);
    if (tile + 1 != ch->stall_tile) {
        drop_graph(ch);
        ch->stall_tile = tile + 1;
    }
    return PCAD_OK;
}

pcad_status pcad_chain_set_row_offset(pcad_chain *ch, int row_off)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (row_off < 0 || row_off > kMaxRowOffset)
        return fail(PCAD_EINVAL, "row offset must lie in [0, %d]", kMaxRowOffset);
    if (ch->model.sampler != PCAD_SAMPLER_PCA && row_off != 0)
        return fail(PCAD_EINVAL, "row bands run the lazy PCA sampler");
    if (row_off != ch->row_off) {
        drop_graph(ch);
        ch->row_off = row_off;
    }
    return PCAD_OK;
}

pcad_status pcad_chain_write_rows_dev(pcad_chain *ch, int row0, int nrows, const uint8_t *src_dev,
                                      int src_pitch)
{
    if (!ch || !src_dev)
        return fail(PCAD_EINVAL, "NULL argument");
    if (row0 < 0 || nrows < 0 || row0 + nrows > ch->H || src_pitch < ch->W)
        return fail(PCAD_EINVAL, "rows [%d, %d) outside the chain's %d rows or src_pitch < W",
                    row0, row0 + nrows, ch->H);
    if (nrows == 0)
        return PCAD_OK;
    CUDA_TRY(cudaMemcpy2DAsync(ch->x[ch->cur] + (size_t)row0 * ch->pitch, ch->pitch, src_dev,
                               src_pitch, ch->W, nrows, cudaMemcpyDefault, ch->stream));
    return PCAD_OK;
}

pcad_status pcad_chain_set_blocking(pcad_chain *ch, int k)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (k != 0 && k != 1 && k != 2 && k != 4 && k != 8)
        return fail(PCAD_EINVAL, "sweeps per launch must be 0 (unblocked), 1, 2, 4 or 8");
    if (k > 0 && ch->model.sampler != PCAD_SAMPLER_PCA)
        return fail(PCAD_EINVAL, "temporal blocking applies to the PCA sampler");
    if (k > 0 && ch->dm.norm != 0)
        return fail(PCAD_EINVAL, "temporal blocking runs the L0 inertia price only");
    if (k > 0 && ch->track.trace)
        return fail(PCAD_ESTATE, "energy tracking needs every sweep's state: no temporal blocking");
    if (k > 0 && !ensure_maps(ch))
        return fail(PCAD_ECUDA, "TMA descriptor encoding failed");
    if (k != ch->tb_k && ch->graph) {
        cudaStreamSynchronize(ch->stream);
        cudaGraphExecDestroy(ch->graph);
        ch->graph = nullptr;
    }
    ch->tb_k = k;
    return PCAD_OK;
}

pcad_status pcad_chain_read_sample(pcad_chain *ch, uint8_t *host_out, int out_pitch)
{
    if (!ch || !host_out)
        return fail(PCAD_EINVAL, "NULL argument");
    if (out_pitch < ch->W)
        return fail(PCAD_EINVAL, "out_pitch < W");
    CUDA_TRY(cudaMemcpy2DAsync(host_out, out_pitch, ch->x[ch->cur], ch->pitch, ch->W, ch->H,
                               cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    return PCAD_OK;
}

pcad_status pcad_chain_read_sample_dev(pcad_chain *ch, uint8_t *dev_out, int out_pitch)
{
    if (!ch || !dev_out)
        return fail(PCAD_EINVAL, "NULL argument");
    if (out_pitch < ch->W)
        return fail(PCAD_EINVAL, "out_pitch < W");
    CUDA_TRY(cudaMemcpy2DAsync(dev_out, out_pitch, ch->x[ch->cur], ch->pitch, ch->W, ch->H,
                               cudaMemcpyDeviceToDevice, ch->stream));
    return PCAD_OK;
}

pcad_status pcad_chain_read_mean(pcad_chain *ch, float *host_out)
{
    if (!ch || !host_out)
        return fail(PCAD_EINVAL, "NULL argument");
    if (ch->n_acc == 0)
        return fail(PCAD_ESTATE, "no sweep accumulated yet");
    const long n = (long)ch->H * ch->W;
    CUDA_TRY(launch_mean(ch->acc, (float)ch->n_acc, ch->fplane, n, ch->stream));
    CUDA_TRY(cudaMemcpyAsync(host_out, ch->fplane, n * sizeof(float), cudaMemcpyDeviceToHost,
                             ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    return PCAD_OK;
}

pcad_status pcad_chain_write_sample(pcad_chain *ch, const uint8_t *host_in, int in_pitch)
{
    if (!ch || !host_in)
        return fail(PCAD_EINVAL, "NULL argument");
    if (in_pitch < ch->W)
        return fail(PCAD_EINVAL, "in_pitch < W");
    uint8_t *dst = ch->x[ch->cur];
    CUDA_TRY(cudaMemcpy2DAsync(dst, ch->pitch, host_in, in_pitch, ch->W, ch->H,
                               cudaMemcpyHostToDevice, ch->stream));
    int *bad = (int *)ch->mscratch;
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), ch->stream));
    CUDA_TRY(launch_check_labels(dst, ch->pitch, ch->H, ch->W, ch->model.L, bad, ch->stream));
    int hbad = 0;
    CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    if (hbad)
        return fail(PCAD_EINVAL, "%d labels are >= L", hbad);
    return PCAD_OK;
}

pcad_status pcad_chain_sweeps(const pcad_chain *ch, uint64_t *t, uint64_t *n_accumulated)
{
    if (!ch)
        return fail(PCAD_EINVAL, "chain is NULL");
    if (t)
        *t = ch->t;
    if (n_accumulated)
        *n_accumulated = ch->n_acc;
    return PCAD_OK;
}

pcad_status pcad_chain_stats(pcad_chain *ch, uint64_t *fp64_draws)
{
    if (!ch || !fp64_draws)
        return fail(PCAD_EINVAL, "NULL argument");
    unsigned long long v = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, ch->fp64, sizeof(v), cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    *fp64_draws = v;
    return PCAD_OK;
}

pcad_status pcad_chain_metrics(pcad_chain *ch, const uint8_t *clean_host, int clean_pitch,
                               int which, double *psnr_db, double *ssim)
{
    if (!ch || !clean_host)
        return fail(PCAD_EINVAL, "NULL argument");
    if (clean_pitch < ch->W)
        return fail(PCAD_EINVAL, "clean_pitch < W");
    const long n = (long)ch->H * ch->W;
    if (which == 0) {
        if (ch->n_acc == 0)
            return fail(PCAD_ESTATE, "no sweep accumulated yet");
        CUDA_TRY(launch_mean(ch->acc, (float)ch->n_acc, ch->fplane, n, ch->stream));
    } else {
        CUDA_TRY(launch_labels_to_float(ch->x[ch->cur], ch->pitch, ch->H, ch->W, ch->fplane,
                                        ch->stream));
    }
    CUDA_TRY(cudaMemcpy2DAsync(ch->clean, ch->W, clean_host, clean_pitch, ch->W, ch->H,
                               cudaMemcpyHostToDevice, ch->stream));
    CUDA_TRY(launch_metrics(ch->fplane, ch->clean, ch->H, ch->W, ch->model.L, ch->mscratch,
                            ch->mscratch + 8, ch->stream));
    double res[2];
    CUDA_TRY(cudaMemcpyAsync(res, ch->mscratch + 8, sizeof(res), cudaMemcpyDeviceToHost,
                             ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    if (psnr_db)
        *psnr_db = res[0];
    if (ssim)
        *ssim = res[1];
    return PCAD_OK;
}

pcad_status pcad_metrics(const float *est_host, const uint8_t *clean_host, int H, int W, int L,
                         double *psnr_db, double *ssim)
{
    if (!est_host || !clean_host)
        return fail(PCAD_EINVAL, "NULL argument");
    if (H < 1 || W < 1 || L < 2 || L > 256 || (long long)H * W < 2)
        return fail(PCAD_EINVAL, "bad sizes");
    const size_t n = (size_t)H * W;
    void *blk = nullptr;
    const size_t fb = align_up(n * sizeof(float), 256), cb = align_up(n, 256);
    CUDA_TRY(cudaMalloc(&blk, fb + cb + 16 * sizeof(double)));
    float *est = (float *)blk;
    uint8_t *clean = (uint8_t *)((char *)blk + fb);
    double *scr = (double *)((char *)blk + fb + cb);
    double res[2] = {0, 0};
    cudaError_t e = cudaMemcpy(est, est_host, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(clean, clean_host, n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_metrics(est, clean, H, W, L, scr, scr + 8, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(res, scr + 8, sizeof(res), cudaMemcpyDeviceToHost);
    cudaFree(blk);
    if (e != cudaSuccess)
        return fail(PCAD_ECUDA, "metrics: %s", cudaGetErrorString(e));
    if (psnr_db)
        *psnr_db = res[0];
    if (ssim)
        *ssim = res[1];
    return PCAD_OK;
}

namespace {
struct BlobHeader {
    char magic[8];
    uint32_t version;
    int32_t H, W, burn_in;
    pcad_model model;
    uint64_t seed;
    uint32_t chain_id;
    int32_t row_off;     // 0 for a whole image
    uint64_t t, n_acc, fp64;
};
const char kMagic[8] = {'P', 'C', 'A', 'D', 'C', 'H', 'N', '1'};
}  // namespace

pcad_status pcad_chain_export(pcad_chain *ch, void *host_blob, size_t *bytes)
{
    if (!ch || !bytes)
        return fail(PCAD_EINVAL, "NULL argument");
    const size_t n = (size_t)ch->H * ch->W;
    const size_t need = sizeof(BlobHeader) + 2 * n + n * sizeof(float);
    if (!host_blob) {
        *bytes = need;
        return PCAD_OK;
    }
    if (*bytes < need)
        return fail(PCAD_EINVAL, "blob too small: %zu < %zu", *bytes, need);
    BlobHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.H = ch->H;
    h.W = ch->W;
    h.burn_in = ch->burn_in;
    h.model = ch->model;
    h.seed = ch->seed;
    h.chain_id = ch->chain_id;
    h.row_off = ch->row_off;
    h.t = ch->t;
    h.n_acc = ch->n_acc;
    pcad_status st = pcad_chain_stats(ch, &h.fp64);
    if (st != PCAD_OK)
        return st;
    char *b = (char *)host_blob;
    memcpy(b, &h, sizeof(h));
    // layout: header | current labels | observation | accumulator
    CUDA_TRY(cudaMemcpy2DAsync(b + sizeof(h), ch->W, ch->x[ch->cur], ch->pitch, ch->W, ch->H,
                               cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaMemcpy2DAsync(b + sizeof(h) + n, ch->W, ch->g, ch->pitch, ch->W, ch->H,
                               cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaMemcpyAsync(b + sizeof(h) + 2 * n, ch->acc, n * sizeof(float),
                             cudaMemcpyDeviceToHost, ch->stream));
    CUDA_TRY(cudaStreamSynchronize(ch->stream));
    *bytes = need;
    return PCAD_OK;
}

pcad_status pcad_chain_import(const void *host_blob, size_t bytes, void *cuda_stream,
                              pcad_chain **out)
{
    if (!out)
        return fail(PCAD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!host_blob || bytes < sizeof(BlobHeader))
        return fail(PCAD_EINVAL, "blob too small");
    BlobHeader h;
    memcpy(&h, host_blob, sizeof(h));
    if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 1)
        return fail(PCAD_EINVAL, "not a pcaden chain blob");
    if (h.H < 1 || h.W < 1 || h.H > 65535 || h.W > 65535 || h.t > 0xFFFFFFFFull ||
        h.row_off < 0 || h.row_off > kMaxRowOffset)
        return fail(PCAD_EINVAL, "corrupt blob header");
    const size_t n = (size_t)h.H * h.W;
    if (bytes < sizeof(h) + 2 * n + n * sizeof(float))
        return fail(PCAD_EINVAL, "blob truncated");
    const char *b = (const char *)host_blob;
    pcad_chain *ch = nullptr;
    pcad_status st = pcad_chain_create((const uint8_t *)(b + sizeof(h) + n), h.H, h.W, h.W,
                                       &h.model, h.seed, h.chain_id, h.burn_in, cuda_stream, &ch);
    if (st != PCAD_OK)
        return st;
    ch->row_off = h.row_off;
    st = pcad_chain_write_sample(ch, (const uint8_t *)(b + sizeof(h)), h.W);
    if (st != PCAD_OK) {
        pcad_chain_destroy(ch);
        return st;
    }
    const uint32_t t32 = (uint32_t)h.t;
    const unsigned long long f = h.fp64;
    cudaError_t e = cudaMemcpyAsync(ch->acc, b + sizeof(h) + 2 * n, n * sizeof(float),
                                    cudaMemcpyHostToDevice, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ch->tdev, &t32, sizeof(t32), cudaMemcpyHostToDevice, ch->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ch->fp64, &f, sizeof(f), cudaMemcpyHostToDevice, ch->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ch->stream);
    if (e != cudaSuccess) {
        pcad_chain_destroy(ch);
        return fail(PCAD_ECUDA, "import: %s", cudaGetErrorString(e));
    }
    ch->t = h.t;
    ch->n_acc = h.n_acc;
    *out = ch;
    return PCAD_OK;
}

void pcad_chain_destroy(pcad_chain *ch)
{
    if (!ch)
        return;
    cudaStreamSynchronize(ch->stream);
    if (ch->graph)
        cudaGraphExecDestroy(ch->graph);
    if (ch->track_block)
        cudaFreeAsync(ch->track_block, ch->stream);
    cudaFreeAsync(ch->block, ch->stream);
    cudaStreamSynchronize(ch->stream);
    delete ch;
}

const char *pcad_status_str(pcad_status s)
{
    switch (s) {
    case PCAD_OK: return "ok";
    case PCAD_EINVAL: return "invalid argument";
    case PCAD_ENOMEM: return "out of memory";
    case PCAD_ECUDA: return "CUDA error";
    case PCAD_ETIMEOUT: return "device wait timed out";
    case PCAD_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char *pcad_last_error(void) { return g_err.c_str(); }

const char *pcad_version(void) { return "pcaden 0.1.0 (sm_103a)"; }

pcad_status pcad_model_margins(const pcad_model *m, double *out, int n)
{
    if (!m || !out || n < PCAD_N_MARGINS)
        return fail(PCAD_EINVAL, "model_margins: null argument or n < %d", PCAD_N_MARGINS);
    pcad_status st = validate_model(m);
    if (st != PCAD_OK)
        return st;
    ModelTables t;
    build_tables(*m, t);
    const DevModel &d = t.dm;
    const float v[PCAD_N_MARGINS] = {d.alpha, d.gam, d.eta, d.cb, d.hb, d.kb0, d.kb1, d.kbr};
    for (int i = 0; i < PCAD_N_MARGINS; ++i)
        out[i] = (double)v[i];
    return PCAD_OK;
}

}  // extern "C"

// Helpers shared with other translation units of the library.
namespace pcad {

pcad_status check_model(const pcad_model *m) { return validate_model(m); }

void model_tables(const pcad_model &m, double *ta64, std::vector<double> &pr64, DevModel &dm)
{
    ModelTables t;
    build_tables(m, t);
    memcpy(ta64, t.ta64, sizeof(t.ta64));
    pr64 = t.pr64;
    dm = t.dm;
}

pcad_status set_error(pcad_status st, const char *msg) { return fail(st, "%s", msg); }

uint8_t *chain_state(pcad_chain *ch) { return ch->x[ch->cur]; }
int chain_pitch(const pcad_chain *ch) { return ch->pitch; }
cudaStream_t chain_stream(const pcad_chain *ch) { return ch->stream; }

}  // namespace pcad
