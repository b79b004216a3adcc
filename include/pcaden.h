/*
 * pcaden -- lazy Probabilistic Cellular Automaton (PCA) sampler for Bayesian
 * image denoising on one NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Method: Costarelli, Piconi, Troiani, "Bayesian Inversion via Probabilistic
 * Cellular Automata: an application to image denoising" (arXiv 2507.14869).
 *
 * A chain holds a label image x (H x W, labels 0..L-1) and samples, sweep by
 * sweep, an approximation of the denoising posterior of Section 2 (Bayes'
 * rule with a Gibbs prior, Eq. gibbs-prior, and a noise likelihood,
 * Eq. likelihood_general_expression).  Two samplers:
 *
 *   PCAD_SAMPLER_PCA       the lazy PCA of Section 5.2 (Eq.
 *                          posterior_pca_transition_matrix): every pixel is
 *                          resampled simultaneously from its conditional on
 *                          the previous configuration, with an inertial price
 *                          lambda * 1{s != x_i} for changing label;
 *   PCAD_SAMPLER_GIBBS_CB  the single-site Gibbs sampler of Section 5.1
 *                          (Eq. gibbs_sampler_elementary_step) in checkerboard
 *                          colour order (2 colours for the 4-neighbourhood, 4
 *                          for the 8-neighbourhood), in place.
 *
 * Energy of label s at site i (lower = likelier), in natural-log units:
 *   E_i(s) = sum_{j in N(i)} V(s, x_j) + U(g_i, s) + lambda * 1{s != x_i}
 *   V(s,t) = -pair_coef * 1{s = t}              (Potts, Eq. prior_pair_potential;
 *                                                pair_coef = c_P = 2 beta J)
 *          =  pair_coef * min(|s - t|, pair_T)  (truncated linear)
 *   U(g,s) = (g - s)^2 / (2 sigma^2)            (Gaussian, sigma in label units)
 *          = -ln(1-p) if s = g else -ln p       (flip channel, L = 2 only)
 * N(i) is the 4- or 8-neighbourhood (Eq. neighborhood); neighbours outside
 * the image are dropped (free boundary).  The initial state is the
 * observation g.  Draws are inverse-CDF in label order with a 24-bit uniform
 * from Philox4x32-10 keyed by (seed, chain, sweep, row, col) (see DRAWS).
 *
 * DRAWS.  Counter (col >> 2, row, sweep, (tag << 24) | chain), key (seed low,
 * seed high), word col & 3, u = (word >> 8) * 2^-24; tag 0 = PCA, 1 = Gibbs.
 * New label = smallest k with u * Z < C_k, C_k = sum_{s <= k} exp(-E_i(s)),
 * Z = C_{L-1}.  The kernels evaluate this in FP32 with a rigorous error
 * bound and re-evaluate in FP64 every draw whose uniform lies within that
 * bound of a CDF boundary; such draws are counted (pcad_chain_stats).
 *
 * CONVENTIONS.
 *   - Every function returns a pcad_status; nothing throws across the ABI.
 *     On failure, output handles are set to NULL and pcad_last_error()
 *     returns a message for the calling thread.
 *   - Images are row-major uint8 label planes; "pitch" is the distance in
 *     bytes between rows (>= W).  Host buffers are owned by the caller.
 *   - A chain owns its device memory (allocated on its stream) and is not
 *     thread-safe: one host thread at a time.  cuda_stream is a cudaStream_t
 *     (NULL = the legacy default stream); run calls are asynchronous on it,
 *     read calls synchronise it.
 *   - Limits: 2 <= L <= 256; nbhd 4 or 8; 1 <= H, W <= 65535 (H*W <= 2^31);
 *     prior range (pair_coef * nbhd * pair_T, or |pair_coef| * nbhd for
 *     Potts) <= 40; 0 <= lambda <= 40; flip only with L = 2 and
 *     |ln((1-p)/p)| <= 40; chain id < 2^24.  The posterior-mean accumulator
 *     is FP32 and exact while (L-1) * (accumulated sweeps) < 2^24; run calls
 *     that would pass that bound fail with PCAD_EINVAL.
 */
#ifndef PCADEN_H
#define PCADEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PCAD_OK = 0,
    PCAD_EINVAL = 1,   /* invalid argument or parameter outside the limits */
    PCAD_ENOMEM = 2,   /* device or host allocation failed / budget exceeded */
    PCAD_ECUDA = 3,    /* a CUDA runtime call failed */
    PCAD_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    PCAD_ESTATE = 5    /* call not valid in the object's current state */
} pcad_status;

typedef enum { PCAD_PAIR_POTTS = 0, PCAD_PAIR_TRUNC_LINEAR = 1 } pcad_pair;
/* PCAD_NOISE_NONE: no likelihood (U = 0): the chain samples the prior; used
 * to synthesise MRF test images from random labels (Section 6). */
typedef enum { PCAD_NOISE_GAUSS = 0, PCAD_NOISE_FLIP = 1, PCAD_NOISE_NONE = 2 } pcad_noise;
typedef enum { PCAD_SAMPLER_PCA = 0, PCAD_SAMPLER_GIBBS_CB = 1 } pcad_sampler;

/* Model parameters (Sections 4-5).  pair_coef: Potts reward c_P = 2 beta J or
 * truncated-linear slope c_T; pair_T: truncation (ignored for Potts); sigma:
 * Gaussian std in label units; flip_p: flip probability; inertia: lambda =
 * beta q (0 gives the naive synchronous update; ignored by Gibbs);
 * inertia_norm: the inertia price of changing label x_i to s (Section 3) --
 * 0: lambda 1{s != x_i} (L0), 1 or 2: lambda (|s - x_i| / (L - 1))^p on
 * intensities (L1 / L2).  The norms run on the single-chain sweep kernel
 * (not with temporal blocking, batches or the tensor-core kernel). */
typedef struct {
    int L;
    int nbhd;
    int pair;        /* pcad_pair */
    float pair_coef;
    int pair_T;
    int noise;       /* pcad_noise */
    float sigma;
    float flip_p;
    float inertia;
    int sampler;     /* pcad_sampler */
    int inertia_norm; /* 0 (L0), 1 (L1) or 2 (L2) */
} pcad_model;

typedef struct pcad_chain pcad_chain;

/* Create a chain from a host observation g (H x W labels, row pitch g_pitch
 * bytes).  The state starts at g, the sweep counter at 0.  burn_in: number
 * of initial sweeps not accumulated into the posterior mean.  Problem
 * statement: Section 2 (noisy g, noise model, prior, inertia). */
pcad_status pcad_chain_create(const uint8_t *g_host, int H, int W, int g_pitch,
                              const pcad_model *m, uint64_t seed, uint32_t chain_id,
                              int burn_in, void *cuda_stream, pcad_chain **out);

/* Same, from a device observation (borrowed for the duration of the call and
 * copied on cuda_stream). */
pcad_status pcad_chain_create_dev(const uint8_t *g_dev, int H, int W, int g_pitch,
                                  const pcad_model *m, uint64_t seed, uint32_t chain_id,
                                  int burn_in, void *cuda_stream, pcad_chain **out);

/* Run nsweeps sweeps (asynchronous; continues the sweep counter).  After the
 * k-th sweep overall (k = 1, 2, ...), the state is added to the accumulator
 * when k > burn_in (conditional-mean estimator, Section 2). */
pcad_status pcad_chain_run(pcad_chain *ch, int nsweeps);

/* Restart the chain from its observation (state = g, accumulator and
 * counters zero, sweep counter 0) without reallocating (asynchronous). */
pcad_status pcad_chain_reset(pcad_chain *ch);

/* Temporal blocking of the PCA sweep: k = 1, 2, 4 or 8 sweeps per kernel
 * launch on shared-memory tiles loaded by TMA with a k-site halo (the tile
 * recomputes its halo, so the labels are bit-identical to unblocked runs);
 * k = 0 (the default) issues one launch per sweep with no tiles.  Fewer
 * than k remaining sweeps of a run use single-sweep launches.  PCAD_EINVAL
 * for other k or the Gibbs sampler; PCAD_ECUDA if the driver cannot encode
 * the tile descriptors.  pcad_chain_sync reports PCAD_ETIMEOUT if a tile
 * load ever failed to complete within its bounded wait. */
pcad_status pcad_chain_set_blocking(pcad_chain *ch, int k);

/* Kernel of the unblocked PCA sweep (k = 0 above) and of the Gibbs sweep.  The prior sum of
 * Eq. posterior_pca_transition_matrix is a sum of tents
 * max(T - |x_j - s|, 0) over the neighbours.  PCAD_KERNEL_TENSOR computes
 * it on the tensor cores (tcgen05): each site histograms its neighbour
 * labels relative to its own base label (64 bins), one MMA chain gives the
 * tent sums over the 128-label window holding them, labels outside it take
 * chunk sums of the Gaussian data term from a shared-memory table, and
 * neighbours beyond the 64 bins are added on the CUDA cores; sweeps run as
 * a wavefront (below).  PCAD_KERNEL_CUDA_CORE evaluates every label's prior
 * on the CUDA cores.  All kernels draw exactly the same labels.  The
 * tensor-core kernel accepts 64 <= L <= 256, truncation T <= 33 (Potts:
 * T = 1) and the L0 price, for the PCA sampler and for the checkerboard
 * Gibbs sampler with the 4-neighbourhood (colour phases over 8 x 32 tiles,
 * in place, as a wavefront of phases; Section 5.1); PCAD_EINVAL for an
 * unknown kind or PCAD_KERNEL_TENSOR on another model.  PCAD_KERNEL_AUTO
 * (the default) takes it for L >= 192 without energy tracking (where it
 * measured faster on GB300), except on images of at least 8 blocks of
 * 4 x 32 sites per multiprocessor, which take the windowed kernels (below;
 * see pcad_chain_kernel_in_use); else the per-sweep or the wavefront
 * CUDA-core kernel.  PCAD_KERNEL_WAVE runs the
 * CUDA-core draw as one persistent launch per block of sweeps, a tile of
 * 4 x 32 sites starting sweep k as soon as its 3 x 3 neighbouring tiles
 * finished sweep k - 1 (no sweep-wide barrier, so one sweep's tail
 * overlaps the next one's start); same labels; L0 price only (PCAD_EINVAL
 * with an Lp norm).  Energy tracking runs the wavefront kernels one sweep
 * per launch.  pcad_chain_sync reports PCAD_ETIMEOUT if a tensor-core
 * completion wait or a wavefront dependency wait ever gave up.
 * PCAD_KERNEL_SMALL (3 <= L <= 16, pair_coef >= 0, L0 price, PCA sampler;
 * PCAD_EINVAL otherwise) runs one launch per sweep that takes the prior sums
 * of all labels of a site from a table of neighbour pairs (16 bytes per pair
 * of labels, in shared memory) and draws from chunk prefix sums in
 * registers; same labels as the other kernels.  Images of at least 2^23
 * sites sweep on TMA-loaded 64 x 46 tiles in persistent blocks (the next
 * tile's copy in flight during the draw), smaller ones on persistent
 * 16 x 32 tiles staged by the threads.  AUTO takes it for every model it
 * accepts.  PCAD_KERNEL_RESIDENT (L = 2, 4- or 8-neighbourhood,
 * either sampler, H * ceil(W / 4) <= 4096, e.g. up to 128 x 128, and at most
 * 200 KB of shared memory; PCAD_EINVAL otherwise) runs all the sweeps of a
 * run in one launch of one 1024-thread CTA that keeps the state in shared
 * memory and draws each site from a table of exact thresholds on its
 * uniform, one per site configuration (x_i, g_i, label-1 neighbours,
 * neighbours outside the image), computed at set-up from the FP32 draw and
 * FP64 re-draw of the other kernels; same labels and the same FP64 re-draw
 * count (with two labels every inertia price is the L0 one).  AUTO takes it
 * for the images it accepts (no energy tracking, no temporal blocking).
 * PCAD_KERNEL_WINDOW (9 <= L <= 256, truncation 1 <= T <= 33 with
 * nbhd T <= 255, the L0 price, either sampler and neighbourhood;
 * PCAD_EINVAL otherwise)
 * runs one launch per sweep (per Gibbs colour phase) on the CUDA cores with
 * the tensor-core sweep's weights: each site evaluates only the label chunks
 * its neighbours' tents reach, their tent sums read from a table of 8 tents
 * per 8-byte shared-memory entry, the other chunks' sums from a table of the
 * observation, the sites of a block sorted by the number of such chunks so
 * that a warp's lanes do similar work; same labels.  PCAD_KERNEL_WINDOW_WAVE
 * (the same models, either sampler) runs the windowed draw as one
 * persistent wavefront launch per block of sweeps (of Gibbs colour phases),
 * as PCAD_KERNEL_WAVE does the CUDA-core draw (energy tracking: one launch
 * per sweep); same labels.  PCAD_KERNEL_BINARY (L = 2, 4- or 8-neighbourhood,
 * PCA sampler; PCAD_EINVAL otherwise) runs one launch per sweep that draws
 * each site by one read of the resident kernel's threshold table and a
 * compare (persistent blocks over tiles of 16 x 128 sites staged in shared
 * memory); same labels and the same FP64 re-draw count.  AUTO takes it for
 * two-label images of at least 2^18 sites. */
typedef enum {
    PCAD_KERNEL_AUTO = 0,
    PCAD_KERNEL_CUDA_CORE = 1,
    PCAD_KERNEL_TENSOR = 2,
    PCAD_KERNEL_WAVE = 3,
    PCAD_KERNEL_SMALL = 4,
    PCAD_KERNEL_RESIDENT = 5,
    PCAD_KERNEL_WINDOW = 6,
    PCAD_KERNEL_WINDOW_WAVE = 7,
    PCAD_KERNEL_BINARY = 8
} pcad_kernel;
pcad_status pcad_chain_set_kernel(pcad_chain *ch, int kind);

/* The kernel the chain's next sweeps run: PCAD_KERNEL_CUDA_CORE (one launch
 * per sweep or Gibbs colour phase), PCAD_KERNEL_WAVE, PCAD_KERNEL_TENSOR,
 * PCAD_KERNEL_SMALL, PCAD_KERNEL_RESIDENT, PCAD_KERNEL_WINDOW,
 * PCAD_KERNEL_BINARY, or -k for temporal blocking with k sweeps per launch.
 * With PCAD_KERNEL_AUTO the resident kernel
 * is taken for the two-label images it accepts without energy tracking, the
 * two-label sweep for two-label images of at least 2^18 sites; the
 * windowed kernels for chains of models they accept with L >= 32 (any
 * neighbourhood for Gibbs) without energy tracking, by image size in blocks
 * of 4 x 32 sites per
 * multiprocessor: PCAD_KERNEL_WINDOW from 100, PCAD_KERNEL_WINDOW_WAVE from 8
 * (8-neighbourhood Gibbs: from 3); the tensor-core kernel for the
 * other eligible models with L >= 192 and no energy tracking;
 * PCAD_KERNEL_SMALL for the models it accepts; otherwise
 * the wavefront kernel for L >= 16 when the
 * image has between 1/2 and 3 waves of 4 x 32 tiles at 10 resident tiles
 * per multiprocessor (the sizes where it measured faster on GB300), the
 * per-sweep kernel otherwise. */
pcad_status pcad_chain_kernel_in_use(const pcad_chain *ch, int *kind);

/* Change the model's coefficients (pair_coef, sigma, flip_p, inertia) for
 * the sweeps queued after this call; L, nbhd, pair, pair_T, noise and
 * sampler must stay (PCAD_EINVAL otherwise).  The state, the accumulator
 * and the sweep counter carry on.  This is the annealing step of Section 6:
 * with beta rising, c_P = 2 beta J and lambda = beta q are rescaled while
 * the likelihood stays (its 1/(2 sigma^2) is not multiplied by beta). */
pcad_status pcad_chain_set_model(pcad_chain *ch, const pcad_model *m);

/* Run a schedule: for each stage k, set models[k] and run sweeps[k] sweeps
 * (the annealed protocol of Section 6: beta = 1.25 + 0.25 k for 4 stages of
 * 250 sweeps, with the last sample as the estimate). */
pcad_status pcad_chain_run_schedule(pcad_chain *ch, const pcad_model *models, const int *sweeps,
                                    int nstages);

/* Posterior energy of the current sample x (Section 4, Eq.
 * mrf_gauss_noise_posterior_distribution; pi_post ~ exp(-H)):
 *   H(x) = sum over unordered neighbour pairs V(x_i, x_j) + sum_i U(g_i, x_i)
 * with the per-edge pair weight of the single-site conditional (Potts
 * V = -c_P 1{x_i = x_j}, truncated linear V = c_T min(|x_i - x_j|, T);
 * Gaussian U = (g - x)^2 / (2 sigma^2), flip U = -ln(1 - p) or -ln p), free
 * boundary.  Optional outputs: the integer sums it is made of -- pair_sum
 * (Potts: pairs with equal labels; truncated linear: sum of
 * min(|x_i - x_j|, T)) and data_sum (Gaussian: sum of (g - x)^2; flip:
 * sites with x != g); H = (-c_P or c_T) pair_sum + data_sum / (2 sigma^2)
 * (Gaussian) or -ln(1-p) (H W - data_sum) - ln(p) data_sum (flip), in FP64.
 * Synchronises the chain's stream. */
pcad_status pcad_chain_energy(pcad_chain *ch, double *energy, uint64_t *pair_sum,
                              uint64_t *data_sum);

/* Minimum-energy tracking (the maximum a posteriori state by lowest
 * posterior energy, Section 2): with capacity > 0, every later sweep also
 * computes H of its result, records it (the first `capacity` values) and
 * keeps the lowest-energy state seen with the number of completed sweeps
 * at which it occurred; pcad_chain_reset clears the record.  capacity = 0
 * turns tracking off and frees its memory (pitch x H bytes + 8 capacity
 * bytes).  PCAD_ESTATE with temporal blocking on (and set_blocking refuses
 * k > 0 while tracking).  Not part of an exported checkpoint. */
pcad_status pcad_chain_track_energy(pcad_chain *ch, int capacity);

/* Energies recorded so far: *n = their number (may exceed max; the first
 * min(*n, max) are copied to host).  PCAD_ESTATE when tracking is off. */
pcad_status pcad_chain_read_energies(pcad_chain *ch, double *host, int max, int *n);

/* The lowest-energy state recorded (H rows of W bytes, row pitch
 * out_pitch), its energy and its sweep count.  PCAD_ESTATE when tracking is
 * off or no sweep was tracked yet. */
pcad_status pcad_chain_read_min_state(pcad_chain *ch, uint8_t *host_out, int out_pitch,
                                      double *energy, uint64_t *sweep);

/* Failure detection (no counterpart in the paper: the sweep of Section 5.2
 * needs no waits, but the wavefront, tensor-core and TMA-tiled kernels
 * that run it wait on one another's tiles, on MMA completion and on tile
 * loads).  Every such device-side wait is bounded by elapsed time: after
 * `seconds` (default 1.0; accepted range [1e-4, 60], PCAD_EINVAL outside)
 * it gives up and sets the chain's error flag, every other wait and work
 * item of the launch stops as soon as it sees the flag, the kernel returns
 * and pcad_chain_sync reports PCAD_ETIMEOUT.  The sample and accumulator
 * are then undefined; pcad_chain_reset clears the flag and restarts the
 * chain.  Applies to sweeps queued after the call. */
pcad_status pcad_chain_set_wait_limit(pcad_chain *ch, double seconds);

/* Test aid for the failure path above: with tile >= 0, tile `tile` of the
 * wavefront CUDA-core kernel's and the tensor-core kernel's grid (4 x 32
 * sites, row-major; Gibbs: 8 x 32) never reports a finished sweep, so the
 * tiles around it wait for a dependency that never arrives until their
 * bounded wait runs out.  tile = -1 (the default) turns it off; PCAD_EINVAL
 * for tile outside [-1, tiles).  Applies to sweeps queued after the call;
 * no other kernel is affected. */
pcad_status pcad_chain_inject_stall(pcad_chain *ch, int tile);

/* Row offset of a chain that holds a band of rows of a larger image: its
 * local row r is global row r + row_off, and the Philox counter of every
 * draw uses the global row (DRAWS), so a band draws what the whole-image
 * chain draws at those rows.  row_off in [0, 2^30]; PCAD_EINVAL otherwise
 * or for the Gibbs sampler (its colour classes follow the local rows).
 * Exported with the chain.  Applies to sweeps queued after the call.  The
 * row-band runner below uses it; a multi-process runner (one band per
 * rank) uses it with pcad_chain_write_rows_dev for its halo exchange. */
pcad_status pcad_chain_set_row_offset(pcad_chain *ch, int row_off);

/* Overwrite rows [row0, row0 + nrows) of the current state with nrows rows
 * of W labels from device (or peer / host-mapped) memory at src_dev, row
 * pitch src_pitch; stream-ordered on the chain's stream, asynchronous.  The
 * labels must be < L (not checked here: a halo exchange copies labels that
 * another band of the same model drew).  PCAD_EINVAL for rows outside the
 * chain or src_pitch < W. */
pcad_status pcad_chain_write_rows_dev(pcad_chain *ch, int row0, int nrows, const uint8_t *src_dev,
                                      int src_pitch);

/* Block until the chain's queued work is done. */
pcad_status pcad_chain_sync(pcad_chain *ch);

/* Copy the current sample (the paper's retrieved image is the last sample,
 * Section 6) to host memory (H rows of W bytes, row pitch out_pitch). */
pcad_status pcad_chain_read_sample(pcad_chain *ch, uint8_t *host_out, int out_pitch);

/* Copy the current sample to device memory (asynchronous on the chain's stream). */
pcad_status pcad_chain_read_sample_dev(pcad_chain *ch, uint8_t *dev_out, int out_pitch);

/* Posterior-mean estimate in label units (mean of the accumulated samples;
 * for L = 2 the mean spin is 2 * value - 1), H x W floats, host memory.
 * PCAD_ESTATE when nothing has been accumulated yet. */
pcad_status pcad_chain_read_mean(pcad_chain *ch, float *host_out);

/* Overwrite the current state with host labels (every label < L). */
pcad_status pcad_chain_write_sample(pcad_chain *ch, const uint8_t *host_in, int in_pitch);

/* Sweeps done so far and sweeps accumulated into the mean. */
pcad_status pcad_chain_sweeps(const pcad_chain *ch, uint64_t *t, uint64_t *n_accumulated);

/* Draws re-evaluated in FP64 because their uniform fell within the FP32
 * error bound of a CDF boundary (synchronises the chain). */
pcad_status pcad_chain_stats(pcad_chain *ch, uint64_t *fp64_draws);

/* PSNR (dB) and SSIM of the chain's posterior mean against a clean host
 * label image, luminance label/(L-1) (Section 6: PSNR with max x of the
 * original; SSIM of Wang et al. 2004, 11x11 Gaussian window sigma 1.5,
 * K1 = 0.01, K2 = 0.03, range 1, over window positions inside the image;
 * images smaller than 11 use the single-window form).  Computed on the GPU
 * in FP64.  which = 0: posterior mean, 1: current sample. */
pcad_status pcad_chain_metrics(pcad_chain *ch, const uint8_t *clean_host, int clean_pitch,
                               int which, double *psnr_db, double *ssim);

/* PSNR / SSIM of an arbitrary estimate (label units, H x W floats, host)
 * against clean labels (host), as above. */
pcad_status pcad_metrics(const float *est_host, const uint8_t *clean_host, int H, int W,
                         int L, double *psnr_db, double *ssim);

/* Checkpoint: serialise the whole chain state (labels, accumulator,
 * counters, model, RNG key) to a host blob.  With host_blob = NULL only the
 * required size is written to *bytes.  Synchronises the chain. */
pcad_status pcad_chain_export(pcad_chain *ch, void *host_blob, size_t *bytes);

/* Re-create a chain from an exported blob on cuda_stream; continuing it is
 * bit-identical to continuing the original. */
pcad_status pcad_chain_import(const void *host_blob, size_t bytes, void *cuda_stream,
                              pcad_chain **out);

/* Release the chain's device memory (synchronises its stream).  NULL is a no-op. */
void pcad_chain_destroy(pcad_chain *ch);

/* ------------------------------------------------------------- batches
 * Many independent lazy-PCA chains (the paper's repeated runs, e.g. 10 runs
 * x 14 inertia values in Section 6, are such a batch) advanced together: one
 * persistent launch per sweep covers every chain, whatever its size, label
 * count or model.  A chain's draws depend only on its own (seed, chain id,
 * sweep, row, col), so each chain's results are bit-identical to running it
 * alone with pcad_chain_create + pcad_chain_run. */
typedef struct {
    const uint8_t *g_host;   /* observation (H rows of g_pitch bytes, labels < L:
                                PCAD_EINVAL otherwise); copied at creation */
    int H, W, g_pitch;
    pcad_model model;        /* sampler must be PCAD_SAMPLER_PCA */
    uint64_t seed;
    uint32_t chain_id;
    int burn_in;
} pcad_job;

typedef struct pcad_batch pcad_batch;

/* Create a batch of n chains (one per job) on cuda_stream.  autotune != 0
 * times the tilings below on this batch and keeps the fastest, cached per
 * batch signature for the process: one persistent launch per sweep with
 * work items of 4/8/16 rows x 32 sites in cost order (order 1) or image
 * order (order 0), or one wavefront launch per 16 sweeps with 4/8-row
 * tiles (order 2; a tile's sweep starts when its 3 x 3 neighbourhood
 * finished the previous one).  Without autotuning: 4 rows, order 1. */
pcad_status pcad_batch_create(const pcad_job *jobs, int n, int autotune, void *cuda_stream,
                              pcad_batch **out);
/* Advance every chain by nsweeps sweeps (asynchronous). */
pcad_status pcad_batch_run(pcad_batch *b, int nsweeps);

/* Change chain i's coefficients for the sweeps queued after this call (as
 * pcad_chain_set_model: L, nbhd, pair, pair_T, noise and sampler stay).
 * Synchronises the batch's stream. */
pcad_status pcad_batch_set_model(pcad_batch *b, int i, const pcad_model *m);
/* Restart every chain from its observation (asynchronous). */
pcad_status pcad_batch_reset(pcad_batch *b);
/* Wait for the batch's queued work.  PCAD_ETIMEOUT: a bounded wait inside a
 * wavefront launch gave up (the batch's results are invalid). */
pcad_status pcad_batch_sync(pcad_batch *b);
/* Choose the tiling: tile_rows a multiple of 4 in [4, 64], order 0 (image
 * order), 1 (costliest first) or 2 (wavefront, one launch per 16 sweeps).
 * Results do not depend on it.  Stream-ordered; PCAD_EINVAL otherwise. */
pcad_status pcad_batch_set_tiling(pcad_batch *b, int tile_rows, int order);
/* Sweeps per captured slice: 8, 16 (the default) or 32; a wavefront slice
 * is one persistent launch, so this is the number of sweeps per launch.
 * sweeps > 0 sets it, 0 keeps it; *current (may be NULL) receives the value
 * in use.  The autotuner chooses it together with the tiling (wavefront
 * orders try 8, 16 and 32, per-sweep orders 16).  Results do not depend on
 * it.  PCAD_EINVAL for other values. */
pcad_status pcad_batch_slice(pcad_batch *b, int sweeps, int *current);
/* Current sample / posterior mean of chain i (host memory, as for a chain). */
pcad_status pcad_batch_read_sample(pcad_batch *b, int i, uint8_t *host_out, int out_pitch);
pcad_status pcad_batch_read_mean(pcad_batch *b, int i, float *host_out);
/* Sweeps done, chosen tiling (tile rows, order 0/1/2 as for
 * pcad_batch_set_tiling), per-sweep grid size, autotuner's best slice time
 * (ms per 16 sweeps) and the FP64 re-draw count summed over chains. */
pcad_status pcad_batch_info(pcad_batch *b, uint64_t *t, int *tile_rows, int *lpt_order,
                            int *grid, float *tune_ms, uint64_t *fp64_draws);
void pcad_batch_destroy(pcad_batch *b);

/* -------------------------------------------------------------- server
 * Continuous batching of denoising requests (no counterpart in the paper:
 * a serving loop around the sweep of Section 5.2).  Submitted requests are
 * admitted into slots as slots free up and their device memory fits the HBM
 * budget; every pcad_server_step chooses the requests to run, advances them
 * by one slice of sweeps in shared launches, and retires the requests whose
 * sweep budget is spent (their sample and posterior mean are copied to host
 * memory held by the server until polled).  State and sweep counters stay
 * on the device between slices; a request's results do not depend on what
 * else was running, nor on the policy below. */
typedef struct pcad_server pcad_server;

/* Scheduling policy.  PCAD_SERVE_FIFO: admit first come first served and
 * run every admitted request in every slice (the GPU is shared among all
 * of them).  PCAD_SERVE_SRPT (the default): shortest remaining work first
 * -- each step orders queued and admitted requests by estimated remaining
 * GPU time (sites x sweeps left x a per-label-count cost) minus `aging` x
 * the seconds since submission, and runs the shortest ones until they hold
 * the fill target of sites (pcad_server_set_limits; by default two waves
 * of 4 x 32-site tiles); admitted requests outside that set keep their
 * device state and pause.  Default aging 0.2.  PCAD_EINVAL for an unknown
 * policy or aging outside [0, 1e6].  Takes effect at the next step. */
typedef enum { PCAD_SERVE_FIFO = 0, PCAD_SERVE_SRPT = 1 } pcad_serve_policy;

pcad_status pcad_server_create(int max_slots, size_t hbm_budget_bytes, void *cuda_stream,
                               pcad_server **out);
/* How much work runs at once.  FIFO: a queued request waits while the
 * admitted requests hold max_active_sites sites or more (its own included),
 * unless none is admitted; 0 (the default) admits whenever a slot and the
 * HBM budget allow.  SRPT: the run set is filled up to max_active_sites
 * sites (0: the default fill target).  Takes effect at the next step. */
pcad_status pcad_server_set_limits(pcad_server *sv, size_t max_active_sites);
pcad_status pcad_server_set_policy(pcad_server *sv, int policy, double aging);
/* Queue a request for nsweeps sweeps (job->g_host is copied).  *id is its handle. */
pcad_status pcad_server_submit(pcad_server *sv, const pcad_job *job, int nsweeps, uint64_t *id);
/* Admit, run one slice of slice_sweeps (1..16) sweeps of every request in
 * the run set in one wavefront launch (tiles of 4 or 8 rows x 32 sites; a
 * tile's sweep starts when its 3 x 3 neighbourhood finished the previous
 * sweep), retire finished requests.  When the slice retires a request it
 * returns after the slice is done (the outputs are then in host memory);
 * otherwise it returns once the previous slice is done, so the host
 * prepares the next slice while this one runs.  PCAD_ETIMEOUT: a bounded
 * wait inside the launch gave up (the results of that slice are invalid). */
pcad_status pcad_server_step(pcad_server *sv, int slice_sweeps, int *n_active, int *n_pending,
                             int *n_finished);
/* *state: 0 queued, 1 running, 2 done.  When done and an output pointer is
 * given, copies the sample (H x W bytes) and mean (H x W floats) and
 * forgets the request. */
pcad_status pcad_server_poll(pcad_server *sv, uint64_t id, int *state, uint8_t *sample_out,
                             float *mean_out);
pcad_status pcad_server_info(pcad_server *sv, size_t *hbm_used, uint64_t *slices,
                             uint64_t *fp64_draws);
void pcad_server_destroy(pcad_server *sv);

/* ------------------------------------------------------------ row bands
 * One image split into nbands bands of whole rows, each run by its own chain
 * (on its own stream, and on devices[b] when devices is not NULL; NULL puts
 * every band on the current device).  The lazy PCA updates every site from
 * the previous state only (Section 3, Eq. general_pca_definition), so a
 * label after k sweeps depends only on sites within k rows: band b owns rows
 * [floor(b H / nbands), floor((b + 1) H / nbands)) and its chain holds
 * `halo` extra rows on each inner side; after every block of `halo` sweeps
 * each band copies its neighbours' owned rows into its halo rows (device to
 * device, peer copies across devices).  Draws are keyed by the global row,
 * so the sample and posterior mean equal the whole-image chain's bit for
 * bit.  Limits: 1 <= nbands <= 64, 1 <= halo <= 64, every band owns at
 * least `halo` rows, lazy PCA only (PCAD_EINVAL otherwise).  g_host is
 * copied; the image size limits of pcad_chain_create apply per band. */
typedef struct pcad_bands pcad_bands;
pcad_status pcad_bands_create(const uint8_t *g_host, int H, int W, int g_pitch,
                              const pcad_model *m, uint64_t seed, uint32_t chain_id, int burn_in,
                              int nbands, int halo, const int *devices, pcad_bands **out);
/* nsweeps sweeps of every band, in blocks of `halo` with an exchange after
 * each (asynchronous on the bands' streams). */
pcad_status pcad_bands_run(pcad_bands *b, int nsweeps);
/* Wait for every band; PCAD_ETIMEOUT if a band's bounded wait gave up. */
pcad_status pcad_bands_sync(pcad_bands *b);
/* The whole image's sample (H rows of W bytes, pitch out_pitch) and posterior
 * mean (H x W floats) assembled from the bands' owned rows (synchronous). */
pcad_status pcad_bands_read_sample(pcad_bands *b, uint8_t *host_out, int out_pitch);
pcad_status pcad_bands_read_mean(pcad_bands *b, float *host_out);
/* Band `band`'s owned rows [*own_row0, *own_row1), its chain's rows
 * [*buf_row0, *buf_row1) and the sweeps run so far (any pointer may be NULL). */
pcad_status pcad_bands_info(const pcad_bands *b, int band, int *own_row0, int *own_row1,
                            int *buf_row0, int *buf_row1, uint64_t *t);
void pcad_bands_destroy(pcad_bands *b);

/* Allocation-free lazy-PCA run (no counterpart in the paper: a library
 * convenience).  For callers that must not allocate device memory: the GPU
 * memory is already owned by another pool, or the calling loop cannot afford
 * cudaMalloc / cudaFree, which may synchronise the whole device.
 * Runs nsweeps PCA sweeps from the device observation g_dev (H x W labels,
 * row pitch `pitch` bytes) with the chain semantics of pcad_chain_create +
 * pcad_chain_run, and writes the final sample to sample_dev (same pitch) and
 * the posterior mean (label units, zeros when nsweeps <= burn_in) to mean_dev
 * (H x W contiguous floats; also used as the accumulator).  Asynchronous on
 * cuda_stream.  The second label plane, the model tables and the counters
 * live in one 8 MiB array in the library's own device memory, held by every
 * GPU that loads the library until the process exits: pitch * H may not
 * exceed 8,355,840 bytes, m->sampler must be PCAD_SAMPLER_PCA and the
 * inertia price the L0 one (inertia_norm 0), and g_dev, sample_dev and
 * mean_dev must not overlap (PCAD_EINVAL otherwise).  All calls share that
 * array, so calls whose GPU work overlaps (unordered streams) race.  The
 * first call on a device looks up the array's address with that device
 * current and keeps it with the device's context; a call that finds another
 * context current (after cudaDeviceReset, say) looks it up again.  Make the
 * first call on a device before any stream capture.  The model tables travel
 * as a kernel parameter, so the call reads no host memory after it returns.
 * No allocation of any kind is made. */
pcad_status pcad_pca_run_noalloc(const uint8_t *g_dev, int H, int W, int pitch,
                                 const pcad_model *m, uint64_t seed, uint32_t chain_id,
                                 int nsweeps, int burn_in, uint8_t *sample_dev,
                                 float *mean_dev, void *cuda_stream);

/* Static description of a status code. */
const char *pcad_status_str(pcad_status s);

/* Message describing the last failure on the calling thread ("" if none). */
const char *pcad_last_error(void);

/* Library version string. */
const char *pcad_version(void);

/* The FP32 constants behind the certified draw of model m from its
 * conditional (Section 5.2, Eq. posterior_pca_transition_matrix; host only,
 * no device work; the paper fixes no precision, so these are this library's):
 * out[0] alpha and out[1] gam, the data and prior exponent coefficients in
 * base 2 (alpha = -log2(e) / (2 sigma^2) for Gaussian noise, -log2(e)
 * ln((1 - p) / p) for flips, 0 without a likelihood; gam = -c log2(e)); out[2] eta, the
 * CUDA-core kernels' CDF margin (a draw is re-done in FP64 when u Z lies
 * within eta Z of the chosen label's CDF interval; the constant margin,
 * used by the Lp prices, the two-label draw and gam > 0); out[3..7] cb, hb,
 * kb0, kb1, kbr: the tensor-core window weights are 2^(alpha (g - s)^2 +
 * mu Pb + cb) (mu = -gam, Pb the tent sum), and the tensor-core sweep and
 * the CUDA-core sweeps with gam <= 0 take the per-site margin
 * eta = kb1 (hb - log2 Z) + kb0 + kbr delta / Z (Z the site's total with the
 * inertia weight delta).  out must hold n >= PCAD_N_MARGINS doubles.
 * PCAD_EINVAL for an invalid model or buffer. */
#define PCAD_N_MARGINS 8
pcad_status pcad_model_margins(const pcad_model *m, double *out, int n);

#ifdef __cplusplus
}
#endif

#endif /* PCADEN_H */
