"""The paper's restoration protocol (Section 6) on top of the C ABI.

* Prior: Potts with the 8-neighbourhood, coupling J; the per-edge reward of
  the single-site conditional is c_P = 2 beta J (Eq.
  gibbs_sampler_elementary_step).  Likelihood: Gaussian noise with sigma
  given in intensity units on levels k / (L - 1), i.e. sigma (L - 1) in
  label units; the observation is rounded to the nearest level.
* Simulated annealing: beta starts at 1.25 and rises by 0.25 every 250
  sweeps, over 1000 sweeps; the inertia lambda = beta q rises with it, the
  likelihood is not rescaled.  The estimate is the last sample.
* Gibbs sampling visits the sites in 4 colour classes (8-neighbourhood);
  the lazy PCA updates every site at once.
* Synthetic MRF test images: Gibbs sampling of the prior alone (no
  likelihood) with J = 1/3 from uniformly random levels.
* The q grid: 14 values 0.06 ... 0.71 with several runs each, as one batch
  of chains per image (the q-sensitivity experiment).

Every sweep runs in the library's kernels; this module only builds the
models and the schedules and calls the C entry points.
"""
from __future__ import annotations

import numpy as np

from ._capi import (NOISE_GAUSS, NOISE_NONE, PAIR_POTTS, SAMPLER_GIBBS_CB, SAMPLER_PCA, Chain,
                    pcad_batch_create, pcad_batch_destroy, pcad_batch_read_sample, pcad_batch_run,
                    pcad_batch_set_model, pcad_batch_sync, pcad_metrics)

Q_GRID = tuple(round(0.06 + 0.05 * k, 2) for k in range(14))   # 0.06 ... 0.71


def betas(beta0: float = 1.25, dbeta: float = 0.25, stages: int = 4):
    """Inverse temperatures of the annealing stages."""
    return [beta0 + dbeta * k for k in range(stages)]


def model(L: int, J: float, beta: float, q: float, sigma: float, nbhd: int = 8,
          sampler: int = SAMPLER_PCA) -> dict:
    """Potts prior c_P = 2 beta J, Gaussian likelihood sigma (intensity units),
    inertia lambda = beta q."""
    return dict(L=L, nbhd=nbhd, pair=PAIR_POTTS, pair_coef=2.0 * beta * J, pair_T=1,
                noise=NOISE_GAUSS, sigma=sigma * (L - 1), flip_p=0.1, inertia=beta * q,
                sampler=sampler)


def schedule(L: int, J: float, q: float, sigma: float, nbhd: int = 8, sampler: int = SAMPLER_PCA,
             beta0: float = 1.25, dbeta: float = 0.25, stages: int = 4, stage_sweeps: int = 250):
    """(models, sweeps) of the annealed run."""
    ms = [model(L, J, b, q, sigma, nbhd, sampler) for b in betas(beta0, dbeta, stages)]
    return ms, [stage_sweeps] * stages


def restore(g: np.ndarray, L: int, J: float, q: float, sigma: float, seed: int,
            chain_id: int = 0, sampler: int = SAMPLER_PCA, nbhd: int = 8, stream=None,
            **sched) -> np.ndarray:
    """Annealed run from x0 = g; returns the last sample."""
    ms, sw = schedule(L, J, q, sigma, nbhd, sampler, **sched)
    with Chain(g, ms[0], seed=seed, chain_id=chain_id, burn_in=sum(sw), stream=stream) as ch:
        ch.run_schedule(ms, sw)
        return ch.sample()


def mrf_image(init: np.ndarray, L: int, J: float = 1.0 / 3.0, beta: float = 1.5,
              sweeps: int = 200, seed: int = 0, nbhd: int = 8, stream=None) -> np.ndarray:
    """A sample of the Potts prior: `sweeps` Gibbs sweeps (no likelihood,
    c_P = 2 beta J) started from the labels `init`."""
    m = dict(L=L, nbhd=nbhd, pair=PAIR_POTTS, pair_coef=2.0 * beta * J, pair_T=1,
             noise=NOISE_NONE, sigma=1.0, flip_p=0.1, inertia=0.0, sampler=SAMPLER_GIBBS_CB)
    with Chain(init, m, seed=seed, chain_id=0, burn_in=sweeps, stream=stream) as ch:
        ch.run(sweeps)
        return ch.sample()


def metrics(est_labels: np.ndarray, clean: np.ndarray, L: int):
    """(PSNR dB, SSIM) of a label image against the clean one (Section 6)."""
    return pcad_metrics(est_labels.astype(np.float32), clean, L)


def q_grid(g: np.ndarray, clean: np.ndarray, L: int, J: float, sigma: float, seed: int,
           qs=Q_GRID, runs: int = 10, nbhd: int = 8, stream=None, return_samples: bool = False,
           **sched):
    """Annealed lazy-PCA runs for every q in qs, `runs` chains each, as one
    batched launch per sweep; returns {q: [(psnr, ssim) per run]} (and
    {q: [last sample per run]} with return_samples)."""
    jobs_q = [q for q in qs for _ in range(runs)]
    ms0 = [schedule(L, J, q, sigma, nbhd, SAMPLER_PCA, **sched) for q in qs]
    total = sum(ms0[0][1])
    jobs = [(g, ms0[k // runs][0][0], seed, k, total) for k in range(len(jobs_q))]
    h = pcad_batch_create(jobs, autotune=False, stream=stream)
    try:
        n_stages = len(ms0[0][0])
        for st in range(n_stages):
            if st > 0:
                for k in range(len(jobs_q)):
                    pcad_batch_set_model(h, k, ms0[k // runs][0][st])
            pcad_batch_run(h, ms0[0][1][st])
        pcad_batch_sync(h)
        H, W = g.shape
        out = {q: [] for q in qs}
        samples = {q: [] for q in qs}
        for k, q in enumerate(jobs_q):
            x = pcad_batch_read_sample(h, k, H, W)
            out[q].append(metrics(x, clean, L))
            if return_samples:
                samples[q].append(x)
        return (out, samples) if return_samples else out
    finally:
        pcad_batch_destroy(h)


def concavity(values) -> dict:
    """Second differences of a curve sampled on an even grid: the number of
    positive ones (0 for a concave curve) and the largest."""
    v = np.asarray(values, dtype=np.float64)
    d2 = v[2:] - 2.0 * v[1:-1] + v[:-2]
    return dict(positive=int((d2 > 0).sum()), max=float(d2.max()) if d2.size else 0.0,
                n=int(d2.size))
