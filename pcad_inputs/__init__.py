"""Seeded synthetic inputs for the PCA denoising sampler.

This module is shared by the FP64 oracle tests, the GPU tests and the
benchmark.  It only *draws* inputs: clean label images, their noisy
observations and per-image parameter tables.  It contains none of the
sampler's arithmetic (no energies, no conditionals, no random numbers the
sampler consumes -- those come from the counter-based Philox stream that
each side implements on its own).

The paper's test images are not public (Section "Availability of data"), so
every workload here is synthetic: piecewise-constant / piecewise-smooth
scenes of the kind the paper uses (uniform regions, few sharp edges,
Section 6), degraded by flip noise (binary) or additive Gaussian noise that
is rounded to the nearest grey level (Section 6, degradation recipe).

All generators use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Model",
    "shapes_binary",
    "flip_noise",
    "greyscale_scene",
    "gaussian_noise",
    "binary_64",
    "greyscale_512",
    "large_image",
    "batched_jobs",
    "serving_requests",
    "random_lattice",
]

PAIR_POTTS = 0
PAIR_TRUNC_LINEAR = 1
NOISE_GAUSS = 0
NOISE_FLIP = 1
NOISE_NONE = 2   # prior only (synthetic MRF images)
SAMPLER_PCA = 0
SAMPLER_GIBBS = 1


@dataclass
class Model:
    """Model parameters in the units the sampler consumes (label units).

    pair_coef is the reward c_P = 2*beta*J for the Potts prior or the slope
    c_T of the truncated-linear prior; sigma is in label units; inertia is
    lambda = beta*q.
    """

    L: int
    nbhd: int = 4
    pair: int = PAIR_TRUNC_LINEAR
    pair_coef: float = 0.05
    pair_T: int = 30
    noise: int = NOISE_GAUSS
    sigma: float = 20.0
    flip_p: float = 0.1
    inertia: float = 2.0
    sampler: int = SAMPLER_PCA
    inertia_norm: int = 0   # 0: lambda 1{s != x_i}; 1, 2: lambda (|s - x_i| / (L-1))^p

    def as_dict(self) -> dict:
        return dict(L=self.L, nbhd=self.nbhd, pair=self.pair,
                    pair_coef=self.pair_coef, pair_T=self.pair_T,
                    noise=self.noise, sigma=self.sigma, flip_p=self.flip_p,
                    inertia=self.inertia, sampler=self.sampler,
                    inertia_norm=self.inertia_norm)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _paint_shapes(rng, img, n_shapes, value_fn, side_lo, side_hi):
    """Paint n axis-aligned rectangles or disks, in order, onto img."""
    H, W = img.shape
    for _ in range(n_shapes):
        kind = rng.integers(0, 2)            # 0 = rectangle, 1 = disk
        cr = int(rng.integers(0, H))
        cc = int(rng.integers(0, W))
        hr = int(rng.integers(side_lo, side_hi + 1))
        hc = int(rng.integers(side_lo, side_hi + 1))
        val = value_fn(rng)
        r0, r1 = max(cr - hr, 0), min(cr + hr + 1, H)
        if kind == 0:
            c0, c1 = max(cc - hc, 0), min(cc + hc + 1, W)
            img[r0:r1, c0:c1] = val
        else:
            c0, c1 = max(cc - hr, 0), min(cc + hr + 1, W)
            if r1 <= r0 or c1 <= c0:
                continue
            rr = np.arange(r0, r1)[:, None] - cr
            cc_ = np.arange(c0, c1)[None, :] - cc
            mask = rr * rr + cc_ * cc_ <= hr * hr
            sub = img[r0:r1, c0:c1]
            sub[mask] = val
    return img


def shapes_binary(seed: int, H: int, W: int, n_shapes: int = 8) -> np.ndarray:
    """Binary scene: shapes painted with label 0/1 (spin -1/+1) over label 0."""
    rng = _rng(seed)
    img = np.zeros((H, W), dtype=np.uint8)
    side = min(H, W)
    lo, hi = max(side // 16, 1), max(side // 4, 1)
    return _paint_shapes(rng, img, n_shapes, lambda r: np.uint8(r.integers(0, 2)), lo, hi)


def flip_noise(seed: int, clean: np.ndarray, p: float) -> np.ndarray:
    """Binary-symmetric channel: each label flipped independently with prob. p."""
    rng = _rng(seed)
    flips = rng.random(clean.shape) < p
    return (clean ^ flips.astype(np.uint8)).astype(np.uint8)


def greyscale_scene(seed: int, H: int, W: int, L: int, n_shapes: int = 20) -> np.ndarray:
    """Smooth gradient (linear ramp + low-frequency sinusoid) plus shapes.

    Intensities live on the label scale [0, L-1]; shapes take a value
    uniform on [0, L-1]; the result is rounded to the nearest label.
    """
    rng = _rng(seed)
    top = float(L - 1)
    lo, hi = np.sort(rng.uniform(0.0, top, 2))
    theta = rng.uniform(0.0, 2 * math.pi)
    amp = rng.uniform(0.05, 0.15) * top
    fr, fc = rng.uniform(0.5, 2.0, 2)
    phase = rng.uniform(0.0, 2 * math.pi)
    r = (np.arange(H, dtype=np.float32) / max(H - 1, 1))[:, None]
    c = (np.arange(W, dtype=np.float32) / max(W - 1, 1))[None, :]
    ramp = math.cos(theta) * r + math.sin(theta) * c
    rmin, rmax = float(ramp.min()), float(ramp.max())
    ramp = (ramp - rmin) / max(rmax - rmin, 1e-12)
    img = (lo + (hi - lo) * ramp).astype(np.float32)
    img += (amp * np.sin(2 * math.pi * (fr * r + fc * c) + phase)).astype(np.float32)
    side = min(H, W)
    lo_s, hi_s = max(side // 16, 1), max(side // 4, 1)
    _paint_shapes(rng, img, n_shapes, lambda g: np.float32(g.uniform(0.0, top)), lo_s, hi_s)
    np.clip(img, 0.0, top, out=img)
    return np.rint(img).astype(np.uint8)


def gaussian_noise(seed: int, clean: np.ndarray, sigma: float, L: int) -> np.ndarray:
    """Add N(0, sigma^2) per pixel (label units), clip to [0, L-1], round."""
    rng = _rng(seed)
    noise = rng.standard_normal(clean.shape, dtype=np.float32) * np.float32(sigma)
    out = clean.astype(np.float32) + noise
    np.clip(out, 0.0, float(L - 1), out=out)
    return np.rint(out).astype(np.uint8)


# ---------------------------------------------------------------- workloads

def binary_64(seed: int = 1, side: int = 64, p: float = 0.1):
    """Binary side x side scene, 8 shapes, flip noise p; Ising J=0.6 (c_P = 2J),
    q = 1.0, 4-neighbourhood, free boundary."""
    clean = shapes_binary(seed, side, side, n_shapes=8)
    noisy = flip_noise(seed + 1_000_003, clean, p)
    model = Model(L=2, nbhd=4, pair=PAIR_POTTS, pair_coef=1.2, pair_T=1,
                  noise=NOISE_FLIP, sigma=1.0, flip_p=p, inertia=1.0)
    return clean, noisy, model


def greyscale_512(seed: int = 2, side: int = 512, L: int = 256, sigma: float = 20.0):
    """Greyscale scene with L labels, Gaussian noise sigma (label units),
    truncated-linear prior beta=0.05, T=30, q=2.0, 4-neighbourhood."""
    clean = greyscale_scene(seed, side, side, L, n_shapes=20)
    noisy = gaussian_noise(seed + 1_000_003, clean, sigma, L)
    model = Model(L=L, nbhd=4, pair=PAIR_TRUNC_LINEAR, pair_coef=0.05, pair_T=30,
                  noise=NOISE_GAUSS, sigma=sigma, flip_p=0.0, inertia=2.0)
    return clean, noisy, model


def large_image(seed: int = 3, side: int = 8192, L: int = 16):
    """Large single image: L=16 with sigma=1.0 or L=256 with sigma=25 (label
    units); same generator and prior as greyscale_512."""
    sigma = 1.0 if L <= 16 else 25.0
    return greyscale_512(seed=seed, side=side, L=L, sigma=sigma)


def _binary_from_scene(seed, H, W):
    return shapes_binary(seed, H, W, n_shapes=max(8, (H * W) // 16384))


@dataclass
class Job:
    """One image of a batch with its model, seed and chain count."""
    clean: np.ndarray
    noisy: np.ndarray
    model: Model
    seed: int
    chains: int
    sweeps: int
    burn_in: int
    meta: dict = field(default_factory=dict)


def _image_params(rng, L):
    """Per-image prior/inertia table (label units)."""
    if L == 2:
        J = float(rng.uniform(0.4, 0.8))
        q = float(rng.uniform(0.5, 1.5))
        return dict(pair=PAIR_POTTS, pair_coef=2.0 * J, pair_T=1, inertia=q)
    beta255 = float(rng.uniform(0.03, 0.08))
    q = float(rng.uniform(1.0, 3.0))
    scale = 255.0 / (L - 1)
    T = max(1, int(round(30.0 / scale)))
    return dict(pair=PAIR_TRUNC_LINEAR, pair_coef=beta255 * scale, pair_T=T, inertia=q)


def _degraded_image(seed, H, W, L, sigma255):
    """Scene at L levels; Gaussian sigma given on the 0..255 scale (L > 2) or
    as flip probability p = sigma/200 (L = 2)."""
    if L == 2:
        clean = _binary_from_scene(seed, H, W)
        p = sigma255 / 200.0
        return clean, flip_noise(seed + 7, clean, p), dict(noise=NOISE_FLIP, flip_p=p, sigma=1.0)
    clean = greyscale_scene(seed, H, W, L, n_shapes=20)
    s_lab = sigma255 * (L - 1) / 255.0
    return clean, gaussian_noise(seed + 7, clean, s_lab, L), dict(noise=NOISE_GAUSS, sigma=s_lab, flip_p=0.0)


def batched_jobs(seed: int = 4, n_images: int = 128, chains: int = 4,
                 side_lo: int = 64, side_hi: int = 2048, sweeps: int = 200,
                 burn_in: int = 50, labels=(2, 16, 256)):
    """Uneven batch: short side log-uniform in [side_lo, side_hi], aspect
    ratio uniform in [1, 3] (random orientation), L drawn from `labels`,
    sigma uniform in [5, 40] (0..255 scale), per-image prior/inertia table."""
    rng = _rng(seed)
    jobs = []
    for i in range(n_images):
        s = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        a = float(rng.uniform(1.0, 3.0))
        long_ = int(round(s * a))
        if rng.integers(0, 2):
            H, W = s, long_
        else:
            H, W = long_, s
        L = int(labels[int(rng.integers(0, len(labels)))])
        sigma255 = float(rng.uniform(5.0, 40.0))
        params = _image_params(rng, L)
        clean, noisy, noise = _degraded_image(seed * 100_003 + i, H, W, L, sigma255)
        model = Model(L=L, nbhd=4, **params, **noise)
        jobs.append(Job(clean=clean, noisy=noisy, model=model, seed=1000 + i,
                        chains=chains, sweeps=sweeps, burn_in=burn_in,
                        meta=dict(sigma255=sigma255)))
    return jobs


def serving_requests(seed: int, rate: float, n: int, side_lo: int = 128,
                     side_hi: int = 2048, labels=(16, 256),
                     sweeps_lo: int = 300, sweeps_hi: int = 3000):
    """Open-loop Poisson arrivals (rate per second) of denoising requests:
    square side log-uniform, L from `labels`, sigma uniform [5, 40] on the
    0..255 scale, sweep budget uniform in [sweeps_lo, sweeps_hi], burn-in a
    quarter of the budget, one chain each."""
    rng = _rng(seed)
    t = 0.0
    reqs = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        s = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        L = int(labels[int(rng.integers(0, len(labels)))])
        sigma255 = float(rng.uniform(5.0, 40.0))
        params = _image_params(rng, L)
        sweeps = int(rng.integers(sweeps_lo, sweeps_hi + 1))
        clean, noisy, noise = _degraded_image(seed * 1_000_003 + i, s, s, L, sigma255)
        model = Model(L=L, nbhd=4, **params, **noise)
        reqs.append(dict(arrival=t, job=Job(clean=clean, noisy=noisy, model=model,
                                            seed=5000 + i, chains=1, sweeps=sweeps,
                                            burn_in=sweeps // 4,
                                            meta=dict(sigma255=sigma255))))
    return reqs


def random_lattice(seed: int, H: int, W: int, L: int) -> np.ndarray:
    """Uniformly random labels (used for tiny exhaustive-enumeration cases)."""
    rng = _rng(seed)
    return rng.integers(0, L, size=(H, W), dtype=np.int64).astype(np.uint8)
