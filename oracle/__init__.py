"""FP64 CPU oracle for the lazy-PCA denoising sampler -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

Contents
  * ``pcad_oracle.c`` (compiled on demand with gcc, FP64, no FMA contraction):
    Philox4x32-10, the per-site conditional and inverse-CDF draw, lazy-PCA
    and single-site Gibbs sweeps (row-major, column-major or colour order),
    chain runner with the posterior-mean accumulator.
  * ``exact``: exhaustive enumeration of the posterior (Eq.
    mrf_gauss_noise_posterior_distribution) and of the PCA stationary measure
    (Eq. symm_ham_pca_stationary_measure with the symmetric lifted pair
    Hamiltonian), PCA transition matrices, the J = 0 closed forms.
  * ``metrics``: PSNR and SSIM as defined in Section 6.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcad_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

POTTS, TRUNC_LINEAR = 0, 1
GAUSS, FLIP, NONE = 0, 1, 2
PCA, GIBBS = 0, 1
ORDER_ROW, ORDER_COL, ORDER_COLOUR = 0, 1, 2


class OrcModel(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("nbhd", ctypes.c_int), ("pair", ctypes.c_int),
                ("pair_T", ctypes.c_int), ("noise", ctypes.c_int), ("inertia_norm", ctypes.c_int),
                ("pair_coef", ctypes.c_double), ("sigma", ctypes.c_double),
                ("flip_p", ctypes.c_double), ("inertia", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            mp = ctypes.POINTER(OrcModel)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_site_probs.argtypes = [mp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                         ctypes.c_double, dp]
            L.orc_site_probs.restype = None
            L.orc_site_draw.argtypes = [mp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ip]
            L.orc_site_draw.restype = ctypes.c_int
            L.orc_pca_sweep.argtypes = [mp, ctypes.c_int, ctypes.c_int, u8p, u8p, u8p,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u8p]
            L.orc_pca_sweep.restype = ctypes.c_long
            L.orc_pca_sites.argtypes = [mp, ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_long,
                                        i32p, i32p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, u8p, u8p]
            L.orc_pca_sites.restype = ctypes.c_long
            L.orc_gibbs_sweep.argtypes = [mp, ctypes.c_int, ctypes.c_int, u8p, u8p,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int, u8p]
            L.orc_gibbs_sweep.restype = ctypes.c_long
            L.orc_run_chain.argtypes = [mp, ctypes.c_int, ctypes.c_int, u8p, u8p, dp,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_run_chain.restype = ctypes.c_long
            L.orc_state_histogram.argtypes = [mp, ctypes.c_int, ctypes.c_int, u8p, u8p,
                                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, dp]
            L.orc_state_histogram.restype = ctypes.c_long
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def _f32(x) -> float:
    """Parameters cross the library boundary as FP32; the oracle uses the same
    FP32-rounded values, widened to FP64."""
    return float(np.float32(x))


def model_struct(m) -> OrcModel:
    """Build the C model struct from a pcad_inputs.Model (or a dict)."""
    d = m.as_dict() if hasattr(m, "as_dict") else dict(m)
    s = OrcModel()
    s.L = int(d["L"]); s.nbhd = int(d.get("nbhd", 4)); s.pair = int(d.get("pair", 1))
    s.pair_T = int(d.get("pair_T", 1)); s.noise = int(d.get("noise", 0))
    s.inertia_norm = int(d.get("inertia_norm", 0))
    s.pair_coef = _f32(d.get("pair_coef", 0.0)); s.sigma = _f32(d.get("sigma", 1.0))
    s.flip_p = _f32(d.get("flip_p", 0.1)); s.inertia = _f32(d.get("inertia", 0.0))
    return s


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(seed, chain, tag, sweep, row, col) -> float:
    return float(lib().orc_uniform(seed, chain, tag, sweep, row, col))


def site_probs(m, g, xi, nbrs, lam):
    ms = model_struct(m)
    nb = (ctypes.c_int * max(len(nbrs), 1))(*[int(v) for v in nbrs])
    p = (ctypes.c_double * ms.L)()
    lib().orc_site_probs(ctypes.byref(ms), int(g), int(xi), nb, len(nbrs), float(lam), p)
    return np.array(p[:], dtype=np.float64)


def site_draw(m, g, xi, nbrs, lam, u):
    ms = model_struct(m)
    nb = (ctypes.c_int * max(len(nbrs), 1))(*[int(v) for v in nbrs])
    near = ctypes.c_int(0)
    k = lib().orc_site_draw(ctypes.byref(ms), int(g), int(xi), nb, len(nbrs), float(lam),
                            float(u), ctypes.byref(near))
    return int(k), bool(near.value)


def pca_sweep(m, g, x, seed, chain, sweep):
    """One lazy-PCA sweep from x; returns (x_next, near_flags)."""
    ms = model_struct(m)
    g, gp = _u8(g)
    x, xp = _u8(x)
    H, W = x.shape
    out = np.empty_like(x)
    near = np.empty_like(x)
    lib().orc_pca_sweep(ctypes.byref(ms), H, W, gp, xp, _u8(out)[1], seed, chain, sweep,
                        _u8(near)[1])
    return out, near


def pca_sites(m, g, x, rows, cols, seed, chain, sweep):
    """Lazy-PCA draws at the listed sites only."""
    ms = model_struct(m)
    g, gp = _u8(g)
    x, xp = _u8(x)
    H, W = x.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    n = rows.size
    out = np.empty(n, dtype=np.uint8)
    near = np.empty(n, dtype=np.uint8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib().orc_pca_sites(ctypes.byref(ms), H, W, gp, xp, n, rows.ctypes.data_as(i32p),
                        cols.ctypes.data_as(i32p), seed, chain, sweep,
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        near.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out, near


def gibbs_sweep(m, g, x, seed, chain, sweep, order=ORDER_COLOUR):
    """One single-site Gibbs sweep; returns (x_next, near_flags)."""
    ms = model_struct(m)
    g, gp = _u8(g)
    x = np.array(x, dtype=np.uint8, copy=True)
    H, W = x.shape
    near = np.zeros_like(x)
    lib().orc_gibbs_sweep(ctypes.byref(ms), H, W, gp, _u8(x)[1], seed, chain, sweep, order,
                          _u8(near)[1])
    return x, near


def run_chain(m, g, nsweeps, burn_in, seed, chain=0, sampler=PCA, order=ORDER_COLOUR,
              x0=None, acc=None, t0=0):
    """Run a chain from x0 (default: the observation g, the initial state of
    the retrieval); returns (x, acc, n_accumulated, n_near)."""
    ms = model_struct(m)
    g, gp = _u8(g)
    x = np.array(g if x0 is None else x0, dtype=np.uint8, copy=True)
    H, W = x.shape
    acc = np.zeros((H, W), dtype=np.float64) if acc is None else np.array(acc, dtype=np.float64)
    n_near = lib().orc_run_chain(ctypes.byref(ms), H, W, gp, _u8(x)[1],
                                 acc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), seed,
                                 chain, t0, nsweeps, burn_in, sampler, order)
    n_acc = max(0, t0 + nsweeps - max(burn_in, t0))
    return x, acc, n_acc, int(n_near)


def state_histogram(m, g, nsweeps, seed, chain=0, sampler=PCA, order=ORDER_COLOUR, x0=None):
    """Visit counts of every state of a tiny lattice (index sum_i x_i L^i)."""
    ms = model_struct(m)
    g, gp = _u8(g)
    x = np.array(g if x0 is None else x0, dtype=np.uint8, copy=True)
    H, W = x.shape
    hist = np.zeros(int(ms.L) ** (H * W), dtype=np.float64)
    rc = lib().orc_state_histogram(ctypes.byref(ms), H, W, gp, _u8(x)[1], seed, chain,
                                   nsweeps, sampler, order,
                                   hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc < 0:
        raise ValueError("lattice too large for a state histogram")
    return hist


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))
