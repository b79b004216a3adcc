"""ctypes binding of libpcaden (include/pcaden.h): argument marshalling only.

Every function here has the name of the C entry point it calls and raises
PcadError on a non-zero status.  All computation happens in the library's
CUDA kernels; there is no fallback path.  Device pointers and CUDA streams
may come from PyTorch (``tensor.data_ptr()``, ``stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PAIR_POTTS, PAIR_TRUNC_LINEAR = 0, 1
NOISE_GAUSS, NOISE_FLIP, NOISE_NONE = 0, 1, 2
SAMPLER_PCA, SAMPLER_GIBBS_CB = 0, 1


class PcadError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: status {status} ({_status_name(status)}): {msg}")
        self.status = status


def _status_name(s: int) -> str:
    return {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE"}.get(s, "?")


class PcadModel(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("nbhd", ctypes.c_int), ("pair", ctypes.c_int),
                ("pair_coef", ctypes.c_float), ("pair_T", ctypes.c_int),
                ("noise", ctypes.c_int), ("sigma", ctypes.c_float),
                ("flip_p", ctypes.c_float), ("inertia", ctypes.c_float),
                ("sampler", ctypes.c_int), ("inertia_norm", ctypes.c_int)]


class PcadJob(ctypes.Structure):
    _fields_ = [("g_host", ctypes.POINTER(ctypes.c_uint8)), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("g_pitch", ctypes.c_int), ("model", PcadModel),
                ("seed", ctypes.c_uint64), ("chain_id", ctypes.c_uint32),
                ("burn_in", ctypes.c_int)]


def as_model(m, sampler=None) -> PcadModel:
    """PcadModel from a PcadModel, a dict or any object with the same fields."""
    if isinstance(m, PcadModel):
        out = PcadModel.from_buffer_copy(m)
    else:
        d = m if isinstance(m, dict) else {f: getattr(m, f) for f, _ in PcadModel._fields_
                                           if hasattr(m, f)}
        out = PcadModel(L=int(d["L"]), nbhd=int(d.get("nbhd", 4)), pair=int(d.get("pair", 1)),
                        pair_coef=float(d.get("pair_coef", 0.0)), pair_T=int(d.get("pair_T", 1)),
                        noise=int(d.get("noise", 0)), sigma=float(d.get("sigma", 1.0)),
                        flip_p=float(d.get("flip_p", 0.1)), inertia=float(d.get("inertia", 0.0)),
                        sampler=int(d.get("sampler", 0)),
                        inertia_norm=int(d.get("inertia_norm", 0)))
    if sampler is not None:
        out.sampler = int(sampler)
    return out


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libpcaden.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libpcaden.so is missing and could not be built")
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    vp, u8p, fp, dp = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8),
                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double))
    u64p = ctypes.POINTER(ctypes.c_uint64)
    mp = ctypes.POINTER(PcadModel)
    sig = {
        "pcad_chain_create": [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, mp, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_int, vp, ctypes.POINTER(vp)],
        "pcad_chain_create_dev": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, mp,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, vp,
                                  ctypes.POINTER(vp)],
        "pcad_chain_run": [vp, ctypes.c_int],
        "pcad_model_margins": [mp, dp, ctypes.c_int],
        "pcad_chain_sync": [vp],
        "pcad_chain_reset": [vp],
        "pcad_chain_set_blocking": [vp, ctypes.c_int],
        "pcad_chain_set_kernel": [vp, ctypes.c_int],
        "pcad_chain_set_wait_limit": [vp, ctypes.c_double],
        "pcad_chain_set_row_offset": [vp, ctypes.c_int],
        "pcad_chain_write_rows_dev": [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int],
        "pcad_bands_create": [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, mp, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp)],
        "pcad_bands_run": [vp, ctypes.c_int],
        "pcad_bands_sync": [vp],
        "pcad_bands_read_sample": [vp, u8p, ctypes.c_int],
        "pcad_bands_read_mean": [vp, fp],
        "pcad_bands_info": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), u64p],
        "pcad_chain_inject_stall": [vp, ctypes.c_int],
        "pcad_chain_kernel_in_use": [vp, ctypes.POINTER(ctypes.c_int)],
        "pcad_chain_energy": [vp, dp, u64p, u64p],
        "pcad_chain_set_model": [vp, mp],
        "pcad_chain_run_schedule": [vp, mp, ctypes.POINTER(ctypes.c_int), ctypes.c_int],
        "pcad_batch_set_model": [vp, ctypes.c_int, mp],
        "pcad_chain_track_energy": [vp, ctypes.c_int],
        "pcad_chain_read_energies": [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "pcad_chain_read_min_state": [vp, u8p, ctypes.c_int, dp, u64p],
        "pcad_chain_read_sample": [vp, u8p, ctypes.c_int],
        "pcad_chain_read_sample_dev": [vp, vp, ctypes.c_int],
        "pcad_chain_read_mean": [vp, fp],
        "pcad_chain_write_sample": [vp, u8p, ctypes.c_int],
        "pcad_chain_sweeps": [vp, u64p, u64p],
        "pcad_chain_stats": [vp, u64p],
        "pcad_chain_metrics": [vp, u8p, ctypes.c_int, ctypes.c_int, dp, dp],
        "pcad_metrics": [fp, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp],
        "pcad_chain_export": [vp, vp, ctypes.POINTER(ctypes.c_size_t)],
        "pcad_chain_import": [vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pcad_batch_create": [ctypes.POINTER(PcadJob), ctypes.c_int, ctypes.c_int, vp,
                              ctypes.POINTER(vp)],
        "pcad_batch_run": [vp, ctypes.c_int],
        "pcad_batch_reset": [vp],
        "pcad_batch_sync": [vp],
        "pcad_batch_set_tiling": [vp, ctypes.c_int, ctypes.c_int],
        "pcad_batch_slice": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "pcad_batch_read_sample": [vp, ctypes.c_int, u8p, ctypes.c_int],
        "pcad_batch_read_mean": [vp, ctypes.c_int, fp],
        "pcad_batch_info": [vp, u64p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), u64p],
        "pcad_server_create": [ctypes.c_int, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pcad_server_submit": [vp, ctypes.POINTER(PcadJob), ctypes.c_int, u64p],
        "pcad_server_set_limits": [vp, ctypes.c_size_t],
        "pcad_server_set_policy": [vp, ctypes.c_int, ctypes.c_double],
        "pcad_server_step": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "pcad_server_poll": [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), u8p, fp],
        "pcad_server_info": [vp, ctypes.POINTER(ctypes.c_size_t), u64p, u64p],
        "pcad_pca_run_noalloc": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, mp,
                                 ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                 vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.pcad_chain_destroy.argtypes = [vp]
    L.pcad_chain_destroy.restype = None
    L.pcad_batch_destroy.argtypes = [vp]
    L.pcad_batch_destroy.restype = None
    L.pcad_server_destroy.argtypes = [vp]
    L.pcad_server_destroy.restype = None
    L.pcad_bands_destroy.argtypes = [vp]
    L.pcad_bands_destroy.restype = None
    L.pcad_status_str.argtypes = [ctypes.c_int]
    L.pcad_status_str.restype = ctypes.c_char_p
    L.pcad_last_error.argtypes = []
    L.pcad_last_error.restype = ctypes.c_char_p
    L.pcad_version.argtypes = []
    L.pcad_version.restype = ctypes.c_char_p


def _check(name: str, status: int):
    if status != 0:
        raise PcadError(name, status, lib().pcad_last_error().decode(errors="replace"))


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(int(s.cuda_stream))
    return ctypes.c_void_p(int(s))


# ------------------------------------------------------------- entry points

def pcad_chain_create(g, model, seed: int, chain_id: int = 0, burn_in: int = 0, stream=None):
    g = _u8(g)
    H, W = g.shape
    h = ctypes.c_void_p()
    m = as_model(model)
    _check("pcad_chain_create",
           lib().pcad_chain_create(g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), H, W, W,
                                   ctypes.byref(m), int(seed), int(chain_id), int(burn_in),
                                   _stream(stream), ctypes.byref(h)))
    return h


def pcad_chain_create_dev(g_dev_ptr: int, H: int, W: int, pitch: int, model, seed: int,
                          chain_id: int = 0, burn_in: int = 0, stream=None):
    h = ctypes.c_void_p()
    m = as_model(model)
    _check("pcad_chain_create_dev",
           lib().pcad_chain_create_dev(ctypes.c_void_p(int(g_dev_ptr)), H, W, pitch,
                                       ctypes.byref(m), int(seed), int(chain_id), int(burn_in),
                                       _stream(stream), ctypes.byref(h)))
    return h


def pcad_chain_run(h, nsweeps: int):
    _check("pcad_chain_run", lib().pcad_chain_run(h, int(nsweeps)))


def pcad_chain_sync(h):
    _check("pcad_chain_sync", lib().pcad_chain_sync(h))


def pcad_chain_reset(h):
    _check("pcad_chain_reset", lib().pcad_chain_reset(h))


def pcad_chain_read_sample(h, H: int, W: int) -> np.ndarray:
    out = np.empty((H, W), dtype=np.uint8)
    _check("pcad_chain_read_sample",
           lib().pcad_chain_read_sample(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W))
    return out


def pcad_chain_read_sample_dev(h, dev_ptr: int, pitch: int):
    _check("pcad_chain_read_sample_dev",
           lib().pcad_chain_read_sample_dev(h, ctypes.c_void_p(int(dev_ptr)), int(pitch)))


def pcad_chain_read_mean(h, H: int, W: int, out=None) -> np.ndarray:
    if out is None:
        out = np.empty((H, W), dtype=np.float32)
    if out.dtype != np.float32 or out.size != H * W or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a contiguous float32 array of H*W elements")
    _check("pcad_chain_read_mean",
           lib().pcad_chain_read_mean(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def pcad_chain_write_sample(h, x):
    x = _u8(x)
    _check("pcad_chain_write_sample",
           lib().pcad_chain_write_sample(h, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                         x.shape[1]))


def pcad_chain_sweeps(h):
    t = ctypes.c_uint64()
    n = ctypes.c_uint64()
    _check("pcad_chain_sweeps", lib().pcad_chain_sweeps(h, ctypes.byref(t), ctypes.byref(n)))
    return int(t.value), int(n.value)


def pcad_chain_stats(h) -> int:
    v = ctypes.c_uint64()
    _check("pcad_chain_stats", lib().pcad_chain_stats(h, ctypes.byref(v)))
    return int(v.value)


def pcad_chain_metrics(h, clean, which: int = 0):
    clean = _u8(clean)
    p = ctypes.c_double()
    s = ctypes.c_double()
    _check("pcad_chain_metrics",
           lib().pcad_chain_metrics(h, clean.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                    clean.shape[1], int(which), ctypes.byref(p), ctypes.byref(s)))
    return float(p.value), float(s.value)


def pcad_metrics(est, clean, L: int):
    est = np.ascontiguousarray(est, dtype=np.float32)
    clean = _u8(clean)
    H, W = clean.shape
    p = ctypes.c_double()
    s = ctypes.c_double()
    _check("pcad_metrics",
           lib().pcad_metrics(est.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              clean.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), H, W, int(L),
                              ctypes.byref(p), ctypes.byref(s)))
    return float(p.value), float(s.value)


def pcad_chain_export(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check("pcad_chain_export", lib().pcad_chain_export(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check("pcad_chain_export", lib().pcad_chain_export(h, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def pcad_chain_import(blob: bytes, stream=None):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check("pcad_chain_import",
           lib().pcad_chain_import(buf, len(blob), _stream(stream), ctypes.byref(h)))
    return h


def pcad_pca_run_noalloc(g_dev_ptr: int, H: int, W: int, pitch: int, model, seed: int,
                         chain_id: int, nsweeps: int, burn_in: int, sample_dev_ptr: int,
                         mean_dev_ptr: int, stream=None):
    """Lazy-PCA run that allocates no device memory (device pointers in and
    out, e.g. from torch tensors); see include/pcaden.h."""
    m = as_model(model)
    _check("pcad_pca_run_noalloc",
           lib().pcad_pca_run_noalloc(ctypes.c_void_p(int(g_dev_ptr)), int(H), int(W),
                                      int(pitch), ctypes.byref(m), int(seed), int(chain_id),
                                      int(nsweeps), int(burn_in),
                                      ctypes.c_void_p(int(sample_dev_ptr)),
                                      ctypes.c_void_p(int(mean_dev_ptr)), _stream(stream)))


def pcad_chain_destroy(h):
    if h is not None and h.value:
        lib().pcad_chain_destroy(h)


def pcad_status_str(s: int) -> str:
    return lib().pcad_status_str(int(s)).decode()


def pcad_last_error() -> str:
    return lib().pcad_last_error().decode(errors="replace")


def pcad_version() -> str:
    return lib().pcad_version().decode()


N_MARGINS = 8
_MARGIN_KEYS = ("alpha", "gam", "eta", "cb", "hb", "kb0", "kb1", "kbr")


def pcad_model_margins(model) -> dict:
    """The FP32 coefficients and certified-draw margins of a model (host only)."""
    m = as_model(model)
    out = (ctypes.c_double * N_MARGINS)()
    _check("pcad_model_margins", lib().pcad_model_margins(ctypes.byref(m), out, N_MARGINS))
    return dict(zip(_MARGIN_KEYS, list(out)))


class Chain:
    """Owning wrapper of a pcad_chain handle."""

    def __init__(self, g, model, seed: int, chain_id: int = 0, burn_in: int = 0, stream=None,
                 sampler=None, _handle=None, _shape=None):
        if _handle is not None:
            self.h = _handle
            self.H, self.W = _shape
            self.L = None
            self.sampler = None
            return
        g = _u8(g)
        self.H, self.W = g.shape
        m = as_model(model, sampler)
        self.L = m.L
        self.sampler = m.sampler
        self.h = pcad_chain_create(g, m, seed, chain_id, burn_in, stream)

    @classmethod
    def from_blob(cls, blob: bytes, stream=None):
        h = pcad_chain_import(blob, stream)
        import struct
        H, W = struct.unpack_from("<ii", blob, 12)
        return cls(None, None, 0, _handle=h, _shape=(H, W))

    def run(self, n: int):
        pcad_chain_run(self.h, n)
        return self

    def sync(self):
        pcad_chain_sync(self.h)

    def reset(self):
        pcad_chain_reset(self.h)
        return self

    def set_blocking(self, k: int):
        pcad_chain_set_blocking(self.h, k)
        return self

    def set_kernel(self, kind: int):
        pcad_chain_set_kernel(self.h, kind)
        return self

    def set_wait_limit(self, seconds: float):
        pcad_chain_set_wait_limit(self.h, seconds)
        return self

    def inject_stall(self, tile: int):
        pcad_chain_inject_stall(self.h, tile)
        return self

    def set_row_offset(self, row_off: int):
        pcad_chain_set_row_offset(self.h, row_off)
        return self

    def write_rows_dev(self, row0: int, nrows: int, src_ptr: int, src_pitch: int):
        pcad_chain_write_rows_dev(self.h, row0, nrows, src_ptr, src_pitch)
        return self

    def set_model(self, model):
        """New coefficients; the chain's sampler is kept."""
        pcad_chain_set_model(self.h, as_model(model, self.sampler))
        return self

    def run_schedule(self, models, sweeps):
        pcad_chain_run_schedule(self.h, [as_model(m, self.sampler) for m in models], sweeps)
        return self

    def kernel_in_use(self) -> int:
        return pcad_chain_kernel_in_use(self.h)

    def energy(self):
        """(H, pair_sum, data_sum) of the current sample."""
        return pcad_chain_energy(self.h)

    def track_energy(self, capacity: int):
        pcad_chain_track_energy(self.h, capacity)
        return self

    def energies(self) -> np.ndarray:
        return pcad_chain_read_energies(self.h)

    def min_state(self):
        """(state, energy, sweep) of the lowest-energy state tracked."""
        return pcad_chain_read_min_state(self.h, self.H, self.W)

    def sample(self) -> np.ndarray:
        return pcad_chain_read_sample(self.h, self.H, self.W)

    def mean(self) -> np.ndarray:
        return pcad_chain_read_mean(self.h, self.H, self.W)

    def set_sample(self, x):
        pcad_chain_write_sample(self.h, x)

    def sweeps(self):
        return pcad_chain_sweeps(self.h)

    def fp64_draws(self) -> int:
        return pcad_chain_stats(self.h)

    def metrics(self, clean, which: int = 0):
        return pcad_chain_metrics(self.h, clean, which)

    def export(self) -> bytes:
        return pcad_chain_export(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            pcad_chain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ batch / server

def _job(g, model, seed, chain_id, burn_in):
    g = _u8(g)
    H, W = g.shape
    j = PcadJob(g_host=g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), H=H, W=W, g_pitch=W,
                model=as_model(model), seed=int(seed), chain_id=int(chain_id),
                burn_in=int(burn_in))
    return j, g


def pcad_batch_create(jobs, autotune: bool = True, stream=None):
    """jobs: sequence of (g, model, seed, chain_id, burn_in)."""
    keep, arr = [], (PcadJob * len(jobs))()
    for k, (g, m, seed, chain, burn) in enumerate(jobs):
        arr[k], gg = _job(g, m, seed, chain, burn)
        keep.append(gg)
    h = ctypes.c_void_p()
    _check("pcad_batch_create",
           lib().pcad_batch_create(arr, len(jobs), int(bool(autotune)), _stream(stream),
                                   ctypes.byref(h)))
    return h


def pcad_batch_run(h, nsweeps: int):
    _check("pcad_batch_run", lib().pcad_batch_run(h, int(nsweeps)))


def pcad_batch_reset(h):
    _check("pcad_batch_reset", lib().pcad_batch_reset(h))


def pcad_batch_sync(h):
    _check("pcad_batch_sync", lib().pcad_batch_sync(h))


def pcad_batch_set_tiling(h, tile_rows: int, order: int):
    """order 0: image order, 1: costliest first (one launch per sweep);
    2: wavefront (one launch per 16 sweeps)."""
    _check("pcad_batch_set_tiling", lib().pcad_batch_set_tiling(h, int(tile_rows), int(order)))


def pcad_batch_read_sample(h, i: int, H: int, W: int) -> np.ndarray:
    out = np.empty((H, W), dtype=np.uint8)
    _check("pcad_batch_read_sample",
           lib().pcad_batch_read_sample(h, int(i),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W))
    return out


def pcad_batch_read_mean(h, i: int, H: int, W: int) -> np.ndarray:
    out = np.empty((H, W), dtype=np.float32)
    _check("pcad_batch_read_mean",
           lib().pcad_batch_read_mean(h, int(i),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def pcad_batch_slice(h, sweeps: int = 0) -> int:
    """Set (8, 16 or 32; 0 keeps) and return the batch's sweeps per slice."""
    cur = ctypes.c_int()
    _check("pcad_batch_slice", lib().pcad_batch_slice(h, int(sweeps), ctypes.byref(cur)))
    return cur.value


def pcad_batch_info(h) -> dict:
    t = ctypes.c_uint64()
    rows, lpt, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_float()
    f = ctypes.c_uint64()
    _check("pcad_batch_info", lib().pcad_batch_info(h, ctypes.byref(t), ctypes.byref(rows),
                                                    ctypes.byref(lpt), ctypes.byref(grid),
                                                    ctypes.byref(ms), ctypes.byref(f)))
    return dict(t=t.value, tile_rows=rows.value, lpt_order=lpt.value, grid=grid.value,
                tune_ms=ms.value, fp64_draws=f.value)


def pcad_batch_destroy(h):
    if h is not None and h.value:
        lib().pcad_batch_destroy(h)


def pcad_server_create(max_slots: int, hbm_budget_bytes: int, stream=None):
    h = ctypes.c_void_p()
    _check("pcad_server_create", lib().pcad_server_create(int(max_slots), int(hbm_budget_bytes),
                                                          _stream(stream), ctypes.byref(h)))
    return h


def pcad_server_set_limits(h, max_active_sites: int):
    """Admit while the admitted requests hold fewer sites (0: no cap)."""
    _check("pcad_server_set_limits", lib().pcad_server_set_limits(h, int(max_active_sites)))


SERVE_FIFO, SERVE_SRPT = 0, 1


def pcad_server_set_policy(h, policy: int, aging: float = 0.2):
    """FIFO (every admitted request runs) or shortest remaining work first."""
    _check("pcad_server_set_policy", lib().pcad_server_set_policy(h, int(policy), float(aging)))


def pcad_server_submit(h, g, model, seed, chain_id, burn_in, nsweeps) -> int:
    j, gg = _job(g, model, seed, chain_id, burn_in)
    rid = ctypes.c_uint64()
    _check("pcad_server_submit",
           lib().pcad_server_submit(h, ctypes.byref(j), int(nsweeps), ctypes.byref(rid)))
    return int(rid.value)


def pcad_server_step(h, slice_sweeps: int = 16):
    a, p, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("pcad_server_step", lib().pcad_server_step(h, int(slice_sweeps), ctypes.byref(a),
                                                      ctypes.byref(p), ctypes.byref(f)))
    return a.value, p.value, f.value


def pcad_server_poll(h, rid: int, H: int = 0, W: int = 0):
    """Returns (state, sample, mean); sample/mean are None unless state == 2
    and H, W are given (the request is then forgotten by the server)."""
    st = ctypes.c_int()
    if H and W:
        smp = np.empty((H, W), dtype=np.uint8)
        mean = np.empty((H, W), dtype=np.float32)
        _check("pcad_server_poll", lib().pcad_server_poll(
            h, int(rid), ctypes.byref(st), smp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            mean.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        if st.value == 2:
            return st.value, smp, mean
        return st.value, None, None
    _check("pcad_server_poll", lib().pcad_server_poll(h, int(rid), ctypes.byref(st), None, None))
    return st.value, None, None


def pcad_server_info(h) -> dict:
    used = ctypes.c_size_t()
    sl = ctypes.c_uint64()
    f = ctypes.c_uint64()
    _check("pcad_server_info", lib().pcad_server_info(h, ctypes.byref(used), ctypes.byref(sl),
                                                      ctypes.byref(f)))
    return dict(hbm_used=used.value, slices=sl.value, fp64_draws=f.value)


def pcad_server_destroy(h):
    if h is not None and h.value:
        lib().pcad_server_destroy(h)


def pcad_chain_set_blocking(h, k: int):
    """k sweeps per launch on TMA-loaded shared-memory tiles (0: unblocked)."""
    _check("pcad_chain_set_blocking", lib().pcad_chain_set_blocking(h, int(k)))


def pcad_chain_kernel_in_use(h) -> int:
    """Kernel kind of the chain's next sweeps (-k: temporal blocking, k per launch)."""
    k = ctypes.c_int()
    _check("pcad_chain_kernel_in_use", lib().pcad_chain_kernel_in_use(h, ctypes.byref(k)))
    return k.value


def pcad_chain_set_model(h, model):
    """New coefficients (annealing); the model's structure must stay."""
    m = as_model(model)
    _check("pcad_chain_set_model", lib().pcad_chain_set_model(h, ctypes.byref(m)))


def pcad_chain_run_schedule(h, models, sweeps):
    """For each stage: set models[k], run sweeps[k] sweeps."""
    n = len(models)
    if len(sweeps) != n:
        raise ValueError("one sweep count per model")
    arr = (PcadModel * n)(*[as_model(m) for m in models])
    sw = (ctypes.c_int * n)(*[int(k) for k in sweeps])
    _check("pcad_chain_run_schedule", lib().pcad_chain_run_schedule(h, arr, sw, n))


def pcad_batch_set_model(h, i: int, model):
    m = as_model(model)
    _check("pcad_batch_set_model", lib().pcad_batch_set_model(h, int(i), ctypes.byref(m)))


def pcad_chain_energy(h):
    """Posterior energy H of the chain's current sample and its integer sums."""
    e = ctypes.c_double()
    p, d = ctypes.c_uint64(), ctypes.c_uint64()
    _check("pcad_chain_energy", lib().pcad_chain_energy(h, ctypes.byref(e), ctypes.byref(p),
                                                        ctypes.byref(d)))
    return e.value, p.value, d.value


def pcad_chain_track_energy(h, capacity: int):
    _check("pcad_chain_track_energy", lib().pcad_chain_track_energy(h, int(capacity)))


def pcad_chain_read_energies(h) -> np.ndarray:
    n = ctypes.c_int()
    _check("pcad_chain_read_energies", lib().pcad_chain_read_energies(h, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.float64)
    if n.value:
        _check("pcad_chain_read_energies",
               lib().pcad_chain_read_energies(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              n.value, ctypes.byref(n)))
    return out


def pcad_chain_read_min_state(h, H: int, W: int):
    out = np.zeros((H, W), dtype=np.uint8)
    e = ctypes.c_double()
    t = ctypes.c_uint64()
    _check("pcad_chain_read_min_state",
           lib().pcad_chain_read_min_state(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W,
                                           ctypes.byref(e), ctypes.byref(t)))
    return out, e.value, t.value


PCAD_KERNEL_AUTO = 0
PCAD_KERNEL_CUDA_CORE = 1
PCAD_KERNEL_TENSOR = 2
PCAD_KERNEL_WAVE = 3
PCAD_KERNEL_SMALL = 4
PCAD_KERNEL_RESIDENT = 5
PCAD_KERNEL_WINDOW = 6
PCAD_KERNEL_WINDOW_WAVE = 7
PCAD_KERNEL_BINARY = 8


def pcad_chain_set_kernel(h, kind: int):
    """Kernel of unblocked PCA sweeps: auto, CUDA cores, or tensor-core prior sums."""
    _check("pcad_chain_set_kernel", lib().pcad_chain_set_kernel(h, int(kind)))


def pcad_chain_set_wait_limit(h, seconds: float):
    """Elapsed-time limit of every bounded device-side wait of the chain's sweeps."""
    _check("pcad_chain_set_wait_limit", lib().pcad_chain_set_wait_limit(h, float(seconds)))


def pcad_chain_set_row_offset(h, row_off: int):
    """Global row of the chain's local row 0 (a band of a larger image)."""
    _check("pcad_chain_set_row_offset", lib().pcad_chain_set_row_offset(h, int(row_off)))


def pcad_chain_write_rows_dev(h, row0: int, nrows: int, src_ptr: int, src_pitch: int):
    """Overwrite rows of the current state from device memory (stream-ordered)."""
    _check("pcad_chain_write_rows_dev",
           lib().pcad_chain_write_rows_dev(h, int(row0), int(nrows), ctypes.c_void_p(int(src_ptr)),
                                           int(src_pitch)))


def pcad_bands_create(g, model, seed: int, chain_id: int = 0, burn_in: int = 0, nbands: int = 2,
                      halo: int = 32, devices=None):
    g = _u8(g)
    H, W = g.shape
    m = as_model(model)
    h = ctypes.c_void_p()
    dv = None if devices is None else (ctypes.c_int * len(devices))(*[int(d) for d in devices])
    _check("pcad_bands_create",
           lib().pcad_bands_create(g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), H, W, W,
                                   ctypes.byref(m), int(seed), int(chain_id), int(burn_in),
                                   int(nbands), int(halo), dv, ctypes.byref(h)))
    return h


def pcad_bands_run(h, nsweeps: int):
    _check("pcad_bands_run", lib().pcad_bands_run(h, int(nsweeps)))


def pcad_bands_sync(h):
    _check("pcad_bands_sync", lib().pcad_bands_sync(h))


def pcad_bands_read_sample(h, H: int, W: int) -> np.ndarray:
    out = np.zeros((H, W), dtype=np.uint8)
    _check("pcad_bands_read_sample",
           lib().pcad_bands_read_sample(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W))
    return out


def pcad_bands_read_mean(h, H: int, W: int) -> np.ndarray:
    out = np.zeros((H, W), dtype=np.float32)
    _check("pcad_bands_read_mean",
           lib().pcad_bands_read_mean(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def pcad_bands_info(h, band: int) -> dict:
    v = [ctypes.c_int() for _ in range(4)]
    t = ctypes.c_uint64()
    _check("pcad_bands_info", lib().pcad_bands_info(h, int(band), *[ctypes.byref(x) for x in v],
                                                    ctypes.byref(t)))
    return dict(own0=v[0].value, own1=v[1].value, buf0=v[2].value, buf1=v[3].value, t=t.value)


def pcad_bands_destroy(h):
    if h is not None and h.value:
        lib().pcad_bands_destroy(h)


def pcad_chain_inject_stall(h, tile: int):
    """Test aid: wavefront tile `tile` never reports a finished sweep (-1: off)."""
    _check("pcad_chain_inject_stall", lib().pcad_chain_inject_stall(h, int(tile)))
