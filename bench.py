"""Benchmark: lazy-PCA denoising on one GB300, against its roofline, with
checkerboard Gibbs on the same GPU, a batched and a served form.

Headline workload (one "step"): the large single image of the roofline
run -- 8192 x 8192, L = 256 labels (uint8), smooth gradients plus 20
rectangles/disks, additive Gaussian noise sigma = 25 (label units, clipped,
rounded), truncated-linear prior c_T = 0.05, T = 30 on the 4-neighbourhood,
inertia lambda = 2.0 -- 200 lazy-PCA sweeps from the observation with
burn-in 50 and the FP32 posterior-mean accumulator.  Synthetic, seeded
inputs (the paper's images are not public).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  `value` is site-updates/s with the inputs resident in
HBM (CUDA events on the chain's stream, L2 flushed between steps); `e2e` is
the same metric through the public C ABI with host buffers (create from
pinned host memory, run, read the mean back).  Beside it, each measured
once or twice: the same image at L = 16 and with k = 4 / 8 sweeps per
TMA-tiled launch (`config3`), checkerboard Gibbs on the same image
(`gibbs`), the 512 x 512 L = 256 chain of 2000 sweeps (`greyscale512`),
128 uneven images x 4 chains in one batch against one chain per launch
(`batch`), a Poisson request stream through the continuous-batching server
against one request at a time (`serve`), and the FP64 oracle on the host
cores (`cpu_baseline`).  `--impl reference` times the oracle alone.  Under
torchrun each rank runs its own independent chain (weak scaling).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIDE, LABELS, SWEEPS, BURN_IN = 8192, 256, 200, 50
WORKLOAD = ("large single image 8192x8192, L=256 (uint8), Gaussian sigma=25, truncated-linear "
            "c_T=0.05 T=30 4-nbhd, lambda=2.0, 200 sweeps, burn-in 50, FP32 posterior mean")
G512_SWEEPS, G512_BURN = 2000, 500
G512_WORKLOAD = ("greyscale 512x512, L=256 (uint8), Gaussian sigma=20, truncated-linear "
                 "c_T=0.05 T=30 4-nbhd, lambda=2.0, 2000 sweeps, burn-in 500")
# SFU ex2 issue: 32 per SM per clock (4 SM sub-partitions x 8) x 152 SMs x 2070 MHz
SFU_PEAK_T = 152 * 32 * 2.070e9 / 1e12
SFU_PEAK_SOURCE = ("152 SMs x 32 ex2/clk/SM x 2070 MHz (unit count x max clock; an "
                   "ex2.approx.ftz loop measured 29.9/clk/SM)")
HBM_PEAK_FALLBACK = 6800.0   # GB/s, used only if MEASURED_PEAKS.json is absent

# DRAM bytes (read + write) per site-update of each kernel, from ncu captures
# (profiles/); None until the current kernel is captured.  The tensor-core
# figure is one 32-sweep launch at 4096^2 (planes, observation and
# accumulator exceed L2); the small-label figure one accumulating per-sweep
# launch of its TMA-tile form at 8192^2 L = 16; the per-sweep CUDA-core
# kernel has no current capture at 8192^2.
NCU_TC_BYTES_PER_SITE = (3.213934e9 + 2.634401e9) / (32 * 4096 * 4096)
NCU_TC_NOTE = ("ncu dram__bytes_read+write of one accumulating 32-sweep pca_tcw_kernel launch "
               "at 4096^2 L=256 (profiles/pca_tc_l256_4096sq.md), scaled by sites to 8192^2")
NCU_DIRECT_BYTES_PER_SITE = None
NCU_DIRECT_NOTE = "ncu dram__bytes_read+write of one pca_direct_kernel launch at 8192^2 L=16"
NCU_WIN_BYTES_PER_SITE = (402903040 + 286483712) / (8192 * 8192)
NCU_WIN_NOTE = ("ncu dram__bytes_read+write of one accumulating pca_win_kernel launch at "
                "8192^2 L=256 (profiles/pca_win_l256_8192sq.md)")
NCU_SMALL_BYTES_PER_SITE = (408240384 + 280811264) / (8192 * 8192)
NCU_SMALL_NOTE = ("ncu dram__bytes_read+write of one accumulating pca_small_tma_kernel launch "
                  "at 8192^2 L=16 (profiles/pca_small_tma_l16_6144sq.md)")

KERNEL_KINDS = {"auto": 0, "cuda_core": 1, "tensor": 2, "wave": 3, "small": 4, "resident": 5,
                "window": 6, "window_wave": 7, "binary": 8}
KERNEL_NAMES = {
    1: "pca_direct_kernel (CUDA cores, one launch per sweep)",
    2: "pca_tcw_kernel<4,0,0,0> (tcgen05 windowed tent sums, CUDA-core CDF, wavefront, "
       "one launch per 32 sweeps)",
    3: "pca_wave_kernel (CUDA cores, wavefront, one launch per 32 sweeps)",
    4: "small-label draw (CUDA cores, prior sums from a pair table, one launch per sweep; "
       "pca_small_tma_kernel on TMA-loaded tiles from 2^23 sites, else pca_small_kernel)",
    5: "resident_kernel (two labels, whole run in one single-CTA launch, state in shared "
       "memory, exact per-configuration thresholds)",
    6: "pca_win_kernel (CUDA cores, hull chunks from a tent-byte table, one launch per sweep)",
    7: "pca_winw_kernel (the windowed draw as a wavefront, one launch per 32 sweeps)",
    8: "pca_binary_kernel (two labels, threshold table, one launch per sweep)",
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-gibbs", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--only-head", action="store_true",
                   help="print the headline line without the side measurements (config3 "
                        "variants, Gibbs, 512^2 chain, batch, serve)")
    p.add_argument("--profile-case", nargs=3, type=int, metavar=("SIDE", "L", "SWEEPS"),
                   help="run one SIDE x SIDE chain with L labels for SWEEPS sweeps and exit "
                        "(the small case ncu captures; prints no JSON line)")
    p.add_argument("--sampler", type=int, default=0, help="profile case: 0 PCA, 1 Gibbs")
    p.add_argument("--blocking", type=int, default=0,
                   help="profile case: sweeps per TMA-tiled launch (0: unblocked)")
    p.add_argument("--workload", default="chain",
                   choices=["chain", "batch", "serve", "blocking", "protocol", "cpu"],
                   help="chain: the default line; batch: uneven images x 4 chains in one "
                        "persistent launch vs one chain per launch; serve: Poisson request "
                        "stream through the continuous-batching server; blocking: 8192^2 "
                        "unblocked vs k = 1..8; protocol: the paper's annealed runs on MRF "
                        "images and the q grid; cpu: the FP64 oracle on the host cores "
                        "(single-threaded Gibbs and PCA, OpenMP PCA) beside the GPU chain")
    p.add_argument("--kernel", default="auto",
                   choices=list(KERNEL_KINDS),
                   help="kernel of the unblocked PCA sweep (headline chain and profile case): "
                        "auto = for eligible models with L >= 32 the windowed CUDA-core sweep "
                        "on large images and the tensor-core sweep on small ones (L >= 192), "
                        "else the small-label, resident, two-label, per-sweep or wavefront "
                        "CUDA-core kernel; tensor = prior sums by tcgen05.mma; window = the "
                        "windowed sweep; binary = the two-label sweep")
    p.add_argument("--images", type=int, default=128, help="batch: number of images")
    p.add_argument("--requests", type=int, default=200, help="serve: requests per rate")
    p.add_argument("--rates", default="10,25,50,200",
                   help="serve: comma-separated arrival rates (req/s)")
    p.add_argument("--aging", type=float, default=0.2,
                   help="serve: priority seconds a waiting request gains per second "
                        "(shortest-remaining-work scheduling)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(self.out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for name, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _hbm_peak():
    """Measured copy bandwidth (GB/s) and where it came from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_PEAK_FALLBACK, "fallback"


def _inputs(L=LABELS):
    from pcad_inputs import large_image
    return large_image(seed=3, side=SIDE, L=L)


def _algo_bytes(sites, sweeps, burn):
    """Algorithmic DRAM bytes of `sweeps` sweeps from sweep 0: per site-update
    1 B label and 1 B observation in, 1 B label out, plus the 8 B FP32
    accumulator read-modify-write once past burn-in."""
    return sites * (3 * sweeps + 8 * max(0, sweeps - burn))


def _sfu_roofline(sites, L, ms_per_sweep, kernel, traffic=None, traffic_note=None,
                  sweeps_per_launch=1):
    """The exponential-per-label bound: one label evaluation = one ex2."""
    achieved = sites * L / (ms_per_sweep * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": SFU_PEAK_T, "unit": "T ex2/s",
            "frac": achieved / SFU_PEAK_T, "traffic": traffic, "traffic_source": traffic_note,
            "traffic_unit": f"DRAM bytes per launch ({sweeps_per_launch} sweeps)",
            "kernel": kernel, "peak_source": SFU_PEAK_SOURCE, "ms_per_sweep": ms_per_sweep,
            "work_per_unit": f"one label evaluation (one exponential on the SFU in a direct "
                             f"evaluation), L={L} per site-update"}


def _crop(a, side):
    return a[:side, :side].copy()


def cpu_baseline(seconds: float = 10.0):
    """FP64 oracle lazy-PCA sweeps of a 2048 x 2048 crop of the headline image
    on all host cores (OpenMP over rows)."""
    import oracle
    clean, noisy, m = _inputs()
    g = _crop(noisy, 2048)
    x = g.copy()
    t0 = time.perf_counter()
    n = 0
    while True:
        x, _ = oracle.pca_sweep(m, g, x, 3, 0, n)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 64:
            break
    dt = time.perf_counter() - t0
    return {"value": g.size * n / dt, "unit": "site-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{n} lazy-PCA sweeps of a 2048x2048 crop of the "
                                        f"8192x8192 L=256 image ({dt:.1f} s, OpenMP over rows)"}


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    clean, noisy, m = _inputs()
    g = _crop(noisy, 2048)
    x = g.copy()
    for t in range(a.warmup):
        x, _ = oracle.pca_sweep(m, g, x, 3, 0, t)
    times = []
    for k in range(a.steps):
        t0 = time.perf_counter()
        x, _ = oracle.pca_sweep(m, g, x, 3, 0, a.warmup + k)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    v = g.size * a.steps / T
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": "site-updates/s", "value": v,
            "unit": "site-updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * T / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "one lazy-PCA sweep of a 2048x2048 crop "
                                                    "(bounded sample of the 200-sweep chain)"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v,
                             "sample": f"{a.steps} sweeps of a 2048x2048 crop of the "
                                       f"8192x8192 L=256 image"},
            "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _launches_per_run(kind, sweeps, sampler=0):
    """Kernel launches of one `sweeps`-sweep run: 32-sweep captured blocks
    plus the rest.  Wavefront kernels: one sweep launch and the counter
    advance per block; per-sweep kernels: one launch per sweep (or per Gibbs
    colour phase) plus the advance."""
    if kind == 5:
        return 2                       # the run's launch and the counter advance
    blocks, rest = divmod(sweeps, 32)
    if kind in (2, 3, 7):
        return 2 * blocks + (2 if rest else 0)
    per = 2 if sampler else 1
    return blocks * (32 * per + 1) + ((rest * per + 1) if rest else 0)


def _safe(fn, *args, **kw):
    """A side measurement that fails is recorded, not fatal to the line."""
    try:
        return fn(*args, **kw)
    except Exception as e:   # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(a):
    import numpy as np
    import torch

    import paper_2507_14869_gb300 as pc
    from paper_2507_14869_gb300 import replicas

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    cid = replicas.chain_id(rank, 0, 1)   # one chain per rank, distinct uniforms
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    clean, noisy, m = _inputs()
    H, W = noisy.shape
    sites = H * W
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hbm_peak, hbm_src = _hbm_peak()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(chain, sweeps, steps, warm):
        """K timed runs of `sweeps` sweeps from a reset, L2 flushed before each."""
        for _ in range(warm):
            chain.reset().run(sweeps)
        chain.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(steps):
                chain.reset()
                flush.fill_(k & 0xFF)              # L2 flush between timed steps
                evs[k][0].record(stream)
                chain.run(sweeps)
                evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        chain.sync()
        barrier()
        wall = time.perf_counter() - wall0
        return [e0.elapsed_time(e1) for e0, e1 in evs], wall

    # ---- headline: 8192^2, L = 256, 200 sweeps (default kernel)
    kind = KERNEL_KINDS[a.kernel]
    pca = pc.Chain(noisy, m, seed=3, chain_id=cid, burn_in=BURN_IN, stream=stream)
    pca.set_kernel(kind)
    pca_kind = pca.kernel_in_use()
    with ClockSampler(local) as clk:
        ms, wall = timed(pca, SWEEPS, a.steps, a.warmup)
    T = sum(ms) / 1e3
    T_max = replicas.max_time(T)   # the slowest rank's time
    value = world * sites * SWEEPS * a.steps / T_max
    ms_sweep = 1e3 * T / (a.steps * SWEEPS)
    fp64 = pca.fp64_draws()
    psnr, ssim = pca.metrics(clean, 0)
    last_psnr, _ = pca.metrics(clean, 1)
    x_head = pca.sample()
    pca.close()
    spl = 32 if pca_kind in (2, 3, 7) else 1       # sweeps per launch
    per_site = {2: NCU_TC_BYTES_PER_SITE, 1: NCU_DIRECT_BYTES_PER_SITE,
                6: NCU_WIN_BYTES_PER_SITE}.get(pca_kind)
    traffic = per_site * sites * spl if per_site else None
    note = {2: NCU_TC_NOTE, 6: NCU_WIN_NOTE}.get(pca_kind, NCU_DIRECT_NOTE)
    roof = _sfu_roofline(sites, LABELS, ms_sweep, KERNEL_NAMES.get(pca_kind, str(pca_kind)),
                         traffic, note, spl)
    roof["algorithmic_bytes_per_launch"] = 11 * sites * spl
    roof["hbm_frac"] = (_algo_bytes(sites, SWEEPS, BURN_IN) / (ms_sweep * SWEEPS * 1e-3) / 1e9
                        / hbm_peak)

    # ---- end to end through the public API with host buffers (pinned)
    g_host = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
    g_host.numpy()[:] = noisy
    mean_host = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
    e2e_steps = 2
    torch.cuda.synchronize(dev)
    e2e_t = []
    for k in range(e2e_steps + 1):
        t0 = time.perf_counter()
        ch = pc.Chain(g_host.numpy(), m, seed=3, chain_id=cid, burn_in=BURN_IN, stream=stream)
        ch.set_kernel(kind)
        ch.run(SWEEPS)
        pc.pcad_chain_read_mean(ch.h, H, W, out=mean_host.numpy())
        ch.close()
        if k > 0:                                     # first one warms the allocator
            e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * sites * SWEEPS / statistics.mean(e2e_t)

    side = {}
    if not a.only_head:
        side["config3"] = _safe(_config3, pc, stream, timed, x_head, ms_sweep, pca_kind,
                                hbm_peak, cid)
        side["bands"] = _safe(_bands_8192, pc, torch, noisy, m, cid, x_head, value / world)
        if not a.no_gibbs:
            side["gibbs"] = _safe(_gibbs_8192, pc, stream, timed, noisy, m, clean, cid)
        side["greyscale512"] = _safe(_greyscale512, pc, stream, timed, cid, a.no_gibbs)
        if world == 1:
            side["binary64"] = _safe(_binary64, pc, torch, stream)
        if world == 1:
            side["batch"] = _safe(_batch_object, pc, torch, stream, a.images)
            rates = [float(x) for x in a.rates.split(",") if x]
            side["serve"] = _safe(_serve_object, pc, torch, stream, rates, a.requests,
                                  aging=a.aging)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * T_max / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": sites, "sweeps_per_step": SWEEPS,
                   "burn_in": BURN_IN,
                   "l2": "inputs larger than L2 (8192^2 planes, 256 MiB accumulator) and a "
                         "256 MiB flush write before each timed step",
                   "parallelism": "independent chain per GPU" if world > 1 else "1 GPU"},
        "roofline": roof,
        "gpu_launches": a.steps * _launches_per_run(pca_kind, SWEEPS),
        "e2e": {"value": e2e_v, "unit": "site-updates/s", "h2d_bytes_per_step": sites,
                "d2h_bytes_per_step": sites * 4, "steps": e2e_steps,
                "ms_per_step": 1e3 * statistics.mean(e2e_t),
                "path": "pcad_chain_create(host) + pcad_chain_run + pcad_chain_read_mean(host)"},
        "label_evals_per_s": value * LABELS,
        "fp64_redraw_fraction": fp64 / float(sites * SWEEPS),   # counter restarts each step
        "psnr_db": psnr, "ssim": ssim, "last_sample_psnr_db": last_psnr,
        "wall_s_timed": wall, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
        "kernel": KERNEL_NAMES.get(pca_kind, str(pca_kind)),
    }
    line.update(side)
    line["clocks"] = clk.summary()
    if world == 1 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _config3(pc, stream, timed, x_head, ms_head, head_kind, hbm_peak, cid):
    """The roofline workload's other runs: L = 256 with k = 4 and 8 sweeps per
    TMA-tiled launch, and L = 16 (sigma 1.0) unblocked and with k = 4, 8;
    each a 200-sweep chain from the observation, burn-in 50.  Labels are
    bit-identical across k (checked)."""
    import numpy as np
    out = {"L=256": {"unblocked": {"site_updates_per_s": SIDE * SIDE / (ms_head * 1e-3),
                                   "ms_per_sweep": ms_head, "kernel": head_kind,
                                   "note": "the headline run"}}}
    for L, ks, steps in ((256, (4, 8), 1), (16, (0, 4, 8), 2)):
        clean, noisy, m = _inputs(L)
        sites = noisy.size
        ref = x_head if L == 256 else None
        rows = out.setdefault(f"L={L}", {})
        for k in ks:
            ch = pc.Chain(noisy, m, seed=3, chain_id=cid, burn_in=BURN_IN, stream=stream)
            ch.set_blocking(k)
            ms, _ = timed(ch, SWEEPS, steps, 1)
            kind = ch.kernel_in_use()
            x = ch.sample()
            ch.close()
            same = True if ref is None else bool(np.array_equal(x, ref))
            ref = x if ref is None else ref
            ms_sweep = sum(ms) / (steps * SWEEPS)
            name = "unblocked" if k == 0 else f"k={k}"
            r = {"site_updates_per_s": sites / (ms_sweep * 1e-3), "ms_per_sweep": ms_sweep,
                 "kernel": kind, "identical_labels": same}
            sfu = _sfu_roofline(sites, L, ms_sweep, str(kind))
            gbs = _algo_bytes(sites, SWEEPS, BURN_IN) / (ms_sweep * SWEEPS * 1e-3) / 1e9
            hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                   "frac": gbs / hbm_peak,
                   "algorithmic_bytes_per_site_update": _algo_bytes(1, SWEEPS, BURN_IN) / SWEEPS}
            if L == 16 and k == 0:
                per_site = NCU_SMALL_BYTES_PER_SITE if kind == 4 else (
                    NCU_DIRECT_BYTES_PER_SITE if kind == 1 else None)
                hbm["traffic"] = per_site * sites if per_site else None
                hbm["traffic_source"] = NCU_SMALL_NOTE if kind == 4 else NCU_DIRECT_NOTE
                r["roofline"] = hbm
                r["sfu_frac"] = sfu["frac"]
                # the binding bound: min(HBM / B, SFU / L) site-updates/s
                bound = min(hbm_peak * 1e9 / hbm["algorithmic_bytes_per_site_update"],
                            SFU_PEAK_T * 1e12 / L)
                r["frac_of_binding_bound"] = r["site_updates_per_s"] / bound
            else:
                r["roofline"] = {k2: sfu[k2] for k2 in ("bound", "achieved", "peak", "unit",
                                                        "frac")}
                r["hbm_frac"] = hbm["frac"]
            rows[name] = r
    return out


def _bands_8192(pc, torch, noisy, m, cid, x_head, head_rate, nbands=2, halo=32):
    """The headline chain split into row bands on this one GPU (one chain and
    stream per band, halo rows exchanged after every 32 sweeps): the cost of
    the decomposition a multi-GPU run would use, and its bit-identity."""
    import numpy as np
    H, W = noisy.shape
    b = pc.pcad_bands_create(noisy, m, seed=3, chain_id=cid, burn_in=BURN_IN, nbands=nbands,
                             halo=halo)
    try:
        pc.pcad_bands_run(b, 32)
        pc.pcad_bands_sync(b)
        b2 = pc.pcad_bands_create(noisy, m, seed=3, chain_id=cid, burn_in=BURN_IN,
                                  nbands=nbands, halo=halo)
    finally:
        pc.pcad_bands_destroy(b)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pc.pcad_bands_run(b2, SWEEPS)
        pc.pcad_bands_sync(b2)
        dt = time.perf_counter() - t0
        same = bool(np.array_equal(pc.pcad_bands_read_sample(b2, H, W), x_head))
    finally:
        pc.pcad_bands_destroy(b2)
    rate = H * W * SWEEPS / dt
    return {"nbands": nbands, "halo_rows": halo, "site_updates_per_s": rate,
            "vs_whole_image": rate / head_rate, "identical_labels": same,
            "note": "host-timed; both bands on one GPU, each on its own stream"}


def _gibbs_8192(pc, stream, timed, noisy, m, clean, cid, steps=2):
    """Checkerboard Gibbs (2 colour phases per sweep) on the headline image."""
    ch = pc.Chain(noisy, m, seed=3, chain_id=cid, burn_in=BURN_IN, stream=stream,
                  sampler=pc.SAMPLER_GIBBS_CB)
    ms, _ = timed(ch, SWEEPS, steps, 1)
    kind = ch.kernel_in_use()
    p, s = ch.metrics(clean, 0)
    ch.close()
    ms_sweep = sum(ms) / (steps * SWEEPS)
    sites = noisy.size
    name = {2: "pca_tcw_kernel<4,0,0,0,1> (checkerboard Gibbs on the tensor-core wavefront, 2 "
               "colour phases per sweep)",
            6: "gibbs_win_kernel (CUDA cores, windowed draw, one launch per colour phase, 2 "
               "phases per sweep)"}.get(kind, "gibbs_cb_kernel (2 colour phases)")
    return {"value": sites / (ms_sweep * 1e-3), "unit": "site-updates/s",
            "ms_per_step": sum(ms) / steps, "ms_per_sweep": ms_sweep, "steps": steps,
            "psnr_db": p, "ssim": s, "kernel": name,
            "launches_per_step": _launches_per_run(kind, SWEEPS, sampler=1),
            "roofline": _sfu_roofline(sites, LABELS, ms_sweep, name)}


def _greyscale512(pc, stream, timed, cid, no_gibbs, steps=5):
    """The 512 x 512 L = 256 chain, 2000 sweeps, burn-in 500 (L2-resident)."""
    from pcad_inputs import greyscale_512
    clean, noisy, m = greyscale_512(seed=2)
    out = {"workload": G512_WORKLOAD}
    for name, sampler in (("pca", pc.SAMPLER_PCA), ("gibbs", pc.SAMPLER_GIBBS_CB)):
        if no_gibbs and sampler:
            continue
        ch = pc.Chain(noisy, m, seed=2, chain_id=cid, burn_in=G512_BURN, stream=stream,
                      sampler=sampler)
        ms, _ = timed(ch, G512_SWEEPS, steps, 2)
        p, s = ch.metrics(clean, 0)
        kind = ch.kernel_in_use()
        ch.close()
        ms_sweep = sum(ms) / (steps * G512_SWEEPS)
        out[name] = {"value": noisy.size / (ms_sweep * 1e-3), "unit": "site-updates/s",
                     "ms_per_step": sum(ms) / steps, "psnr_db": p, "ssim": s, "kernel": kind,
                     "roofline": {k: v for k, v in _sfu_roofline(
                         noisy.size, 256, ms_sweep, str(kind)).items()
                         if k in ("bound", "achieved", "peak", "unit", "frac", "ms_per_sweep")}}
    return out


BATCH_SWEEPS, BATCH_BURN = 200, 50


def _binary64(pc, torch, stream, n_batch=512, reps=5):
    """The two-label image workload (64 x 64, Ising c_P = 1.2, flip p = 0.1,
    lambda = 1, 500 sweeps, burn-in 100): one chain on the default kernel
    (the resident one: the whole run in one single-CTA launch) against
    per-sweep launches in CUDA graphs, lazy PCA and checkerboard Gibbs,
    device-timed; the wall clock of create (host image) + run + read mean;
    then n_batch such chains (distinct images) as one batch against the same
    chains run one after another."""
    import numpy as np

    from pcad_inputs import binary_64

    sweeps, burn = 500, 100
    clean, g, m = binary_64()
    out = {"workload": "64x64 binary, Ising c_P=1.2, flip p=0.1, lambda=1.0, 500 sweeps, "
                       "burn-in 100"}

    def dev_ms(ch):
        ch.run(sweeps)
        ch.sync()
        ts = []
        for _ in range(reps):
            ch.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ch.run(sweeps)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for name, sampler in (("pca", 0), ("gibbs", 1)):
        row = {}
        for label, kind in (("default", 0), ("per_sweep_graphs", 1)):
            with pc.Chain(g, m, seed=1, chain_id=0, burn_in=burn, sampler=sampler,
                          stream=stream) as ch:
                ch.set_kernel(kind)
                k_used = ch.kernel_in_use()
                ms = dev_ms(ch)
                psnr = ch.metrics(clean, 0)[0]
            kname = KERNEL_NAMES.get(k_used, str(k_used))
            if sampler and k_used == 1:
                kname = "gibbs_cb_kernel (CUDA cores, one launch per colour phase)"
            row[label] = {"ms": ms, "site_updates_per_s": 4096 * sweeps / (ms * 1e-3),
                          "kernel": kname, "psnr_db": psnr}
        walls = []
        for _ in range(reps):
            t0 = time.perf_counter()
            with pc.Chain(g, m, seed=1, chain_id=0, burn_in=burn, sampler=sampler,
                          stream=stream) as ch:
                ch.run(sweeps)
                ch.mean()
            walls.append(time.perf_counter() - t0)
        row["e2e_wall_ms"] = 1e3 * statistics.median(walls)
        row["speedup_vs_per_sweep"] = row["per_sweep_graphs"]["ms"] / row["default"]["ms"]
        out[name] = row

    jobs = [(binary_64(seed=1 + i)[1], m, 1, i, burn) for i in range(n_batch)]
    b = pc.pcad_batch_create(jobs, autotune=False, stream=stream.cuda_stream)
    try:
        pc.pcad_batch_run(b, 32)
        pc.pcad_batch_reset(b)
        pc.pcad_batch_sync(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pc.pcad_batch_run(b, sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_batch = e0.elapsed_time(e1) * 1e-3
        chains = [pc.Chain(gg, mm, seed=sd, chain_id=c, burn_in=bi, stream=stream)
                  for gg, mm, sd, c, bi in jobs]
        try:
            for ch in chains[:4]:
                ch.run(16)
            for ch in chains:
                ch.reset()
            torch.cuda.synchronize()
            e0.record(stream)
            for ch in chains:
                ch.run(sweeps)
            e1.record(stream)
            torch.cuda.synchronize()
            t_plain = e0.elapsed_time(e1) * 1e-3
            same = all(np.array_equal(pc.pcad_batch_read_mean(b, k, 64, 64), chains[k].mean())
                       for k in range(0, n_batch, 17))
        finally:
            for ch in chains:
                ch.close()
    finally:
        pc.pcad_batch_destroy(b)
    out["batch"] = {"chains": n_batch, "ms": 1e3 * t_batch, "img_per_s": n_batch / t_batch,
                    "site_updates_per_s": n_batch * 4096 * sweeps / t_batch,
                    "one_after_another_ms": 1e3 * t_plain,
                    "one_after_another_img_per_s": n_batch / t_plain,
                    "speedup_vs_one_after_another": t_plain / t_batch,
                    "identical_means": bool(same)}
    return out


def _batch_object(pc, torch, stream, n_images, rank=0, world=1):
    """Uneven images (short side log-uniform 64..2048, aspect 1..3, L in
    {2, 16, 256}, per-image prior/inertia), 4 chains each, 200 sweeps with
    burn-in 50: the batch (autotuned, 16-sweep graph slices) against the same
    chains run one after another through the chain API on the same GPU.
    Outputs are bit-identical, so PSNR is equal by construction (checked)."""
    import numpy as np

    from paper_2507_14869_gb300 import replicas
    from pcad_inputs import batched_jobs

    all_imgs = batched_jobs(seed=4, n_images=n_images, chains=4, sweeps=BATCH_SWEEPS,
                            burn_in=BATCH_BURN)
    # each rank takes its share of the images (cost ~ sites x labels), no collective
    mine = replicas.shard([j.noisy.size * j.model.L for j in all_imgs], world)[rank]
    imgs = [all_imgs[i] for i in mine]
    jobs = [(j.noisy, j.model, j.seed, c, j.burn_in) for j in imgs for c in range(j.chains)]
    sites = sum(g.size for g, *_ in jobs)
    by_L = {}
    for g, m, *_ in jobs:
        by_L[m.L] = by_L.get(m.L, 0) + g.size

    b = pc.pcad_batch_create(jobs, autotune=True, stream=stream)
    info = pc.pcad_batch_info(b)
    info["sweeps_per_slice"] = pc.pcad_batch_slice(b)
    pc.pcad_batch_run(b, 16)
    pc.pcad_batch_reset(b)
    pc.pcad_batch_sync(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    pc.pcad_batch_run(b, BATCH_SWEEPS)
    ev[1].record(stream)
    torch.cuda.synchronize()
    pc.pcad_batch_sync(b)
    t_batch = ev[0].elapsed_time(ev[1]) / 1e3
    fp64 = pc.pcad_batch_info(b)["fp64_draws"]

    chains = [pc.Chain(g, m, seed=s, chain_id=c, burn_in=bi, stream=stream)
              for g, m, s, c, bi in jobs]
    for ch in chains[:8]:
        ch.run(16)
    for ch in chains:
        ch.reset()
    torch.cuda.synchronize()
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev2[0].record(stream)
    for ch in chains:
        ch.run(BATCH_SWEEPS)
    ev2[1].record(stream)
    torch.cuda.synchronize()
    t_plain = ev2[0].elapsed_time(ev2[1]) / 1e3

    # equal PSNR: identical posterior means (checked on a spread of chains)
    same = True
    psnr = []
    for k in range(0, len(jobs), max(1, len(jobs) // 16)):
        g = jobs[k][0]
        mb = pc.pcad_batch_read_mean(b, k, *g.shape)
        same &= bool(np.array_equal(mb, chains[k].mean()))
    for i, j in enumerate(imgs):
        psnr.append(chains[4 * i].metrics(j.clean, 0)[0])
    for ch in chains:
        ch.close()
    pc.pcad_batch_destroy(b)
    # whole job: every rank's images over the slowest rank's time
    t_batch = replicas.max_time(t_batch)
    t_plain = replicas.max_time(t_plain)
    sites = sum(replicas.gather({rank: sites}).values())
    psnr_all = replicas.gather({rank: psnr})
    psnr = [v for r in sorted(psnr_all) for v in psnr_all[r]]
    same = all(replicas.gather({rank: same}).values())
    n_img = len(all_imgs)
    return {"value": n_img / t_batch, "unit": "img/s",
            "workload": f"{n_img} uneven images x 4 chains, {BATCH_SWEEPS} sweeps, burn-in "
                        f"{BATCH_BURN}", "chain_sites": sites,
            "sites_by_L": {str(k): v for k, v in sorted(by_L.items())},
            "ms": 1e3 * t_batch, "site_updates_per_s": sites * BATCH_SWEEPS / t_batch,
            "plain_one_chain_per_launch": {"value": n_img / t_plain, "unit": "img/s",
                                           "ms": 1e3 * t_plain,
                                           "site_updates_per_s": sites * BATCH_SWEEPS / t_plain},
            "speedup_vs_plain": t_plain / t_batch,
            "identical_outputs": same, "mean_psnr_db": float(np.mean(psnr)),
            "autotune": info, "fp64_redraw_fraction": fp64 / float(sites * BATCH_SWEEPS)}


def run_batch(a):
    import torch

    import paper_2507_14869_gb300 as pc

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    with ClockSampler(local) as clk:
        obj = _batch_object(pc, torch, stream, a.images, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {"metric": "img/s (batched, 4 chains per image)", "value": obj["value"],
            "unit": "img/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": obj["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": obj["workload"], "chain_sites": obj["chain_sites"]},
            **{k: v for k, v in obj.items() if k not in ("value", "unit", "workload")},
            "gpu_launches": -(-BATCH_SWEEPS // 16) * 17, "clocks": clk.summary()}
    if world > 1:
        line["config"]["parallelism"] = f"images sharded over {world} ranks (LPT by cost)"
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


PROTO_CASES = ((5, 0.25), (9, 0.2), (33, 0.1))   # (levels, sigma in intensity units)


def run_protocol(a):
    """The paper's restoration protocol on synthetic MRF images (its own test
    images are not public): for each (levels, sigma), a 256 x 256 image drawn
    from the Potts prior (J = 1/3, beta 1.5, 200 Gibbs sweeps from random
    levels), Gaussian noise, then annealed 4-colour Gibbs and annealed lazy
    PCA (beta 1.25 + 0.25 per 250 sweeps, 1000 sweeps, q = 0.46, last sample)
    over 3 runs each: PSNR / SSIM and the time of one 1000-sweep run.  Then
    the q grid (14 values x 10 runs, one batch) on the 9-level image, with
    the mean PSNR per q and the count of positive second differences
    (0 = concave)."""
    import numpy as np
    import torch

    import paper_2507_14869_gb300 as pc
    from paper_2507_14869_gb300 import protocol as pr
    from pcad_inputs import gaussian_noise, random_lattice

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    side, J, q, runs = 256, 1.0 / 3.0, 0.46, 3
    cases = []
    grid_case = None
    with ClockSampler(0) as clk:
        for L, sigma in PROTO_CASES:
            clean = pr.mrf_image(random_lattice(100 + L, side, side, L), L, J=J, beta=1.5,
                                 sweeps=200, seed=L, stream=stream)
            noisy = gaussian_noise(200 + L, clean, sigma * (L - 1), L)
            row = {"levels": L, "sigma": sigma, "noisy_psnr_db": pr.metrics(noisy, clean, L)[0]}
            for name, sampler in (("gibbs", pc.SAMPLER_GIBBS_CB), ("pca", pc.SAMPLER_PCA)):
                ms, sw = pr.schedule(L, J, q, sigma, sampler=sampler)
                res, times = [], []
                for r in range(runs + 1):   # run 0 warms up
                    with pc.Chain(noisy, ms[0], seed=7, chain_id=r, burn_in=sum(sw),
                                  stream=stream) as ch:
                        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                        ev[0].record(stream)
                        ch.run_schedule(ms, sw)
                        ev[1].record(stream)
                        torch.cuda.synchronize()
                        if r > 0:
                            times.append(ev[0].elapsed_time(ev[1]))
                            res.append(pr.metrics(ch.sample(), clean, L))
                row[name] = {"psnr_db": float(np.mean([x[0] for x in res])),
                             "ssim": float(np.mean([x[1] for x in res])),
                             "ms_per_run": float(np.mean(times)),
                             "site_updates_per_s": side * side * sum(sw) / (np.mean(times) / 1e3)}
            cases.append(row)
            if L == 9:
                grid_case = (clean, noisy, L, sigma)
        clean, noisy, L, sigma = grid_case
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        grid = pr.q_grid(noisy, clean, L, J, sigma, seed=11, runs=10, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_grid = ev[0].elapsed_time(ev[1]) / 1e3
    curve = [float(np.mean([x[0] for x in grid[qq]])) for qq in pr.Q_GRID]
    chains = len(pr.Q_GRID) * 10
    line = {"metric": "site-updates/s (annealed lazy PCA, paper protocol)",
            "value": float(np.mean([c["pca"]["site_updates_per_s"] for c in cases])),
            "unit": "site-updates/s", "n_gpus": 1, "steps": runs, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic MRF images (Potts prior samples; the paper's images are not "
                    "public)",
            "config": {"workload": f"{side}x{side} MRF images, levels/sigma {PROTO_CASES}, "
                                   "8-nbhd Potts J=1/3, annealed beta 1.25+0.25/250 sweeps, "
                                   "1000 sweeps, q=0.46, last sample"},
            "cases": cases,
            "q_grid": {"levels": 9, "sigma": 0.2, "q": list(pr.Q_GRID), "runs": 10,
                       "mean_psnr_db": curve, "concavity": pr.concavity(curve),
                       "chains": chains, "s_total": t_grid,
                       "site_updates_per_s": chains * side * side * 1000 / t_grid},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def _serve_stream(pc, sv, reqs, slice_sweeps=16):
    """Drive the server with arrivals at their Poisson times; returns
    (latencies s, makespan s, results {index: (sample, mean)})."""
    t0 = time.perf_counter()
    order = sorted(range(len(reqs)), key=lambda i: reqs[i]["arrival"])
    nxt, live, lat, res = 0, {}, {}, {}
    while len(lat) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(order) and reqs[order[nxt]]["arrival"] <= now:
            i = order[nxt]
            j = reqs[i]["job"]
            rid = pc.pcad_server_submit(sv, j.noisy, j.model, j.seed, 0, j.burn_in, j.sweeps)
            live[rid] = i
            nxt += 1
        if not live:
            time.sleep(max(0.0, reqs[order[nxt]]["arrival"] - now))
            continue
        _, _, fin = pc.pcad_server_step(sv, slice_sweeps)
        done_t = time.perf_counter() - t0
        if fin == 0:
            continue
        for rid in list(live):
            i = live[rid]
            st, smp, mean = pc.pcad_server_poll(sv, rid, *reqs[i]["job"].noisy.shape)
            if st == 2:
                lat[i] = done_t - reqs[i]["arrival"]
                res[i] = (smp, mean)
                del live[rid]
    return [lat[i] for i in range(len(reqs))], time.perf_counter() - t0, res


def _plain_service(pc, torch, reqs, stream):
    """Each request alone through the chain API, one after another: its
    service time and result."""
    service, out = [], {}
    for i, r in enumerate(reqs):
        j = r["job"]
        t = time.perf_counter()
        with pc.Chain(j.noisy, j.model, seed=j.seed, chain_id=0, burn_in=j.burn_in,
                      stream=stream) as ch:
            ch.run(j.sweeps)
            out[i] = (ch.sample(), ch.mean())
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t)
    return service, out


def _fifo_latencies(arrivals, service):
    """First come, first served, one request at a time: latency of each
    request and the makespan, from the measured service times."""
    free, lat = 0.0, [0.0] * len(arrivals)
    for i in sorted(range(len(arrivals)), key=lambda k: arrivals[k]):
        start = max(free, arrivals[i])
        free = start + service[i]
        lat[i] = free - arrivals[i]
    return lat, free


def _serve_object(pc, torch, stream, rates, n, seed=50, aging=0.2, shared_rate=50.0):
    """Poisson arrivals of denoising requests (square side log-uniform
    128..2048, L in {16, 256}, sigma uniform [5, 40] on the 0..255 scale,
    300..3000 sweeps, burn-in a quarter, one chain each) through the
    continuous-batching server (150 GB HBM budget, 16-sweep slices), and the
    same requests one at a time through the chain API, first come first
    served.  One request set serves every rate (the arrival times scale with
    1/rate); the one-at-a-time service times are measured once.  Results are
    bit-identical (checked), so PSNR is equal."""
    import numpy as np

    from pcad_inputs import serving_requests
    base = serving_requests(seed=seed, rate=1.0, n=n)
    service, pres = _plain_service(pc, torch, base, stream)
    work = sum(r["job"].noisy.size * r["job"].sweeps for r in base)
    psnr = [pc.pcad_metrics(pres[i][1], r["job"].clean, r["job"].model.L)[0]
            for i, r in enumerate(base)]
    per_rate = []
    for rate in rates:
        reqs = [dict(r, arrival=r["arrival"] / rate) for r in base]
        sv = pc.pcad_server_create(256, 150 * 10 ** 9, stream)
        pc.pcad_server_set_policy(sv, pc.SERVE_SRPT, aging)
        lat, span, res = _serve_stream(pc, sv, reqs)
        info = pc.pcad_server_info(sv)
        pc.pcad_server_destroy(sv)
        same = all(np.array_equal(res[i][0], pres[i][0]) and np.array_equal(res[i][1], pres[i][1])
                   for i in res)
        flat, fspan = _fifo_latencies([r["arrival"] for r in reqs], service)
        row = {
            "rate_req_s": rate, "requests": n, "img_s": n / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": span, "site_updates_per_s": work / span, "slices": info["slices"],
            "plain_fifo": {"img_s": n / fspan, "p50_s": float(np.percentile(flat, 50)),
                           "p99_s": float(np.percentile(flat, 99)), "makespan_s": fspan},
            "identical_outputs": same}
        if rate == shared_rate:
            # the same server sharing the GPU among every admitted request
            sv = pc.pcad_server_create(256, 150 * 10 ** 9, stream)
            pc.pcad_server_set_policy(sv, pc.SERVE_FIFO, 0.0)
            slat, sspan, _ = _serve_stream(pc, sv, reqs)
            pc.pcad_server_destroy(sv)
            row["server_shared_fifo"] = {"img_s": n / sspan,
                                         "p50_s": float(np.percentile(slat, 50)),
                                         "p99_s": float(np.percentile(slat, 99))}
        per_rate.append(row)
    return {"workload": "Poisson requests, side 128..2048 (square), L in {16,256}, sigma "
                        "5..40, 300..3000 sweeps, 150 GB HBM budget, 16-sweep slices",
            "policy": f"shortest remaining work first, aging {aging}",
            "requests_per_rate": n, "capacity_img_s_one_at_a_time": n / sum(service),
            "work_site_updates": work, "mean_psnr_db": float(np.mean(psnr)),
            "per_rate": per_rate}


def run_serve(a):
    """The served form alone (see _serve_object), one JSON line."""
    import torch

    import paper_2507_14869_gb300 as pc

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rates = [float(x) for x in a.rates.split(",") if x]
    with ClockSampler(0) as clk:
        obj = _serve_object(pc, torch, stream, rates, a.requests, aging=a.aging)
    head = obj["per_rate"][-1]
    line = {"metric": "served img/s (continuous batching)", "value": head["img_s"],
            "unit": "img/s", "n_gpus": 1, "steps": len(rates), "warmup": 0,
            "ms_per_step": 1e3 * head["makespan_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": obj["workload"], "rates": rates,
                       "requests_per_rate": a.requests},
            "p50_s": head["p50_s"], "p99_s": head["p99_s"], **obj, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_blocking(a):
    """Large single image, 8192x8192: L = 16 (sigma 1.0) and L = 256 (sigma 25)
    as in the roofline workload, plus the binary flip-noise image; 200 sweeps
    (40 for L = 256) from the observation, burn-in a quarter, run unblocked
    (one launch per sweep) and with k = 1, 2, 4, 8 sweeps per TMA-tiled
    launch.  Outputs are bit-identical across k (checked)."""
    import numpy as np
    import torch

    import paper_2507_14869_gb300 as pc
    from pcad_inputs import Model, flip_noise, large_image, shapes_binary

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    side = 8192
    cases = []
    for L in (16, 256):
        _, noisy, m = large_image(side=side, L=L)
        cases.append((f"L={L}", noisy, m, 200 if L == 16 else 40))
    b = flip_noise(6, shapes_binary(5, side, side, n_shapes=64), 0.1)
    cases.append(("L=2 flip", b, Model(L=2, pair=0, pair_coef=1.2, noise=1, flip_p=0.1,
                                       inertia=1.0), 200))
    rows = {}
    with ClockSampler(0) as clk:
        for name, g, m, n in cases:
            res, ref = {}, None
            for k in (0, 1, 2, 4, 8):
                ch = pc.Chain(g, m, seed=3, chain_id=0, burn_in=n // 4, stream=stream)
                ch.set_blocking(k)
                ch.run(8)
                ch.reset()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ch.run(n)
                e1.record(stream)
                torch.cuda.synchronize()
                ch.sync()
                ms = e0.elapsed_time(e1)
                x = ch.sample()
                same = True if ref is None else bool(np.array_equal(x, ref))
                ref = x if ref is None else ref
                res[f"k={k}" if k else "unblocked"] = {
                    "ms_per_sweep": ms / n, "site_updates_per_s": g.size * n / (ms * 1e-3),
                    "identical": same}
                ch.close()
            rows[name] = {"sweeps": n, "L": m.L, **res}
    best = max(v["site_updates_per_s"] for k, v in rows["L=16"].items() if k.startswith("k="))
    line = {"metric": "site-updates/s (8192^2, best k)", "value": best, "unit": "site-updates/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8192x8192, L=16 sigma 1 / L=256 sigma 25 (c_T 0.05, T 30, "
                                   "lambda 2) and binary flip p=0.1; unblocked vs k sweeps per "
                                   "TMA-tiled launch"},
            "cases": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_cpu_baselines(a):
    """The CPU baseline table: the FP64 oracle on this machine's host cores --
    sequential single-site Gibbs in column-major order (the paper's CPU
    baseline) and lazy PCA single-threaded and with OpenMP over rows (the
    same labels either way) -- for the binary 64x64 chain (500 sweeps, in
    full), the 512x512 L=256 chain (bounded samples, and the full 2000-sweep
    PCA run with OpenMP) and 1024x1024 crops of the 8192x8192 images (5
    sweeps), next to the same chains on the GPU."""
    import numpy as np
    import torch

    import oracle
    import paper_2507_14869_gb300 as pc
    from pcad_inputs import binary_64, greyscale_512

    torch.cuda.set_device(0)
    cores = os.cpu_count()
    omp = oracle.num_threads()

    def orc_rate(fn, sites, sweeps, threads):
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        oracle.set_threads(omp)
        return {"s": dt, "site_updates_per_s": sites * sweeps / dt, "threads": threads,
                "sweeps": sweeps}

    def gpu_wall(g, m, n, burn, sampler=0, reps=3):
        ts = []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with pc.Chain(g, m, seed=1, chain_id=0, burn_in=burn, sampler=sampler) as ch:
                ch.run(n)
                ch.mean()
            if r:
                ts.append(time.perf_counter() - t0)
        return {"s": min(ts), "site_updates_per_s": g.size * n / min(ts),
                "path": "create + run + read mean (wall clock)"}

    rows = {}
    clean, g1, m1 = binary_64()
    rows["binary_64"] = {
        "workload": "64x64 binary, Ising c_P=1.2, flip p=0.1, lambda=1.0, 500 sweeps",
        "gibbs_column_major_1_thread": orc_rate(
            lambda: oracle.run_chain(m1, g1, 500, 100, seed=1, sampler=1, order=oracle.ORDER_COL),
            g1.size, 500, 1),
        "pca_1_thread": orc_rate(lambda: oracle.run_chain(m1, g1, 500, 100, seed=1), g1.size,
                                 500, 1),
        "gpu_pca": gpu_wall(g1, m1, 500, 100), "gpu_gibbs": gpu_wall(g1, m1, 500, 100, 1)}
    clean2, g2, m2 = greyscale_512(seed=2)
    rows["greyscale_512_L256"] = {
        "workload": G512_WORKLOAD,
        "gibbs_column_major_1_thread": orc_rate(
            lambda: oracle.run_chain(m2, g2, 4, 0, seed=2, sampler=1, order=oracle.ORDER_COL),
            g2.size, 4, 1),
        "pca_1_thread": orc_rate(lambda: oracle.run_chain(m2, g2, 4, 0, seed=2), g2.size, 4, 1),
        "pca_openmp_full_2000": orc_rate(lambda: oracle.run_chain(m2, g2, 2000, 500, seed=2),
                                         g2.size, 2000, omp),
        "gpu_pca": gpu_wall(g2, m2, 2000, 500)}
    for L in (16, 256):
        _, g3, m3 = _inputs(L)
        crop = _crop(g3, 1024)
        rows[f"crop_1024_of_8192_L{L}"] = {
            "pca_1_thread": orc_rate(lambda: oracle.run_chain(m3, crop, 5, 0, seed=3), crop.size,
                                     5, 1),
            "pca_openmp": orc_rate(lambda: oracle.run_chain(m3, crop, 5, 0, seed=3), crop.size,
                                   5, omp)}
    print(json.dumps({"metric": "CPU baseline (FP64 oracle) beside the GPU", "cores": cores,
                      "openmp_threads": omp, "rows": rows}), flush=True)


def profile_case(side: int, L: int, sweeps: int, sampler: int, blocking: int = 0,
                 kernel: str = "auto"):
    """Small seeded case for ncu: greyscale scene at L labels (sigma 20 for
    L > 16, else 1), truncated-linear prior c_T 0.05, T 30 (the roofline
    workload's prior), lambda 2.0; L = 2 uses the binary flip-noise scene
    (Ising c_P 1.2, p 0.1, lambda 1.0).  blocking: sweeps per TMA-tiled
    launch."""
    import paper_2507_14869_gb300 as pc
    from pcad_inputs import Model, flip_noise, gaussian_noise, greyscale_scene, shapes_binary
    if L == 2:
        noisy = flip_noise(6, shapes_binary(5, side, side, n_shapes=16), 0.1)
        m = Model(L=2, pair=0, pair_coef=1.2, noise=1, flip_p=0.1, inertia=1.0, sampler=sampler)
    else:
        sig = 20.0 if L > 16 else 1.0
        clean = greyscale_scene(3, side, side, L)
        noisy = gaussian_noise(4, clean, sig, L)
        m = Model(L=L, pair=1, pair_coef=0.05, pair_T=30, sigma=sig, inertia=2.0,
                  sampler=sampler)
    with pc.Chain(noisy, m, seed=1, chain_id=0, burn_in=0) as ch:
        ch.set_blocking(blocking)
        if sampler == 0 or kernel != "auto":
            ch.set_kernel(KERNEL_KINDS[kernel])
        ch.run(sweeps)
        ch.sync()
        print(f"profile case {side}x{side} L={L} sweeps={sweeps} k={blocking} kernel={kernel} "
              f"fp64 re-draws={ch.fp64_draws()}")


def main():
    a = _args()
    if a.profile_case:
        profile_case(*a.profile_case, a.sampler, a.blocking, a.kernel)
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "blocking":
        run_blocking(a)
    elif a.workload == "protocol":
        run_protocol(a)
    elif a.workload == "cpu":
        run_cpu_baselines(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
