"""Benchmark: lazy-PCA denoising chain on one GB300 (plus Gibbs on the same GPU).

Workload (one "step"): the greyscale 512x512 chain with L = 256 labels --
smooth gradients plus 20 rectangles/disks, additive Gaussian noise sigma = 20
(clipped, rounded), truncated-linear prior c_T = 0.05, T = 30 on the
4-neighbourhood, inertia lambda = 2.0; 2000 lazy-PCA sweeps from the
observation with burn-in 500 and the FP32 posterior-mean accumulator.
Synthetic, seeded inputs (the paper's images are not public).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  `value` is site-updates/s with the inputs resident in
HBM (CUDA events on the chain's stream, L2 flushed between steps); `e2e` is
the same metric through the public C ABI with host buffers (create from
pinned host memory, run, read the mean back).  `--impl reference` times the
FP64 CPU oracle on the host cores on bounded samples of the same workload.
Under torchrun each rank runs its own independent chain (weak scaling).
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

SWEEPS = 2000
BURN_IN = 500
WORKLOAD = ("greyscale 512x512, L=256 (uint8), Gaussian sigma=20, truncated-linear "
            "c_T=0.05 T=30 4-nbhd, lambda=2.0, 2000 sweeps, burn-in 500, FP32 posterior mean")
# SFU ex2 issue: 32 per SM per clock (4 SM sub-partitions x 8) x 152 SMs x 2070 MHz
SFU_PEAK_T = 152 * 32 * 2.070e9 / 1e12
# DRAM bytes (read + write) per site of one pca_direct_kernel<32,4> launch,
# from the ncu capture in profiles/pca_direct_l256_1024sq.md (6.33 MB over
# 1024^2 sites), scaled by the sites of a 512^2 launch.  Set to None when the
# kernel changes until it is captured again.
NCU_DRAM_BYTES_PER_SITE = 6.326784e6 / (1024 * 1024)
NCU_TRAFFIC_NOTE = ("ncu dram__bytes_read+write of the 1024^2 L=256 launch scaled by sites; "
                    "the working set is L2-resident, so DRAM traffic is below the 3-11 B/site "
                    "the sweep touches")


# The same for pca_tcw_kernel<4,0,0,0> (one 32-sweep launch at 512^2,
# profiles/pca_tc_l256_512sq.md) and pca_wave_kernel<32,4> (one 32-sweep
# launch at 1024^2, per site-update).
NCU_TC_DRAM_BYTES_PER_SITE = (1.637888e6 + 0.122880e6) / (32 * 512 * 512)
NCU_TC_TRAFFIC_NOTE = ("ncu dram__bytes_read+write of one 32-sweep launch at 512^2 L=256 (sweeps "
                       "161-192 of a chain): the chain's planes stay in L2")
NCU_WAVE_DRAM_BYTES_PER_SITE = (6.372096e6 + 0.761856e6) / (32 * 1024 * 1024)
NCU_WAVE_TRAFFIC_NOTE = ("ncu dram__bytes_read+write of one 32-sweep launch at 1024^2 L=256, "
                         "scaled by sites to a 512^2 launch (profiles/pca_wave_l256_1024sq.md)")

KERNEL_KINDS = {"auto": 0, "cuda_core": 1, "tensor": 2, "wave": 3}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-gibbs", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--profile-case", nargs=3, type=int, metavar=("SIDE", "L", "SWEEPS"),
                   help="run one SIDE x SIDE chain with L labels for SWEEPS sweeps and exit "
                        "(the small case ncu captures; prints no JSON line)")
    p.add_argument("--sampler", type=int, default=0, help="profile case: 0 PCA, 1 Gibbs")
    p.add_argument("--blocking", type=int, default=0,
                   help="profile case: sweeps per TMA-tiled launch (0: unblocked)")
    p.add_argument("--workload", default="chain",
                   choices=["chain", "batch", "serve", "blocking", "protocol"],
                   help="chain: the 512x512 L=256 chain (default); batch: uneven images x 4 "
                        "chains in one persistent launch vs one chain per launch; serve: "
                        "Poisson request stream through the continuous-batching server; "
                        "protocol: the paper's annealed runs on MRF images and the q grid")
    p.add_argument("--kernel", default="auto", choices=["auto", "cuda_core", "tensor", "wave"],
                   help="kernel of the unblocked PCA sweep (chain workload and profile case): "
                        "auto = cuda_core; tensor = prior sums by tcgen05.mma")
    p.add_argument("--images", type=int, default=128, help="batch: number of images")
    p.add_argument("--requests", type=int, default=24, help="serve: requests per rate")
    p.add_argument("--rates", default="2,50", help="serve: comma-separated arrival rates (req/s)")
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


def _inputs():
    from pcad_inputs import greyscale_512
    return greyscale_512(seed=2)


def cpu_baseline(seconds: float = 12.0):
    """FP64 oracle PCA sweeps of the 512x512 L=256 image on all host cores."""
    import oracle
    clean, noisy, m = _inputs()
    x = noisy.copy()
    t0 = time.perf_counter()
    n = 0
    while True:
        x, _ = oracle.pca_sweep(m, noisy, x, 2, 0, n)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 64:
            break
    dt = time.perf_counter() - t0
    H, W = noisy.shape
    return {"value": H * W * n / dt, "unit": "site-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{n} lazy-PCA sweeps of the 512x512 L=256 image "
                                        f"({dt:.1f} s, OpenMP over rows)"}


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    clean, noisy, m = _inputs()
    H, W = noisy.shape
    x = noisy.copy()
    for t in range(a.warmup):
        x, _ = oracle.pca_sweep(m, noisy, x, 2, 0, t)
    times = []
    for k in range(a.steps):
        t0 = time.perf_counter()
        x, _ = oracle.pca_sweep(m, noisy, x, 2, 0, a.warmup + k)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    v = H * W * a.steps / T
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": "site-updates/s", "value": v,
            "unit": "site-updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * T / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "one lazy-PCA sweep of the full image "
                                                    "(bounded sample of the 2000-sweep chain)"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v,
                             "sample": f"{a.steps} sweeps of the 512x512 L=256 image"},
            "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(chain, steps, warm):
        for _ in range(warm):
            chain.reset().run(SWEEPS)
        chain.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(k & 0xFF)              # L2 flush between timed steps
                evs[k][0].record(stream)
                chain.reset().run(SWEEPS)
                evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        wall = time.perf_counter() - wall0
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        return ms, wall

    kind = KERNEL_KINDS[a.kernel]
    pca = pc.Chain(noisy, m, seed=2, chain_id=cid, burn_in=BURN_IN, stream=stream)
    pca.set_kernel(kind)
    pca_kind = pca.kernel_in_use()
    with ClockSampler(local) as clk:
        ms, wall = timed(pca, a.steps, a.warmup)
    T = sum(ms) / 1e3
    T_max = replicas.max_time(T)   # the slowest rank's time
    sites = H * W * SWEEPS
    value = world * sites * a.steps / T_max
    launch_ms = 1e3 * T / (a.steps * SWEEPS)
    fp64 = pca.fp64_draws()
    psnr, ssim = pca.metrics(clean, 0)
    pca_sample_psnr, _ = pca.metrics(clean, 1)

    gibbs = None
    if not a.no_gibbs:
        gch = pc.Chain(noisy, m, seed=2, chain_id=cid, burn_in=BURN_IN, stream=stream,
                       sampler=pc.SAMPLER_GIBBS_CB)
        gsteps = max(2, a.steps // 2)
        gms, _ = timed(gch, gsteps, 1)
        gT = sum(gms) / 1e3
        gp, gs = gch.metrics(clean, 0)
        g_tc = gch.kernel_in_use() == pc.PCAD_KERNEL_TENSOR
        gblocks = (SWEEPS + 31) // 32
        gibbs = {"value": sites * gsteps / gT, "unit": "site-updates/s",
                 "ms_per_step": 1e3 * gT / gsteps, "steps": gsteps, "psnr_db": gp, "ssim": gs,
                 # per 32-sweep graph: the wavefront launch (or 2 colour-phase launches per
                 # sweep), the counter reset and the sweep-counter advance
                 "launches_per_step": gblocks * 2 if g_tc else 2 * SWEEPS + gblocks,
                 "kernel": ("pca_tcw_kernel<4,0,0,0,1> (checkerboard Gibbs on the tensor-core "
                            "wavefront, 2 colour phases per sweep)") if g_tc else
                           "gibbs_cb_kernel<32,4> (2 colour phases per sweep)"}
        gch.close()

    # end to end through the public API with host buffers (pinned)
    g_host = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
    g_host.numpy()[:] = noisy
    mean_host = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(2, min(a.steps, 5))
    torch.cuda.synchronize(dev)
    e2e_t = []
    for k in range(e2e_steps + 1):
        t0 = time.perf_counter()
        ch = pc.Chain(g_host.numpy(), m, seed=2, chain_id=cid, burn_in=BURN_IN, stream=stream)
        ch.set_kernel(kind)
        ch.run(SWEEPS)
        pc.pcad_chain_read_mean(ch.h, H, W, out=mean_host.numpy())
        ch.close()
        if k > 0:                                     # first one warms the allocator
            e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * sites / statistics.mean(e2e_t)

    if rank != 0:
        return
    per_sweep_labels = H * W * m.L
    achieved = per_sweep_labels / (launch_ms * 1e-3) / 1e12
    in_use = pca_kind   # the kernel the timed chain ran
    kernel_name = {1: "pca_direct_kernel<32,4> (one launch per sweep)",
                   2: "pca_tcw_kernel<4,0,0,0> (tcgen05 windowed tent sums, CUDA-core CDF, "
                      "wavefront, one launch per 32 sweeps)",
                   3: "pca_wave_kernel<32,4> (wavefront, one launch per 32 sweeps)"}[in_use]
    per_site = {1: NCU_DRAM_BYTES_PER_SITE, 2: NCU_TC_DRAM_BYTES_PER_SITE,
                3: NCU_WAVE_DRAM_BYTES_PER_SITE}[in_use]
    note = {1: NCU_TRAFFIC_NOTE, 2: NCU_TC_TRAFFIC_NOTE, 3: NCU_WAVE_TRAFFIC_NOTE}[in_use]
    # per launch, like achieved: 32 sweeps per wavefront launch, one otherwise
    sweeps_per_launch = 32 if in_use in (2, 3) else 1
    traffic = per_site * H * W * sweeps_per_launch if per_site else None
    blocks, rest = divmod(SWEEPS, 32)
    # per chain: the 32-sweep graphs (sweep launches + the counter advance) and the rest
    wave = in_use in (2, 3)   # one launch per block of sweeps + the advance
    launches = (blocks * (2 if wave else 33) + ((2 if wave else rest + 1) if rest else 0))
    line = {
        "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * T_max / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": H * W, "sweeps_per_step": SWEEPS,
                   "burn_in": BURN_IN, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "independent chain per GPU" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": SFU_PEAK_T,
                     "unit": "T ex2/s", "frac": achieved / SFU_PEAK_T,
                     "traffic": traffic, "traffic_source": note,
                     "traffic_unit": f"DRAM bytes per launch ({sweeps_per_launch} sweeps of "
                                     f"{H}x{W})",
                     # 1 B label + 1 B observation in, 1 B label + 8 B accumulator RMW
                     # after burn-in per site-update
                     "algorithmic_bytes_per_launch": 11 * H * W * sweeps_per_launch,
                     "kernel": kernel_name,
                     "work_per_unit": "one label evaluation (one exponential on the SFU in "
                                      "a direct evaluation), L=256 per site-update; the "
                                      "tensor-core kernel takes the chunk sums outside a "
                                      "site's 128-label window from a table, so it evaluates "
                                      "fewer exponentials than labels",
                     "peak_source": "152 SMs x 32 ex2/clk/SM x 2070 MHz (unit count x max "
                                    "clock; 29.9/clk/SM measured)",
                     "ms_per_sweep": launch_ms},
        "gpu_launches": a.steps * launches,
        "e2e": {"value": e2e_v, "unit": "site-updates/s", "h2d_bytes_per_step": H * W,
                "d2h_bytes_per_step": H * W * 4, "steps": e2e_steps,
                "ms_per_step": 1e3 * statistics.mean(e2e_t),
                "path": "pcad_chain_create(host) + pcad_chain_run + pcad_chain_read_mean(host)"},
        "label_evals_per_s": value * m.L,
        "fp64_redraw_fraction": fp64 / float(H * W * SWEEPS),   # counter restarts each step
        "psnr_db": psnr, "ssim": ssim, "last_sample_psnr_db": pca_sample_psnr,
        "wall_s_timed": wall,
    }
    if gibbs:
        line["gibbs"] = gibbs
    clocks = clk.summary()
    line["clocks"] = clocks
    if world == 1 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


BATCH_SWEEPS, BATCH_BURN = 200, 50


def run_batch(a):
    """Uneven images (short side log-uniform 64..2048, aspect 1..3, L in
    {2, 16, 256}, per-image prior/inertia), 4 chains each, 200 sweeps with
    burn-in 50: one persistent launch per sweep for all chains, against the
    same chains run one after another through the chain API on the same GPU.
    Outputs are bit-identical, so PSNR is equal by construction (checked)."""
    import numpy as np
    import torch

    import paper_2507_14869_gb300 as pc
    from paper_2507_14869_gb300 import replicas
    from pcad_inputs import batched_jobs

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    all_imgs = batched_jobs(seed=4, n_images=a.images, chains=4, sweeps=BATCH_SWEEPS,
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
    pc.pcad_batch_run(b, 16)
    pc.pcad_batch_reset(b)
    pc.pcad_batch_sync(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        pc.pcad_batch_run(b, BATCH_SWEEPS)
        ev[1].record(stream)
        torch.cuda.synchronize()
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
        k = 4 * i
        psnr.append(chains[k].metrics(j.clean, 0)[0])
    for ch in chains:
        ch.close()
    pc.pcad_batch_destroy(b)
    # whole job: every rank's images over the slowest rank's time
    t_batch_all = replicas.max_time(t_batch)
    t_plain_all = replicas.max_time(t_plain)
    sites_all = replicas.gather({rank: sites})
    psnr_all = replicas.gather({rank: psnr})
    same_all = replicas.gather({rank: same})
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    n_img = len(all_imgs)
    sites = sum(sites_all.values())
    psnr = [v for r in sorted(psnr_all) for v in psnr_all[r]]
    same = all(same_all.values())
    t_batch, t_plain = t_batch_all, t_plain_all
    line = {"metric": "img/s (batched, 4 chains per image)", "value": n_img / t_batch,
            "unit": "img/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * t_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n_img} uneven images x 4 chains, {BATCH_SWEEPS} sweeps, "
                                   f"burn-in {BATCH_BURN}", "chain_sites": sites,
                       "sites_by_L": {str(k): v for k, v in sorted(by_L.items())}},
            "site_updates_per_s": sites * BATCH_SWEEPS / t_batch,
            "plain_one_chain_per_launch": {"value": n_img / t_plain, "unit": "img/s",
                                           "ms": 1e3 * t_plain,
                                           "site_updates_per_s": sites * BATCH_SWEEPS / t_plain},
            "speedup_vs_plain": t_plain / t_batch,
            "identical_outputs": same, "mean_psnr_db": float(np.mean(psnr)),
            "autotune": info, "fp64_redraw_fraction": fp64 / float(sites * BATCH_SWEEPS),
            "gpu_launches": -(-BATCH_SWEEPS // 16) * 17,
            "clocks": clk.summary()}
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
        pc.pcad_server_step(sv, slice_sweeps)
        done_t = time.perf_counter() - t0
        for rid in list(live):
            i = live[rid]
            st, smp, mean = pc.pcad_server_poll(sv, rid, *reqs[i]["job"].noisy.shape)
            if st == 2:
                lat[i] = done_t - reqs[i]["arrival"]
                res[i] = (smp, mean)
                del live[rid]
    return [lat[i] for i in range(len(reqs))], time.perf_counter() - t0, res


def _plain_fifo(pc, reqs, stream):
    """The same requests one at a time through the chain API, first come first
    served: each request's service time is measured alone; latency is the
    queueing simulation over the real arrival times."""
    import torch
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
    free, lat = 0.0, []
    for i in sorted(range(len(reqs)), key=lambda k: reqs[k]["arrival"]):
        start = max(free, reqs[i]["arrival"])
        free = start + service[i]
        lat.append((i, free - reqs[i]["arrival"]))
    lat = [v for _, v in sorted(lat)]
    return lat, free, out, sum(service)


def run_serve(a):
    """Poisson arrivals of denoising requests (square side log-uniform
    128..2048, L in {16, 256}, sigma uniform [5, 40] on the 0..255 scale,
    300..3000 sweeps, burn-in a quarter, one chain each) through the
    continuous-batching server with a 150 GB HBM budget; the same stream one
    request at a time through the chain API is the comparison.  Results are
    bit-identical (checked), so PSNR is equal."""
    import numpy as np
    import torch

    import paper_2507_14869_gb300 as pc
    from pcad_inputs import serving_requests

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rates = [float(x) for x in a.rates.split(",") if x]
    per_rate = []
    with ClockSampler(0) as clk:
        for k, rate in enumerate(rates):
            reqs = serving_requests(seed=50 + k, rate=rate, n=a.requests)
            sv = pc.pcad_server_create(256, 150 * 10 ** 9, stream)
            lat, span, res = _serve_stream(pc, sv, reqs)
            info = pc.pcad_server_info(sv)
            pc.pcad_server_destroy(sv)
            # the same stream with admission capped at 2M sites of admitted work
            sv = pc.pcad_server_create(256, 150 * 10 ** 9, stream)
            pc.pcad_server_set_limits(sv, 2 << 20)
            clat, cspan, _ = _serve_stream(pc, sv, reqs)
            pc.pcad_server_destroy(sv)
            plat, pspan, pres, busy = _plain_fifo(pc, reqs, stream)
            same = all(np.array_equal(res[i][0], pres[i][0]) and
                       np.array_equal(res[i][1], pres[i][1]) for i in res)
            work = sum(r["job"].noisy.size * r["job"].sweeps for r in reqs)
            psnr = [pc.pcad_metrics(res[i][1], reqs[i]["job"].clean, reqs[i]["job"].model.L)[0]
                    for i in range(min(4, len(reqs)))]
            per_rate.append({
                "rate_req_s": rate, "requests": len(reqs),
                "img_s": len(reqs) / span, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "makespan_s": span,
                "site_updates_per_s": work / span, "slices": info["slices"],
                "plain": {"img_s": len(reqs) / pspan, "p50_s": float(np.percentile(plat, 50)),
                          "p99_s": float(np.percentile(plat, 99)), "busy_s": busy},
                "capped_2M_sites": {"img_s": len(reqs) / cspan,
                                    "p50_s": float(np.percentile(clat, 50)),
                                    "p99_s": float(np.percentile(clat, 99))},
                "identical_outputs": same, "psnr_db_first": psnr})
    head = per_rate[-1]
    line = {"metric": "served img/s (continuous batching)", "value": head["img_s"],
            "unit": "img/s", "n_gpus": 1, "steps": len(rates), "warmup": 0,
            "ms_per_step": 1e3 * head["makespan_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Poisson requests, side 128..2048, L in {16,256}, "
                                   "300..3000 sweeps, 150 GB HBM budget, 16-sweep slices",
                       "rates": rates, "requests_per_rate": a.requests},
            "p50_s": head["p50_s"], "p99_s": head["p99_s"], "per_rate": per_rate,
            "clocks": clk.summary()}
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


def profile_case(side: int, L: int, sweeps: int, sampler: int, blocking: int = 0,
                 kernel: str = "auto"):
    """Small seeded case for ncu: greyscale scene at L labels (sigma 20 for
    L > 16, else 1), truncated-linear prior (c_T 0.05, T 30 for L > 16; 0.85,
    2 otherwise), lambda 2.0; L = 2 uses the binary flip-noise scene (Ising
    c_P 1.2, p 0.1, lambda 1.0).  blocking: sweeps per TMA-tiled launch."""
    import paper_2507_14869_gb300 as pc
    from pcad_inputs import Model, flip_noise, gaussian_noise, greyscale_scene, shapes_binary
    if L == 2:
        noisy = flip_noise(6, shapes_binary(5, side, side, n_shapes=16), 0.1)
        m = Model(L=2, pair=0, pair_coef=1.2, noise=1, flip_p=0.1, inertia=1.0, sampler=sampler)
    else:
        sig = 20.0 if L > 16 else 1.0
        clean = greyscale_scene(3, side, side, L)
        noisy = gaussian_noise(4, clean, sig, L)
        m = Model(L=L, pair=1, pair_coef=0.05 if L > 16 else 0.85, pair_T=30 if L > 16 else 2,
                  sigma=sig, inertia=2.0, sampler=sampler)
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
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
