"""Benchmark of the curved-ray heat-haze hot path on GB300.

One step = the whole hot path on one frame: splat 262,144 plume particles
onto a 256^3 grid (Sec. 3.3.1), Gladstone-Dale + gradient into the FP32
{dn, grad n} volume (Eqs. 12-13), and the adaptive curved-ray march of one
1920x1080 view (Eqs. 14-18) with the background lookup.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `value` is Mrays/s of whole steps (primary rays over
the device time of splat + field + march, inputs resident in HBM, L2 flushed
between timed steps); `e2e` is the same through the C ABI with the particles
copied from pinned host memory and the image copied back inside the timed
region. `--impl reference` times the FP64 CPU oracle on a bounded sample of
the same workload. N > 1 (torchrun) runs independent replicas, one per GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hh_inputs as hi  # noqa: E402

L = 256
DIMS = (L, L, L)
N_PARTICLES = 262144
WIDTH, HEIGHT = 1920, 1080
THETA = hi.THETA_CALIBRATED
METRIC = "curved-ray Mrays/s (1080p, 256^3, splat+field+march per frame)"
WORKLOAD = ("262,144-particle plume splatted (M4, h=2) onto 256^3, FP32 dn/grad-n volume "
            "(K_GD=2.26e-4), one 1920x1080 view 1.5 grid widths away (60 deg vfov), "
            "Eq. 16 march with Eq. 18 adaptive step h in [0.125, 2], theta_max=3e-5, eps=1e-6")
FLUSH_BYTES = 256 << 20  # > 129 MB L2


def f32(x):
    if isinstance(x, dict):
        return {k: f32(v) for k, v in x.items()}
    if isinstance(x, list):
        return [f32(v) for v in x]
    if isinstance(x, float):
        return float(np.float32(x))
    return x


def scene():
    parts = hi.plume_particles(N_PARTICLES, L)
    cam = f32(hi.orbit_camera(DIMS, 0.0, 0.0, WIDTH, HEIGHT))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=THETA))
    return parts, cam, params, hi.checker_background()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- #
# distributed plumbing (replicas only: barrier and max over ranks)
# --------------------------------------------------------------------------- #
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if _cuda() else "gloo")
        return dist, int(os.environ["RANK"]), world, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _cuda():
    import torch

    return torch.cuda.is_available()


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- #
# clocks during the timed region
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()]
        os.unlink(self.file.name)
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
def run_ours(args):
    import torch

    dist, rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_02048_gb300 import build as hb
    from paper_2603_02048_gb300 import hh

    if rank == 0:
        hb.build()
    barrier(dist)
    hb.build()  # no-op when fresh; makes sure every rank sees the library
    hh.load()

    parts, cam, params, bg = scene()
    parts_t = torch.from_numpy(parts).to(dev)
    bg_t = torch.from_numpy(bg).to(dev)
    grid = hh.make_grid(DIMS, 2.0, "fp32")
    K = float(np.float32(hi.K_GD))
    n_rays = WIDTH * HEIGHT
    rgb = torch.empty(n_rays * 3, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # step statistics (deterministic input -> the same steps every frame)
    vol = hh.hh_build_index_field(parts_t, grid, K)
    steps_t = torch.empty(n_rays, dtype=torch.int32, device=dev)
    flags_t = torch.empty(n_rays, dtype=torch.int32, device=dev)
    hh.hh_trace(vol, [cam], params, bg_t, [{"rgb": rgb, "steps": steps_t, "flags": flags_t}])
    torch.cuda.synchronize()
    total_steps = int(steps_t.sum().item())
    hits = int((flags_t & 1).sum().item())

    def step(src, ev=None):
        hh.hh_volume_rebuild(vol, src, K)
        if ev is not None:
            ev[0].record(stream)
        hh.hh_trace(vol, [cam], params, bg_t, [{"rgb": rgb}])
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step(parts_t)
    torch.cuda.synchronize()

    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    ev_march = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    launches0 = hh.hh_kernel_launch_count()
    with ClockSampler(local) as clocks:
        barrier(dist)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev_step[k][0].record(stream)
            step(parts_t, ev_march[k])
            ev_step[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(dist)
    launches = hh.hh_kernel_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    march_ms = [a.elapsed_time(b) for a, b in ev_march]
    ms_step = max_over_ranks(dist, sum(step_ms) / len(step_ms), dev)
    ms_march = sum(march_ms) / len(march_ms)

    # end to end through the C ABI: pinned host particles in, image out
    host_parts = torch.from_numpy(parts).pin_memory()
    host_rgb = torch.empty(n_rays * 3, dtype=torch.float32).pin_memory()
    dev_parts = torch.empty_like(parts_t)
    e2e_ms = []
    for k in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dev_parts.copy_(host_parts, non_blocking=True)
        step(dev_parts)
        host_rgb.copy_(rgb, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    ms_e2e = max_over_ranks(dist, sum(e2e_ms) / max(len(e2e_ms), 1), dev)
    vol.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    # algorithmic bytes of the march: 8 corners x 16 B per Eq. 16 step, plus
    # per ray 12 B of RGB out and 4 x 3 B of background texels
    march_bytes = total_steps * 128 + n_rays * 24
    achieved = march_bytes / (ms_march * 1e-3) / 1e9
    cpu = cpu_baseline(parts, cam, params, bg) if not args.no_cpu_baseline else None
    line = {
        "metric": METRIC,
        "value": round(world * n_rays / (ms_step * 1e-3) / 1e6, 3),
        "unit": "Mrays/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded plume particles, checker+noise equirect background)",
        "config": {"workload": WORKLOAD, "rays_per_step": n_rays, "rays_hit": hits,
                   "march_steps_per_frame": total_steps,
                   "steps_per_hit_ray": round(total_steps / max(hits, 1), 2),
                   "march_ms": round(ms_march, 4),
                   "build_ms": round(ms_step - ms_march, 4),
                   "march_Mrays_s": round(n_rays / (ms_march * 1e-3) / 1e6, 3),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": None if args.no_e2e else {
            "value": round(world * n_rays / (ms_e2e * 1e-3) / 1e6, 3), "unit": "Mrays/s",
            "ms_per_step": round(ms_e2e, 4), "h2d_bytes_per_step": int(parts.nbytes),
            "d2h_bytes_per_step": int(n_rays * 3 * 4)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "march_kernel<FP32, EULER_PAPER, adaptive>",
                     "peak_kind": peak_kind,
                     "algorithmic_bytes": int(march_bytes)},
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- #
# the oracle (CPU baseline and reference arm)
# --------------------------------------------------------------------------- #
def oracle_frame_seconds(parts, cam, params, bg, frac: int, nthreads: int, full_vol=None):
    """FP64 oracle time of one frame, measured on a 1/frac sample of each
    stage and scaled up: splat of every frac-th particle, Gladstone-Dale +
    gradient of a 1/frac slab of the grid, the march of every frac-th pixel
    (on the full oracle volume)."""
    import oracle

    t0 = time.perf_counter()
    rho = oracle.splat(parts[::frac], DIMS, 2.0)
    t1 = time.perf_counter()
    slab = max(2, L // frac)
    oracle.index_field(rho[:slab], float(np.float32(hi.K_GD)))
    t2 = time.perf_counter()
    if full_vol is None:
        full_vol = oracle.index_field(oracle.splat(parts, DIMS, 2.0), float(np.float32(hi.K_GD)))
    pix = np.arange(0, WIDTH * HEIGHT, frac, dtype=np.int64)
    t3 = time.perf_counter()
    oracle.trace_grid(full_vol, cam, params, bg, pixels=pix, nthreads=nthreads)
    t4 = time.perf_counter()
    per_frame = frac * (t1 - t0) + (L / slab) * (t2 - t1) + frac * (t4 - t3)
    return per_frame, full_vol, (t1 - t0) + (t2 - t1) + (t4 - t3)


def cpu_baseline(parts, cam, params, bg):
    import oracle

    oracle.build()
    nthreads = os.cpu_count() or 1
    frac = 1
    sec, _, worked = oracle_frame_seconds(parts, cam, params, bg, frac, nthreads)
    return {"value": round(WIDTH * HEIGHT / sec / 1e6, 4), "unit": "Mrays/s",
            "cores": nthreads, "kind": "oracle",
            "sample": (f"one whole frame: all particles splatted (1 thread), the whole grid "
                       f"through Gladstone-Dale (1 thread), every pixel marched ({nthreads} "
                       f"threads); {worked:.1f} s measured"),
            "ms_per_frame": round(sec * 1e3, 1)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    parts, cam, params, bg = scene()
    nthreads = os.cpu_count() or 1
    frac = 16
    full_vol = None
    times = []
    for k in range(args.warmup + args.steps):
        sec, full_vol, _ = oracle_frame_seconds(parts, cam, params, bg, frac, nthreads, full_vol)
        if k >= args.warmup:
            times.append(sec)
    ms = 1e3 * sum(times) / len(times)
    value = round(WIDTH * HEIGHT / (ms * 1e-3) / 1e6, 4)
    sample = (f"per step 1/{frac} of each stage (every {frac}th particle, 1/{frac} of the grid, "
              f"every {frac}th pixel), scaled to one frame")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
