"""Benchmark of the curved-ray heat-haze hot path on GB300.

One step = the whole hot path on one frame: splat 262,144 plume particles
onto a 256^3 grid (Sec. 3.3.1), Gladstone-Dale + gradient into the FP32
{dn, grad n} volume (Eqs. 12-13), and the adaptive curved-ray march of one
1920x1080 view (Eqs. 14-18) with the background lookup.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload frame|precision|batch|serve]

--workload precision / batch time the FP16 multi-view configurations (8 views
of 1280x720 on the 256^3 scene; 32 uneven views on a 512^3 volume from
2,097,152 particles) through the persistent batched launch, and add the same
views' per-view and plain FP32 single-view march rates for comparison;
--workload serve drives the render server with Poisson request streams.

Prints one JSON line. `value` is Mrays/s of whole steps (primary rays over
the device time of splat + field + march, inputs resident in HBM, L2 flushed
between timed steps); `e2e` is the same end to end through the C ABI with
host buffers (the frame pipeline: particles from pinned host memory in, every
view's RGB8 image back, two frames in flight), with the one-frame-at-a-time
measurement beside it. `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload. N > 1 (torchrun) runs independent
replicas, one per GPU.
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

FLUSH_BYTES = 256 << 20  # > 129 MB L2
METRIC = "curved-ray Mrays/s (1080p, 256^3, splat+field+march per frame)"
K_GD32 = float(np.float32(hi.K_GD))


def f32(x):
    if isinstance(x, dict):
        return {k: f32(v) for k, v in x.items()}
    if isinstance(x, list):
        return [f32(v) for v in x]
    if isinstance(x, float):
        return float(np.float32(x))
    return x


# The workloads. "frame" is the headline (the default); the others are the
# FP16 multi-view precision configuration and the 32-view batching one.
WORKLOADS = {
    "frame": {
        "L": 256, "particles": 262144, "storage": "fp32", "views": "single", "mode": "trace",
        "metric": METRIC,
        "text": ("262,144-particle plume splatted (M4, h=2) onto 256^3, FP32 dn/grad-n volume "
                 "(K_GD=2.26e-4), one 1920x1080 view 1.5 grid widths away (60 deg vfov), "
                 "Eq. 16 march with Eq. 18 adaptive step h in [0.125, 2], theta_max=3e-5, "
                 "eps=1e-6")},
    "precision": {
        "L": 256, "particles": 262144, "storage": "fp16", "views": "arc8", "mode": "batch",
        "metric": "curved-ray Mrays/s (8 x 1280x720 arc, 256^3 FP16, splat+field+march)",
        "text": ("the 256^3 plume with dn/grad-n stored FP16 with per-volume scales, 8 views "
                 "1280x720 evenly over a 90 deg arc, one persistent batched launch "
                 "(autotuned, CUDA graph), Eq. 16 adaptive, theta_max=3e-5")},
    "batch": {
        "L": 512, "particles": 2097152, "storage": "fp16", "views": "mix32", "mode": "batch",
        "metric": "curved-ray Mrays/s (32 uneven views, 512^3 FP16, splat+field+march)",
        "text": ("2,097,152-particle plume -> 512^3 FP16 dn/grad-n volume, 32 views of uneven "
                 "resolution (256^2 .. 1920x1080, seeded mix, eyes 1.5 grid widths away), one "
                 "persistent batched launch (autotuned, CUDA graph), Eq. 16 adaptive, "
                 "theta_max=3e-5")},
}


SERVE = {
    "L": 384, "particles": 1048576, "frames": 60, "duration_s": 2.0, "rates": (25, 50, 100, 200),
    "metric": "serving Mrays/s with p50/p99 latency (Poisson requests of 1-16 views, 384^3 FP16)",
    "text": ("60 device-resident 384^3 FP16 volumes of a drifting 1,048,576-particle plume "
             "(one per sim frame, 30 Hz); Poisson arrivals over 2 s, each request 1-16 views "
             "(uniform) at resolutions from {320x240, 1280x720, 1920x1080, 3840x2160}, eyes "
             "1.5 grid widths away; each returns its rgb8 display images; continuous "
             "batching over 8 slot streams, 16 GiB output budget; Eq. 16 adaptive, "
             "theta_max=3e-5")}


def scene(wl: dict):
    L = wl["L"]
    dims = (L, L, L)
    parts = hi.plume_particles(wl["particles"], L)
    if wl["views"] == "single":
        cams = [hi.orbit_camera(dims, 0.0, 0.0, 1920, 1080)]
    elif wl["views"] == "arc8":
        cams = hi.arc_cameras(dims, n=8, width=1280, height=720)
    else:
        cams = hi.view_mix(dims, n=32)
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    return dims, parts, f32(cams), params, hi.checker_background()


def steps_distribution(outs):
    """Quantiles of the Eq. 16 step count over the rays that entered the volume
    (outs: per-view dicts with device 'steps' and 'flags')."""
    import torch

    st = torch.cat([o["steps"][(o["flags"] & 1) != 0] for o in outs]).cpu().numpy()
    if st.size == 0:
        return None
    q = np.percentile(st, [1, 10, 50, 90, 99])
    return {"mean": round(float(st.mean()), 2), "p1": float(q[0]), "p10": float(q[1]),
            "p50": float(q[2]), "p90": float(q[3]), "p99": float(q[4]), "max": int(st.max())}


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

        backend = os.environ.get("HH_DIST_BACKEND") or ("nccl" if _cuda() else "gloo")
        dist.init_process_group(backend)
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
        if getattr(self, "_summary", None) is not None:
            return self._summary
        self._summary = self._read()
        return self._summary

    def _read(self):
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
# FP32 operations of one Eq. 16 adaptive step as written in the march kernel
# (an FMA counts 2): lattice coordinates 6, trilinear weights 15, the 8-corner
# accumulation 60, n 1, w 3, g_perp and its norm 17, Eq. 18 step 4, ds/n 2,
# Eq. 16 update 6, renormalisation 20, position increment 6, compensated
# position 18.
FLOPS_PER_STEP = 158


def issue_rate(workload: str, ms_march: float, clocks: dict):
    """What bounds the march in practice: warp instructions issued per second
    (the committed ncu count per launch over the event-timed launch) against
    the issue peak of 152 SMs x 4 schedulers x 1 warp-instruction per cycle at
    the median SM clock sampled during the run; None without a count for the
    current source."""
    inst = march_counters(workload).get("warp_instructions_per_launch")
    mhz = (clocks or {}).get("sm_mhz")
    if not inst or not mhz or not ms_march:
        return None
    achieved = inst / (ms_march * 1e-3) / 1e9
    peak = 152 * 4 * mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions_per_launch": int(inst)}


def march_counters(workload: str) -> dict:
    """Counters of one march launch from the committed ncu capture (DRAM bytes,
    warp instructions), or {} when the march source has changed since they
    were taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "march_traffic.json")
    src = os.path.join(ROOT, "paper_2603_02048_gb300", "csrc", "march.cu")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        rec = json.load(f)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("march_cu_sha256") != sha:
        return {}
    return rec.get("workloads", {}).get(workload, {})


def traffic_for(workload: str):
    """DRAM bytes per march launch from the committed ncu capture, or None
    when the march source has changed since the counters were taken."""
    return march_counters(workload).get("dram_bytes_per_launch")

    path = os.path.join(ROOT, "profiles", "march_traffic.json")
    src = os.path.join(ROOT, "paper_2603_02048_gb300", "csrc", "march.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("march_cu_sha256") != sha:
        return None
    w = rec.get("workloads", {}).get(workload)
    return None if w is None else w.get("dram_bytes_per_launch")


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

    wl = WORKLOADS[args.workload]
    dims, parts, cams, params, bg = scene(wl)
    parts_t = torch.from_numpy(parts).to(dev)
    bg_t = torch.from_numpy(bg).to(dev)
    grid = hh.make_grid(dims, 2.0, wl["storage"])
    n_rays = sum(c["width"] * c["height"] for c in cams)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()  # inputs are on the device before any other stream uses them
    stream = torch.cuda.Stream(device=dev) if wl["mode"] == "batch" else \
        torch.cuda.current_stream(dev)
    vol = hh.hh_build_index_field(parts_t, grid, K_GD32, stream)

    # step statistics (deterministic input -> the same steps every frame)
    stats = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device=dev),
              "steps": torch.empty(c["width"] * c["height"], dtype=torch.int32, device=dev),
              "flags": torch.empty(c["width"] * c["height"], dtype=torch.int32, device=dev)}
             for c in cams]
    with torch.cuda.stream(stream):
        hh.hh_trace(vol, cams, params, bg_t, stats, stream)
    torch.cuda.synchronize()
    total_steps = sum(int(o["steps"].sum().item()) for o in stats)
    hits = sum(int((o["flags"] & 1).sum().item()) for o in stats)
    steps_dist = steps_distribution(stats)
    # the paper's theta_max = 3e-3 on the same volume and views (the schedule
    # at which Eq. 18 keeps every step at h_max on this scene), frame only
    theta_paper = None
    if args.workload == "frame" and not args.no_compare:
        p_paper = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_PAPER))
        with torch.cuda.stream(stream):
            hh.hh_trace(vol, cams, p_paper, bg_t, stats, stream)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(10)]
            for e0, e1 in evs:
                flush.zero_()
                e0.record(stream)
                hh.hh_trace(vol, cams, p_paper, bg_t, stats, stream)
                e1.record(stream)
        torch.cuda.synchronize()
        ms_paper = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
        theta_paper = {"theta_max": hi.THETA_PAPER, "march_ms": round(ms_paper, 4),
                       "march_Mrays_s": round(n_rays / (ms_paper * 1e-3) / 1e6, 3),
                       "steps_per_hit_ray": steps_distribution(stats)}
    outs = [{"rgb": o["rgb"]} for o in stats]
    del stats

    batch = None
    tuned = None
    if wl["mode"] == "batch":
        batch = hh.hh_batch_create(vol, cams, params, bg_t, outs)
        with torch.cuda.stream(stream):
            tuned = hh.hh_batch_autotune(batch, reps=3, stream=stream)

    def march():
        if batch is not None:
            hh.hh_batch_launch_graph(batch, stream)
        else:
            hh.hh_trace(vol, cams, params, bg_t, outs, stream)

    def step(src, ev=None):
        hh.hh_volume_rebuild(vol, src, K_GD32, stream)
        if ev is not None:
            ev[0].record(stream)
        march()
        if ev is not None:
            ev[1].record(stream)

    with torch.cuda.stream(stream):
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
        with torch.cuda.stream(stream):
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

    # end to end one frame at a time (reported as e2e.serial): pinned host
    # particles in, the display images (rgb8: what a viewer shows) out, every
    # step, each step synchronised and timed with CUDA events
    host_parts = torch.from_numpy(parts).pin_memory()
    outs8 = [{"rgb8": torch.empty(o["rgb"].numel(), dtype=torch.uint8, device=dev)} for o in outs]
    host_rgb8 = [torch.empty(o["rgb8"].numel(), dtype=torch.uint8).pin_memory() for o in outs8]
    dev_parts = torch.empty_like(parts_t)
    batch8 = None
    if batch is not None and not args.no_e2e:
        batch8 = hh.hh_batch_create(vol, cams, params, bg_t, outs8)
        hh.hh_batch_set_config(batch8, **tuned)
    e2e_ms = []
    with torch.cuda.stream(stream):
        for k in range(0 if args.no_e2e else args.warmup + args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dev_parts.copy_(host_parts, non_blocking=True)
            hh.hh_volume_rebuild(vol, dev_parts, K_GD32, stream)
            if batch8 is not None:
                hh.hh_batch_launch_graph(batch8, stream)
            else:
                hh.hh_trace(vol, cams, params, bg_t, outs8, stream)
            for h, o in zip(host_rgb8, outs8):
                h.copy_(o["rgb8"], non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            if k >= args.warmup:
                e2e_ms.append(a.elapsed_time(b))
    if batch8 is not None:
        batch8.close()
    ms_e2e_serial = max_over_ranks(dist, sum(e2e_ms) / max(len(e2e_ms), 1), dev)

    # end to end through the C ABI with host buffers: the frame pipeline
    # (hh_pipeline_*), pinned host particles in and every view's display image
    # out each step, two frames in flight (uploads and downloads overlap the
    # kernels of the neighbouring frames); host wall clock over the K steps
    ms_e2e = None
    if not args.no_e2e:
        pipe = hh.hh_pipeline_create(grid, K_GD32, len(parts), cams, params, bg_t,
                                     tuned if batch is not None else None)
        host_img = [[torch.empty(c["width"] * c["height"] * 3, dtype=torch.uint8).pin_memory()
                     for c in cams] for _ in range(2)]

        def run_pipeline(n):
            ids = []
            for k in range(n):
                ids.append(hh.hh_pipeline_submit(pipe, host_parts, host_img[k % 2]))
                if k >= 1:
                    hh.hh_pipeline_wait(pipe, ids[-2])
            hh.hh_pipeline_wait(pipe, ids[-1])

        run_pipeline(args.warmup)
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        run_pipeline(args.steps)
        ms_pipe = (time.perf_counter() - t0) * 1e3 / args.steps
        pipe.close()
        ms_e2e = max_over_ranks(dist, ms_pipe, dev)

    # comparisons for the multi-view workloads: the same views as per-view
    # hh_trace launches on this volume, and the plain FP32 single-view march
    # (hh_trace on an FP32 volume of the same scene), march time only
    compare = {}
    if wl["mode"] == "batch" and not args.no_compare:
        def time_march(fn, reps=10):
            for _ in range(3):
                fn()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            with torch.cuda.stream(stream):
                for e0, e1 in evs:
                    flush.zero_()
                    e0.record(stream)
                    fn()
                    e1.record(stream)
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b) for a, b in evs) / reps

        with torch.cuda.stream(stream):
            ms_pv = time_march(lambda: hh.hh_trace(vol, cams, params, bg_t, outs, stream))
            v32 = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp32"), K_GD32,
                                          stream)
            ms_32 = time_march(lambda: hh.hh_trace(v32, cams, params, bg_t, outs, stream))
            v32.close()
        compare = {"batched_march_Mrays_s": round(n_rays / (ms_march * 1e-3) / 1e6, 3),
                   "per_view_launches_march_Mrays_s": round(n_rays / (ms_pv * 1e-3) / 1e6, 3),
                   "fp32_single_view_march_Mrays_s": round(n_rays / (ms_32 * 1e-3) / 1e6, 3)}
    if batch is not None:
        batch.close()
    vol.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    # algorithmic bytes of the march: 8 corners x 16 B (FP32) or 8 B (FP16)
    # per Eq. 16 step, plus per ray 12 B of RGB out and 4 x 3 B of texels
    per_step = 128 if wl["storage"] == "fp32" else 64
    march_bytes = total_steps * per_step + n_rays * 24
    achieved = march_bytes / (ms_march * 1e-3) / 1e9
    # the other roofline leg: FP32 work at the FMA peak (152 SMs x 128 lanes x
    # 2 flops per FMA at the sampled clock); FLOPS_PER_STEP is the per-op tally
    # of one Eq. 16 adaptive step of the kernel source (an FMA counts 2)
    fma_peak = 152 * 128 * 2 * (clocks.summary().get("sm_mhz") or 2070.0) * 1e6
    legs_ms = {"hbm_counted_bytes": round(march_bytes / (peak * 1e9) * 1e3, 4),
               "fp32_fma": round(total_steps * FLOPS_PER_STEP / fma_peak * 1e3, 4)}
    kname = ("march_kernel" if wl["mode"] == "trace" else "march_batch_kernel") + \
        f"<{wl['storage'].upper()}, EULER_PAPER, adaptive>"
    cpu = None
    if args.workload == "frame" and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, parts, cams[0], params, bg)
    clk = clocks.summary()
    line = {
        "metric": wl["metric"],
        "value": round(world * n_rays / (ms_step * 1e-3) / 1e6, 3),
        "unit": "Mrays/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if wl["storage"] == "fp32" else "f32 (fp16 storage)",
        "data": "synthetic (seeded plume particles, checker+noise equirect background)",
        "config": {"workload": wl["text"], "views": len(cams), "rays_per_step": n_rays,
                   "rays_hit": hits, "march_steps_per_frame": total_steps,
                   "steps_per_hit_ray": round(total_steps / max(hits, 1), 2),
                   "steps_per_hit_ray_quantiles": steps_dist,
                   "theta_paper": theta_paper,
                   "march_ms": round(ms_march, 4),
                   "build_ms": round(ms_step - ms_march, 4),
                   "march_Mrays_s": round(n_rays / (ms_march * 1e-3) / 1e6, 3),
                   "batch_config": tuned,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": None if args.no_e2e else {
            "value": round(world * n_rays / (ms_e2e * 1e-3) / 1e6, 3), "unit": "Mrays/s",
            "ms_per_step": round(ms_e2e, 4), "api": "hh_pipeline_submit / hh_pipeline_wait "
            "(host buffers, two frames in flight, host wall clock, L2 not flushed: every step "
            "rewrites the volume)",
            "serial": {"value": round(world * n_rays / (ms_e2e_serial * 1e-3) / 1e6, 3),
                       "ms_per_step": round(ms_e2e_serial, 4),
                       "api": "one frame at a time: pinned copy in, hh_volume_rebuild, "
                              "hh_trace or batch launch, copy out; CUDA events, L2 flushed"},
            "h2d_bytes_per_step": int(parts.nbytes),
            "d2h_bytes_per_step": int(n_rays * 3), "output": "rgb8 display images"},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic_for(args.workload), "kernel": kname,
                     "peak_kind": peak_kind, "algorithmic_bytes": int(march_bytes),
                     "leg_times_ms": legs_ms,
                     "counters": {k: v for k, v in march_counters(args.workload).items()
                                  if k in ("l1_hit_rate", "l2_hit_rate", "fma_pipe_pct",
                                           "active_lanes_per_instruction")} or None},
        "issue": issue_rate(args.workload, ms_march, clk),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if compare:
        line["compare"] = compare
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- #
# serving
# --------------------------------------------------------------------------- #
def run_serve(args):
    """Replays seeded Poisson request streams against the render server in
    real time and reports throughput and latency percentiles per rate."""
    import threading

    import torch

    from paper_2603_02048_gb300 import build as hb
    from paper_2603_02048_gb300 import hh

    hb.build()
    hh.load()
    dev = torch.device("cuda", 0)
    L, nf = SERVE["L"], SERVE["frames"]
    dims = (L, L, L)
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    bg_t = torch.from_numpy(hi.checker_background()).to(dev)
    base = hi.plume_particles(SERVE["particles"], L)
    grid = hh.make_grid(dims, 2.0, "fp16")
    rho = torch.empty(L ** 3, device=dev)
    vols = []
    t0 = time.perf_counter()
    for f in range(nf):
        parts_t = torch.from_numpy(hi.drifting_plume_frame(base, f, L=L)).to(dev)
        hh.hh_splat_density(parts_t, grid, rho)
        vols.append(hh.hh_volume_from_density(rho, grid, K_GD32))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del rho

    srv = hh.hh_serve_create(16 << 30, 8)
    # launch shape: autotuned once on a representative 8-view request of frame 0
    probe = f32([hi.orbit_camera(dims, 45.0 * i, 10.0, *hi.SERVE_RESOLUTIONS[i % 4])
                 for i in range(8)])
    probe_outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device=dev)} for c in probe]
    b = hh.hh_batch_create(vols[0], probe, params, bg_t, probe_outs)
    tuned = hh.hh_batch_autotune(b, reps=2)
    b.close()
    del probe_outs
    hh.hh_serve_set_config(srv, **tuned)
    for f, v in enumerate(vols):
        hh.hh_serve_put_volume(srv, f, v)

    def cams_of(req):
        return f32([hi.orbit_camera(dims, az, el, w, h) for az, el, w, h in req["views"]])

    # warm-up: a few requests through the whole path
    for req in hi.serving_requests(rate_hz=50, duration_s=0.2, n_frames=nf, seed=99)[:4]:
        t = hh.hh_serve_submit(srv, req["frame"], cams_of(req), params, bg_t, hh.HH_OUT_RGB8)
        hh.hh_serve_wait(srv, t, 60000)
        hh.hh_serve_release(srv, t)

    sweep = []
    for rate in SERVE["rates"]:
        reqs = hi.serving_requests(rate_hz=rate, duration_s=SERVE["duration_s"], n_frames=nf)
        prepared = [(r["t"], r["frame"], cams_of(r)) for r in reqs]
        tickets = []
        lock = threading.Lock()
        lat = []
        rays = [0]

        def collector():
            i = 0
            while True:
                with lock:
                    if i >= len(tickets):
                        if len(tickets) == len(prepared):
                            return
                        tk = None
                    else:
                        tk, nr = tickets[i]
                if tk is None:
                    time.sleep(0.0005)
                    continue
                lat.append(hh.hh_serve_wait(srv, tk, 120000))
                hh.hh_serve_release(srv, tk)
                rays[0] += nr
                i += 1

        th = threading.Thread(target=collector)
        th.start()
        start = time.perf_counter()
        for t_arr, frame, cams in prepared:
            delay = start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tk = hh.hh_serve_submit(srv, frame, cams, params, bg_t, hh.HH_OUT_RGB8)
            with lock:
                tickets.append((tk, sum(c["width"] * c["height"] for c in cams)))
        th.join()
        wall = time.perf_counter() - start
        lat_a = np.array(lat)
        offered = sum(sum(c["width"] * c["height"] for c in cams) for _, _, cams in prepared)
        sweep.append({"rate_req_s": rate, "requests": len(prepared),
                      "offered_Mrays_s": round(offered / SERVE["duration_s"] / 1e6, 1),
                      "Mrays_s": round(rays[0] / wall / 1e6, 1),
                      "p50_ms": round(float(np.percentile(lat_a, 50)), 2),
                      "p99_ms": round(float(np.percentile(lat_a, 99)), 2),
                      "max_ms": round(float(lat_a.max()), 2),
                      "wall_s": round(wall, 3)})
    stats = hh.hh_serve_get_stats(srv)
    srv.close()
    for v in vols:
        v.close()
    top = sweep[-1]
    print(json.dumps({
        "metric": SERVE["metric"], "value": top["Mrays_s"], "unit": "Mrays/s", "n_gpus": 1,
        "steps": len(SERVE["rates"]), "warmup": 4, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (fp16 storage)", "data": "synthetic (seeded drifting plume, Poisson)",
        "config": {"workload": SERVE["text"], "volume_build_s_60_frames": round(build_s, 2),
                   "batch_config": tuned},
        "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"], "sweep": sweep,
        "server_stats": {k: int(v) for k, v in stats.items()},
    }), flush=True)


# --------------------------------------------------------------------------- #
# the oracle (CPU baseline and reference arm)
# --------------------------------------------------------------------------- #
def oracle_frame_seconds(wl, parts, cam, params, bg, frac: int, nthreads: int, full_vol=None):
    """FP64 oracle time of one frame, measured on a 1/frac sample of each
    stage and scaled up: splat of every frac-th particle, Gladstone-Dale +
    gradient of a 1/frac slab of the grid, the march of every frac-th pixel
    (on the full oracle volume)."""
    import oracle

    L = wl["L"]
    dims = (L, L, L)
    t0 = time.perf_counter()
    rho = oracle.splat(parts[::frac], dims, 2.0)
    t1 = time.perf_counter()
    slab = max(2, L // frac)
    oracle.index_field(rho[:slab], K_GD32)
    t2 = time.perf_counter()
    if full_vol is None:
        full_vol = oracle.index_field(oracle.splat(parts, dims, 2.0), K_GD32)
    npx = cam["width"] * cam["height"]
    pix = np.arange(0, npx, frac, dtype=np.int64)
    t3 = time.perf_counter()
    oracle.trace_grid(full_vol, cam, params, bg, pixels=pix, nthreads=nthreads)
    t4 = time.perf_counter()
    per_frame = frac * (t1 - t0) + (L / slab) * (t2 - t1) + frac * (t4 - t3)
    return per_frame, full_vol, (t1 - t0) + (t2 - t1) + (t4 - t3)


def cpu_baseline(wl, parts, cam, params, bg):
    import oracle

    oracle.build()
    nthreads = os.cpu_count() or 1
    sec, _, worked = oracle_frame_seconds(wl, parts, cam, params, bg, 1, nthreads)
    npx = cam["width"] * cam["height"]
    return {"value": round(npx / sec / 1e6, 4), "unit": "Mrays/s",
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
    wl = WORKLOADS["frame"]
    dims, parts, cams, params, bg = scene(wl)
    cam = cams[0]
    nthreads = os.cpu_count() or 1
    frac = 16
    full_vol = None
    times = []
    for k in range(args.warmup + args.steps):
        sec, full_vol, _ = oracle_frame_seconds(wl, parts, cam, params, bg, frac, nthreads,
                                                full_vol)
        if k >= args.warmup:
            times.append(sec)
    ms = 1e3 * sum(times) / len(times)
    npx = cam["width"] * cam["height"]
    value = round(npx / (ms * 1e-3) / 1e6, 4)
    sample = (f"per step 1/{frac} of each stage (every {frac}th particle, 1/{frac} of the grid, "
              f"every {frac}th pixel), scaled to one frame")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["text"]},
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
    ap.add_argument("--workload", default="frame", choices=sorted(WORKLOADS) + ["serve"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison marches (per-view and FP32 for the multi-view "
                         "workloads, theta_max = 3e-3 for the frame)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
