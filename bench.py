"""Benchmark of the curved-ray heat-haze hot path on GB300.

One step = the whole hot path on one frame: splat 262,144 plume particles
onto a 256^3 grid (Sec. 3.3.1), Gladstone-Dale + gradient into the FP32
{dn, grad n} volume (Eqs. 12-13), and the adaptive curved-ray march of one
1920x1080 view (Eqs. 14-18) with the background lookup.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload all|frame|precision|batch|serve|theta]

The default (`all`) prints the frame line with the other configurations
nested in it (one GPU only): `precision` (8 views of 1280x720 on the 256^3
scene, FP16 storage), `batch` (32 uneven views on a 512^3 FP16 volume from
2,097,152 particles, one persistent graph-replayed launch) and `serve` (the
render server under seeded Poisson request streams at 25/50/100/200 req/s,
p50/p99 latency). `--workload X` prints X's own line; `theta` sweeps the
Eq. 18 tolerance theta_max over the 256^3 frame (steps per ray, march time,
error against the converged truth).

`value` is Mrays/s of whole steps (primary rays over the device time of K
frames of splat + field + march run back to back, inputs resident in HBM:
two volumes, each frame's build beside the previous frame's march, every
frame rewriting more than L2); `serial` beside it times one frame at a time
with L2 flushed before each; `e2e` is the same end to end through the C ABI
with host buffers (the
frame pipeline: particles from pinned host memory in, every view's RGB8 image
back, two frames in flight). `roofline` names the limit that binds the march
kernel: the largest of its DRAM traffic over HBM bandwidth, its FP32 work over
the FMA peak and its warp instructions over the issue peak. `error` states
the frame's exit-ray errors against the FP64 oracle on a seeded pixel sample,
computed in the CPU-baseline leg. `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload. N > 1 (torchrun) runs
independent replicas, one per GPU.
"""
from __future__ import annotations

import argparse
import json
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


# The workloads. "frame" is the headline; the others are the FP16 multi-view
# precision configuration and the 32-view batching one.
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

THETA_SWEEP = (3e-6, 1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3)

# FP32 operations of one Eq. 16 adaptive step as written in the march kernel
# (an FMA counts 2): lattice coordinates 6, trilinear weights 15, the 8-corner
# accumulation 60, n 1, w 3, g_perp and its norm 17, Eq. 18 step 4, ds/n 2,
# Eq. 16 update 6, renormalisation 20, position increment 6, compensated
# position 18. FP16 storage adds the two scale multiplications of the four
# channels (4).
FLOPS_PER_STEP = {"fp32": 158, "fp16": 162}


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
        self._summary = None

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
        if self._summary is None:
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
# roofline of the march kernel
# --------------------------------------------------------------------------- #
def march_counters(workload: str) -> dict:
    """Counters of one march launch from the committed ncu capture (DRAM bytes,
    warp instructions, hit rates), or {} when the march source has changed
    since they were taken."""
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


def roofline(workload: str, storage: str, ms_march: float, total_steps: int, n_rays: int,
             clocks: dict, sm_count: int, kernel: str) -> dict:
    """The limit that binds the march kernel, from three legs per launch:
    - hbm: DRAM bytes of one launch (committed ncu capture) over the measured
      HBM bandwidth;
    - fp32: its FP32 operations (FLOPS_PER_STEP x steps) over the FMA peak,
      SMs x 128 lanes x 2 x the median SM clock sampled during the run;
    - issue: its warp instructions (same capture) over the issue peak, SMs x 4
      schedulers x 1 warp-instruction per cycle at that clock.
    Each leg's frac is achieved / peak over the event-timed launch; `bound`
    is the leg with the largest frac (the slowest limit), and the line's
    achieved / peak / frac are that leg's. The fetch bytes the march counts
    (8 corners per step) are reported beside them: most are L1 hits, so they
    are not a DRAM figure."""
    peak_hbm, peak_kind = measured_peaks()
    ctr = march_counters(workload)
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    sec = ms_march * 1e-3
    legs = {}
    traffic = ctr.get("dram_bytes_per_launch")
    if traffic:
        a = traffic / sec / 1e9
        legs["hbm"] = {"achieved": round(a, 1), "peak": peak_hbm, "unit": "GB/s",
                       "frac": round(a / peak_hbm, 4), "peak_kind": peak_kind,
                       "bytes_per_launch": int(traffic)}
    flops = total_steps * FLOPS_PER_STEP[storage]
    p32 = sm_count * 128 * 2 * mhz * 1e6 / 1e12
    a = flops / sec / 1e12
    legs["fp32"] = {"achieved": round(a, 2), "peak": round(p32, 2), "unit": "TFLOP/s",
                    "frac": round(a / p32, 4), "flops_per_launch": int(flops),
                    "peak_kind": f"{sm_count} SMs x 128 FP32 lanes x 2 at {mhz:.0f} MHz"}
    inst = ctr.get("warp_instructions_per_launch")
    if inst:
        pi = sm_count * 4 * mhz * 1e6 / 1e9
        a = inst / sec / 1e9
        legs["issue"] = {"achieved": round(a, 1), "peak": round(pi, 1),
                         "unit": "G warp-instructions/s", "frac": round(a / pi, 4),
                         "warp_instructions_per_launch": int(inst),
                         "peak_kind": f"{sm_count} SMs x 4 schedulers x 1/cycle at {mhz:.0f} MHz"}
    bound = max(legs, key=lambda k: legs[k]["frac"])
    per_step = 128 if storage == "fp32" else 64
    fetch = total_steps * per_step + n_rays * 24
    out = {"bound": bound, "achieved": legs[bound]["achieved"], "peak": legs[bound]["peak"],
           "unit": legs[bound]["unit"], "frac": legs[bound]["frac"],
           "traffic": int(traffic) if traffic else None, "kernel": kernel,
           "legs": legs,
           "counted_fetch": {"bytes_per_launch": int(fetch),
                             "GB_s": round(fetch / sec / 1e9, 1),
                             "note": f"{per_step} B per step (8 corners) + 24 B per ray; mostly "
                                     "L1 hits, not DRAM traffic"},
           "counters": {k: v for k, v in ctr.items()
                        if k in ("l1_hit_rate", "l2_hit_rate", "fma_pipe_pct",
                                 "active_lanes_per_instruction")} or None}
    if not traffic:
        out["note"] = "no ncu capture for the current march source: hbm and issue legs absent"
    return out


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
class Ctx:
    """Per-process state shared by the workloads."""

    def __init__(self, args):
        import torch

        self.torch = torch
        self.args = args
        self.dist, self.rank, self.world, self.local = dist_setup(args.gpus)
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        from paper_2603_02048_gb300 import build as hb
        from paper_2603_02048_gb300 import hh

        if self.rank == 0:
            hb.build()
        barrier(self.dist)
        hb.build()  # no-op when fresh; makes sure every rank sees the library
        hh.load()
        self.hh = hh
        self.sm_count = torch.cuda.get_device_properties(self.dev).multi_processor_count
        self.flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)


def measure(ctx: Ctx, name: str, steps: int, warmup: int, with_e2e=True, with_compare=True,
            keep_outputs=False) -> dict:
    """Times `steps` whole steps (rebuild + march) of workload `name` and the
    end-to-end path; returns the figures (and, with keep_outputs, the frame's
    per-pixel GPU outputs and exported volume for the error statistics)."""
    torch, hh, dev, dist = ctx.torch, ctx.hh, ctx.dev, ctx.dist
    wl = WORKLOADS[name]
    dims, parts, cams, params, bg = scene(wl)
    parts_t = torch.from_numpy(parts).to(dev)
    bg_t = torch.from_numpy(bg).to(dev)
    grid = hh.make_grid(dims, 2.0, wl["storage"])
    n_rays = sum(c["width"] * c["height"] for c in cams)
    flush = ctx.flush
    torch.cuda.synchronize()  # inputs are on the device before any other stream uses them
    stream = torch.cuda.Stream(device=dev) if wl["mode"] == "batch" else \
        torch.cuda.current_stream(dev)
    vol = hh.hh_build_index_field(parts_t, grid, K_GD32, stream)
    res = {"wl": wl, "dims": dims, "cams": cams, "params": params, "bg": bg, "parts": parts,
           "n_rays": n_rays}

    # step statistics (deterministic input -> the same steps every frame); the
    # frame keeps its per-pixel outputs for the error statistics
    def trace_outputs(p):
        o = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device=dev),
              "steps": torch.empty(c["width"] * c["height"], dtype=torch.int32, device=dev),
              "flags": torch.empty(c["width"] * c["height"], dtype=torch.int32, device=dev)}
             for c in cams]
        if keep_outputs:
            for d, c in zip(o, cams):
                d["exit_pos"] = torch.empty(c["width"] * c["height"] * 3, device=dev)
                d["exit_dir"] = torch.empty(c["width"] * c["height"] * 3, device=dev)
        with torch.cuda.stream(stream):
            hh.hh_trace(vol, cams, p, bg_t, o, stream)
        torch.cuda.synchronize()
        return o

    stats = trace_outputs(params)
    res["total_steps"] = sum(int(o["steps"].sum().item()) for o in stats)
    res["hits"] = sum(int((o["flags"] & 1).sum().item()) for o in stats)
    res["steps_dist"] = steps_distribution(stats)
    if keep_outputs:
        res["gpu_out"] = {params["theta_max"]: [{k: v.cpu().numpy() for k, v in o.items()}
                                                for o in stats]}
    # the paper's theta_max = 3e-3 on the same volume and views (the schedule
    # at which Eq. 18 keeps every step at h_max on this scene), frame only
    res["theta_paper"] = None
    if name == "frame" and with_compare:
        p_paper = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_PAPER))
        sp = trace_outputs(p_paper)
        if keep_outputs:
            res["gpu_out"][p_paper["theta_max"]] = [{k: v.cpu().numpy() for k, v in o.items()}
                                                    for o in sp]
        with torch.cuda.stream(stream):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(10)]
            for e0, e1 in evs:
                flush.zero_()
                e0.record(stream)
                hh.hh_trace(vol, cams, p_paper, bg_t, sp, stream)
                e1.record(stream)
        torch.cuda.synchronize()
        ms_paper = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
        res["theta_paper"] = {"theta_max": hi.THETA_PAPER, "march_ms": round(ms_paper, 4),
                              "march_Mrays_s": round(n_rays / (ms_paper * 1e-3) / 1e6, 3),
                              "steps_per_hit_ray": steps_distribution(sp)}
        del sp
    if keep_outputs:
        v4 = torch.empty(dims[0] * dims[1] * dims[2] * 4, device=dev)
        hh.hh_volume_export(vol, v4, stream)
        torch.cuda.synchronize()
        res["vol4"] = v4.cpu().numpy().reshape(dims[2], dims[1], dims[0], 4)
        del v4
    outs = [{"rgb": o["rgb"]} for o in stats]
    del stats

    batch = None
    tuned = None
    if wl["mode"] == "batch":
        batch = hh.hh_batch_create(vol, cams, params, bg_t, outs)
        with torch.cuda.stream(stream):
            tuned = hh.hh_batch_autotune(batch, reps=3, stream=stream)
    res["tuned"] = tuned

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
        for _ in range(warmup):
            flush.zero_()
            step(parts_t)
    torch.cuda.synchronize()

    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
    ev_march = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(steps)]
    launches0 = hh.hh_kernel_launch_count()
    with ClockSampler(ctx.local) as clocks:
        barrier(dist)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()
                ev_step[k][0].record(stream)
                step(parts_t, ev_march[k])
                ev_step[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(dist)
    res["launches_serial"] = hh.hh_kernel_launch_count() - launches0
    res["clocks_serial"] = clocks.summary()
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    march_ms = [a.elapsed_time(b) for a, b in ev_march]
    res["ms_step_serial"] = max_over_ranks(dist, sum(step_ms) / len(step_ms), dev)
    res["ms_march"] = sum(march_ms) / len(march_ms)

    # the headline timing: frames back to back, as a renderer runs them. Two
    # volumes; frame k's build (splat + field) runs on a stream of the highest
    # priority beside frame k-1's march, each march waits for its frame's
    # build, and each build for the march that last read its volume. No L2
    # flush: every frame rewrites its volume and its density (together more
    # than L2) and reads particles last touched two frames earlier. CUDA
    # events on the march stream bracket the K frames.
    vol2 = hh.hh_build_index_field(parts_t, grid, K_GD32, stream)
    parts2 = parts_t.clone()
    batch2 = None
    if batch is not None:
        batch2 = hh.hh_batch_create(vol2, cams, params, bg_t, outs)
        hh.hh_batch_set_config(batch2, **tuned)
    torch.cuda.synchronize()
    try:
        hi_prio = torch.cuda.Stream.priority_range()[1]  # (least, greatest)
    except (AttributeError, RuntimeError):
        hi_prio = -1
    s_build = torch.cuda.Stream(device=dev, priority=hi_prio)
    s_march = torch.cuda.Stream(device=dev)
    vols, srcs, batches = (vol, vol2), (parts_t, parts2), (batch, batch2)

    def frames(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marched = [torch.cuda.Event() for _ in range(n)]
        t0.record(s_march)
        s_build.wait_event(t0)
        for k in range(n):
            i = k % 2
            if k >= 2:
                s_build.wait_event(marched[k - 2])
            hh.hh_volume_rebuild(vols[i], srcs[i], K_GD32, s_build)
            built = torch.cuda.Event()
            built.record(s_build)
            s_march.wait_event(built)
            if batches[i] is not None:
                hh.hh_batch_launch_graph(batches[i], s_march)
            else:
                hh.hh_trace(vols[i], cams, params, bg_t, outs, s_march)
            marched[k].record(s_march)
        t1.record(s_march)
        return t0, t1

    frames(max(warmup, 2))
    torch.cuda.synchronize()
    launches0 = hh.hh_kernel_launch_count()
    with ClockSampler(ctx.local) as clocks:
        barrier(dist)
        torch.cuda.synchronize()
        t0, t1 = frames(steps)
        torch.cuda.synchronize()
        barrier(dist)
    res["launches"] = hh.hh_kernel_launch_count() - launches0
    res["clocks"] = clocks.summary()
    res["ms_step"] = max_over_ranks(dist, t0.elapsed_time(t1) / steps, dev)
    if batch2 is not None:
        batch2.close()
    vol2.close()
    del parts2

    # end to end one frame at a time (reported as e2e.serial): pinned host
    # particles in, the display images (rgb8: what a viewer shows) out, every
    # step, each step synchronised and timed with CUDA events
    res["ms_e2e"] = res["ms_e2e_serial"] = None
    if with_e2e:
        host_parts = torch.from_numpy(parts).pin_memory()
        outs8 = [{"rgb8": torch.empty(o["rgb"].numel(), dtype=torch.uint8, device=dev)}
                 for o in outs]
        host_rgb8 = [torch.empty(o["rgb8"].numel(), dtype=torch.uint8).pin_memory()
                     for o in outs8]
        dev_parts = torch.empty_like(parts_t)
        batch8 = None
        if batch is not None:
            batch8 = hh.hh_batch_create(vol, cams, params, bg_t, outs8)
            hh.hh_batch_set_config(batch8, **tuned)
        e2e_ms = []
        with torch.cuda.stream(stream):
            for k in range(warmup + steps):
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
                if k >= warmup:
                    e2e_ms.append(a.elapsed_time(b))
        if batch8 is not None:
            batch8.close()
        res["ms_e2e_serial"] = max_over_ranks(dist, sum(e2e_ms) / max(len(e2e_ms), 1), dev)

        # end to end through the C ABI with host buffers: the frame pipeline
        # (hh_pipeline_*), pinned host particles in and every view's display
        # image out each step, two frames in flight (uploads and downloads
        # overlap the kernels of the neighbouring frames); host wall clock
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

        run_pipeline(warmup)
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        run_pipeline(steps)
        ms_pipe = (time.perf_counter() - t0) * 1e3 / steps
        pipe.close()
        res["ms_e2e"] = max_over_ranks(dist, ms_pipe, dev)
        res["h2d_bytes"] = int(parts.nbytes)
        res["d2h_bytes"] = int(n_rays * 3)

    # comparisons for the multi-view workloads: the same views as per-view
    # hh_trace launches on this volume, and the plain FP32 single-view march
    # (hh_trace on an FP32 volume of the same scene), march time only
    res["compare"] = {}
    if wl["mode"] == "batch" and with_compare:
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
        res["compare"] = {
            "batched_march_Mrays_s": round(n_rays / (res["ms_march"] * 1e-3) / 1e6, 3),
            "per_view_launches_march_Mrays_s": round(n_rays / (ms_pv * 1e-3) / 1e6, 3),
            "fp32_single_view_march_Mrays_s": round(n_rays / (ms_32 * 1e-3) / 1e6, 3)}
    if batch is not None:
        batch.close()
    vol.close()
    torch.cuda.synchronize()
    return res


def kernel_name(wl: dict) -> str:
    return ("march_kernel" if wl["mode"] == "trace" else "march_batch_kernel") + \
        f"<{wl['storage'].upper()}, EULER_PAPER, adaptive>"


def summary_of(ctx: Ctx, name: str, r: dict) -> dict:
    """The figures of one workload as a nested summary (or a line's body)."""
    wl, n_rays, world = r["wl"], r["n_rays"], ctx.world
    out = {"metric": wl["metric"],
           "value": round(world * n_rays / (r["ms_step"] * 1e-3) / 1e6, 3), "unit": "Mrays/s",
           "ms_per_step": round(r["ms_step"], 4),
           "serial": {"value": round(world * n_rays / (r["ms_step_serial"] * 1e-3) / 1e6, 3),
                      "ms_per_step": round(r["ms_step_serial"], 4),
                      "timing": "one frame at a time on one stream: L2 flushed (256 MB "
                                "write), then build and march, CUDA events around both",
                      "gpu_launches": int(r["launches_serial"]),
                      "clocks": r["clocks_serial"]},
           "march_ms": round(r["ms_march"], 4),
           "build_ms": round(r["ms_step_serial"] - r["ms_march"], 4),
           "march_Mrays_s": round(n_rays / (r["ms_march"] * 1e-3) / 1e6, 3),
           "config": {"workload": wl["text"], "views": len(r["cams"]), "rays_per_step": n_rays,
                      "rays_hit": r["hits"], "march_steps_per_frame": r["total_steps"],
                      "steps_per_hit_ray": round(r["total_steps"] / max(r["hits"], 1), 2),
                      "steps_per_hit_ray_quantiles": r["steps_dist"],
                      "batch_config": r["tuned"],
                      "timing": "frames back to back: two volumes, frame k's build on a "
                                "highest-priority stream beside frame k-1's march; CUDA "
                                "events on the march stream around the K frames",
                      "l2": "not flushed: inputs larger than L2 (every frame rewrites its "
                            "volume and density, more than L2; the serial figures flush "
                            "with a 256 MB write)"},
           "clocks": r["clocks"], "gpu_launches": int(r["launches"]),
           "roofline": roofline(name, wl["storage"], r["ms_march"], r["total_steps"], n_rays,
                                r["clocks"], ctx.sm_count, kernel_name(wl))}
    if r["ms_e2e"] is not None:
        out["e2e"] = {
            "value": round(world * n_rays / (r["ms_e2e"] * 1e-3) / 1e6, 3), "unit": "Mrays/s",
            "ms_per_step": round(r["ms_e2e"], 4),
            "api": "hh_pipeline_submit / hh_pipeline_wait (host buffers, two frames in flight, "
                   "host wall clock, L2 not flushed: every step rewrites the volume)",
            "serial": {"value": round(world * n_rays / (r["ms_e2e_serial"] * 1e-3) / 1e6, 3),
                       "ms_per_step": round(r["ms_e2e_serial"], 4),
                       "api": "one frame at a time: pinned copy in, hh_volume_rebuild, "
                              "hh_trace or batch launch, copy out; CUDA events, L2 flushed"},
            "h2d_bytes_per_step": r["h2d_bytes"], "d2h_bytes_per_step": r["d2h_bytes"],
            "output": "rgb8 display images"}
    if r["compare"]:
        out["compare"] = r["compare"]
    if r["theta_paper"]:
        out["config"]["theta_paper"] = r["theta_paper"]
    return out


def run_ours(args):
    ctx = Ctx(args)
    name = "frame" if args.workload == "all" else args.workload
    if name == "serve":
        line = serve_line(ctx, serve_sweep(ctx, SERVE["duration_s"]))
    elif name == "theta":
        line = theta_line(ctx, args)
    else:
        cpu_leg = name == "frame" and not args.no_cpu_baseline and ctx.rank == 0 \
            and ctx.world == 1
        r = measure(ctx, name, args.steps, args.warmup, with_e2e=not args.no_e2e,
                    with_compare=not args.no_compare, keep_outputs=cpu_leg)
        body = summary_of(ctx, name, r)
        line = {"metric": body.pop("metric"), "value": body.pop("value"), "unit": "Mrays/s",
                "n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": body.pop("ms_per_step"), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if r["wl"]["storage"] == "fp32" else "f32 (fp16 storage)",
                "data": "synthetic (seeded plume particles, checker+noise equirect background)"}
        line.update(body)
        line["config"]["parallelism"] = "replicas" if ctx.world > 1 else "single GPU"
        line.setdefault("e2e", None)
        line["cpu_baseline"] = None
        if cpu_leg:
            line["cpu_baseline"], line["error"] = cpu_baseline_leg(r)
        if args.workload == "all" and ctx.world == 1:
            # the other configurations, each a nested summary on the same clock
            nested_steps = {"precision": args.steps, "batch": min(args.steps, 10)}
            for other in ("precision", "batch"):
                rr = measure(ctx, other, nested_steps[other], args.warmup,
                             with_e2e=not args.no_e2e, with_compare=not args.no_compare)
                line[other] = summary_of(ctx, other, rr)
                line[other]["steps"] = nested_steps[other]
                del rr
            line["serve"] = serve_line(ctx, serve_sweep(ctx, SERVE["duration_s"]), nested=True)
        elif args.workload == "all":
            line["nested"] = "precision / batch / serve summaries are measured at N = 1 only"
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    if ctx.dist is not None:
        ctx.dist.destroy_process_group()


# --------------------------------------------------------------------------- #
# serving
# --------------------------------------------------------------------------- #
def serve_sweep(ctx: Ctx, duration_s: float) -> dict:
    """Replays seeded Poisson request streams against the render server in
    real time and reports throughput and latency percentiles per rate."""
    import threading

    torch, hh, dev = ctx.torch, ctx.hh, ctx.dev
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
    with ClockSampler(ctx.local) as clocks:
        for rate in SERVE["rates"]:
            reqs = hi.serving_requests(rate_hz=rate, duration_s=duration_s, n_frames=nf)
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
            offered = sum(sum(c["width"] * c["height"] for c in cams)
                          for _, _, cams in prepared)
            sweep.append({"rate_req_s": rate, "requests": len(prepared),
                          "offered_Mrays_s": round(offered / duration_s / 1e6, 1),
                          "Mrays_s": round(rays[0] / wall / 1e6, 1),
                          "p50_ms": round(float(np.percentile(lat_a, 50)), 2),
                          "p99_ms": round(float(np.percentile(lat_a, 99)), 2),
                          "max_ms": round(float(lat_a.max()), 2),
                          "wall_s": round(wall, 3)})
    stats = hh.hh_serve_get_stats(srv)
    srv.close()
    for v in vols:
        v.close()
    torch.cuda.synchronize()
    return {"sweep": sweep, "build_s": build_s, "tuned": tuned, "clocks": clocks.summary(),
            "stats": {k: int(v) for k, v in stats.items()}}


def serve_line(ctx: Ctx, s: dict, nested: bool = False) -> dict:
    top = max(s["sweep"], key=lambda e: e["Mrays_s"])
    body = {"metric": SERVE["metric"], "value": top["Mrays_s"], "unit": "Mrays/s",
            "saturation_rate_req_s": top["rate_req_s"],
            "p50_p99_ms": {str(e["rate_req_s"]): [e["p50_ms"], e["p99_ms"]] for e in s["sweep"]},
            "sweep": s["sweep"], "clocks": s["clocks"],
            "config": {"workload": SERVE["text"], "volume_build_s_60_frames": round(s["build_s"], 2),
                       "batch_config": s["tuned"]},
            "server_stats": s["stats"]}
    if nested:
        return body
    line = {"metric": body.pop("metric"), "value": body.pop("value"), "unit": "Mrays/s",
            "n_gpus": 1, "steps": len(SERVE["rates"]), "warmup": 4, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (fp16 storage)", "data": "synthetic (seeded drifting plume, Poisson)"}
    line.update(body)
    return line


# --------------------------------------------------------------------------- #
# theta_max sweep (Sec. 4.1's tolerance sweep on the 256^3 frame)
# --------------------------------------------------------------------------- #
def theta_line(ctx: Ctx, args) -> dict:
    """For each theta_max: steps per hit ray, march time (CUDA events, L2
    flushed, median of the steps) and, in the CPU-baseline leg, the exit
    direction error of the GPU march against the converged FP64 truth (RK4
    of Eq. 15 at 1/64 voxel on the same volume) on a seeded pixel sample."""
    torch, hh, dev = ctx.torch, ctx.hh, ctx.dev
    wl = WORKLOADS["frame"]
    dims, parts, cams, _, bg = scene(wl)
    cam = cams[0]
    parts_t = torch.from_numpy(parts).to(dev)
    bg_t = torch.from_numpy(bg).to(dev)
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp32"), K_GD32)
    n = cam["width"] * cam["height"]
    out = {"rgb": torch.empty(n * 3, device=dev), "exit_dir": torch.empty(n * 3, device=dev),
           "exit_pos": torch.empty(n * 3, device=dev),
           "steps": torch.empty(n, dtype=torch.int32, device=dev),
           "flags": torch.empty(n, dtype=torch.int32, device=dev)}
    rows = []
    gpu_dirs = {}
    with ClockSampler(ctx.local) as clocks:
        for theta in THETA_SWEEP:
            p = f32(hi.params_euler_adaptive(dims, theta_max=theta))
            hh.hh_trace(vol, [cam], p, bg_t, [out])
            torch.cuda.synchronize()
            sd = steps_distribution([out])
            gpu_dirs[theta] = (out["exit_dir"].cpu().numpy().reshape(-1, 3).astype(np.float64),
                               out["flags"].cpu().numpy())
            ms = []
            for _ in range(args.warmup + args.steps):
                ctx.flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                hh.hh_trace(vol, [cam], p, bg_t, [out])
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            ms = sorted(ms[args.warmup:])[len(ms[args.warmup:]) // 2]
            rows.append({"theta_max": theta, "march_ms": round(ms, 4),
                         "march_Mrays_s": round(n / (ms * 1e-3) / 1e6, 1),
                         "steps_per_hit_ray": sd})
    v4 = torch.empty(dims[0] * dims[1] * dims[2] * 4, device=dev)
    hh.hh_volume_export(vol, v4)
    torch.cuda.synchronize()
    vol.close()
    line = {"metric": "curved-ray march Mrays/s and error vs theta_max (1080p, 256^3 FP32)",
            "value": rows[[r["theta_max"] for r in rows].index(hi.THETA_CALIBRATED)][
                "march_Mrays_s"],
            "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["text"].replace("theta_max=3e-5", "theta_max swept"),
                       "l2": "flushed between timed marches"},
            "sweep": rows, "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        vol4 = v4.cpu().numpy().astype(np.float64).reshape(dims[2], dims[1], dims[0], 4)
        truth_err(line, vol4, cam, dims, bg, gpu_dirs)
    return line


# --------------------------------------------------------------------------- #
# the oracle (CPU baseline leg: timing, and the error statistics) and the
# reference arm
# --------------------------------------------------------------------------- #
def _sample(flags, n, seed):
    """n seeded pixels, at least half of them rays that hit (when there are)."""
    r = np.random.default_rng(seed)
    hit = np.flatnonzero(flags & 1)
    miss = np.flatnonzero((flags & 1) == 0)
    a = r.choice(hit, min(len(hit), n // 2), replace=False)
    b = r.choice(miss, min(len(miss), n - len(a)), replace=False)
    return np.sort(np.concatenate([a, b]))


def frame_error(r: dict, nthreads: int) -> dict:
    """Error of the timed frame against the FP64 oracle on the GPU's own
    volume, on a seeded 4000-pixel sample (half of them rays that hit), at the
    timed theta_max and at the paper's: exit-direction median / p99 / max over
    the hit rays, largest exit-position difference, image RMSE, rays beyond
    the tolerances, and how many of them the parity rule excuses as ill
    conditioned (all of them must be)."""
    import oracle

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import parity_util as pu

    cam, dims, bg = r["cams"][0], r["dims"], r["bg"]
    vol4 = r["vol4"].astype(np.float64)
    field = {"kind": "grid", "vol4": vol4}
    out = {"sample": "4000 seeded pixels (2000 hit rays), oracle on the GPU's own volume",
           "tolerance": {"exit_pos_voxel": pu.POS_TOL, "exit_dir_rad": pu.DIR_TOL,
                         "rmse": pu.RMSE_TOL}}
    for theta, g in r["gpu_out"].items():
        g = g[0]
        gpu = {"rgb": g["rgb"].reshape(-1, 3).astype(np.float64),
               "exit_pos": g["exit_pos"].reshape(-1, 3).astype(np.float64),
               "exit_dir": g["exit_dir"].reshape(-1, 3).astype(np.float64),
               "steps": g["steps"], "flags": g["flags"].view(np.uint32)}
        pix = _sample(gpu["flags"], 4000, seed=7)
        params = f32(hi.params_euler_adaptive(dims, theta_max=theta))
        ref = oracle.trace_grid(vol4, cam, params, bg, pixels=pix, nthreads=nthreads)
        hit = (ref["flags"] & 1) != 0
        ang = pu.angle(gpu["exit_dir"][pix][hit], ref["exit_dir"][hit])
        q = np.percentile(ang, [50, 99, 100]) if len(ang) else [0.0, 0.0, 0.0]
        rec = {"hit_rays": int(hit.sum()), "exit_dir_median_rad": float(f"{q[0]:.3g}"),
               "exit_dir_p99_rad": float(f"{q[1]:.3g}"), "exit_dir_max_rad": float(f"{q[2]:.3g}")}
        try:
            st = pu.assert_parity_conditioned(gpu, ref, oracle, field, dims, cam, params,
                                              sel=pix, label=f"bench frame theta {theta}")
            rec["parity"] = "pass"
        except AssertionError as e:  # reported, not hidden
            st = pu.compare(gpu, ref, pix, box=dims)
            rec["parity"] = f"FAIL: {str(e)[:300]}"
        rec.update({"exit_pos_max_voxel": float(f"{st['pos_max']:.3g}"),
                    "rmse": float(f"{st['rmse']:.3g}"), "n_beyond_tol": st.get("n_bad"),
                    "n_excused_ill_conditioned": st.get("n_ill"),
                    "step_mismatch": st["step_mismatch"]})
        out[f"theta_{theta:g}"] = rec
    return out


def truth_err(line: dict, vol4, cam, dims, bg, gpu_dirs, n: int = 1000):
    """Adds to each theta row the exit-direction error of the GPU march against
    the converged FP64 truth (RK4 of Eq. 15 at 1/64 voxel) and of the oracle's
    own march at that theta, on a seeded sample of n hit pixels."""
    import oracle

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import parity_util as pu

    nthreads = os.cpu_count() or 1
    flags = next(iter(gpu_dirs.values()))[1]
    r = np.random.default_rng(11)
    pix = np.sort(r.choice(np.flatnonzero(flags & 1), n, replace=False))
    t0 = time.perf_counter()
    truth = oracle.trace_grid(vol4, cam, f32(hi.params_rk4_fixed(dims, 1.0 / 64.0)), bg,
                              pixels=pix, nthreads=nthreads)
    t_truth = time.perf_counter() - t0
    for row in line["sweep"]:
        theta = row["theta_max"]
        d, _ = gpu_dirs[theta]
        own = oracle.trace_grid(vol4, cam, f32(hi.params_euler_adaptive(dims, theta_max=theta)),
                                bg, pixels=pix, nthreads=nthreads)
        for key, dirs in (("gpu_vs_truth", d[pix]), ("oracle_vs_truth", own["exit_dir"])):
            a = pu.angle(dirs, truth["exit_dir"])
            q = np.percentile(a, [50, 99, 100])
            row[key] = {"median_rad": float(f"{q[0]:.3g}"), "p99_rad": float(f"{q[1]:.3g}"),
                        "max_rad": float(f"{q[2]:.3g}")}
    line["truth"] = {"schedule": "RK4 of Eq. 15, fixed h = 1/64 voxel, FP64, on the GPU's FP32 "
                                 "volume", "pixels": f"{n} seeded hit pixels",
                     "seconds": round(t_truth, 1), "cores": nthreads}


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


def cpu_baseline_leg(r: dict):
    """The oracle on the host cores: the whole frame timed (all particles
    splatted, the whole grid through Gladstone-Dale, every pixel marched), and
    the error statistics of the timed frame against it."""
    import oracle

    oracle.build()
    nthreads = os.cpu_count() or 1
    wl, parts, cam, params, bg = r["wl"], r["parts"], r["cams"][0], r["params"], r["bg"]
    sec, _, worked = oracle_frame_seconds(wl, parts, cam, params, bg, 1, nthreads)
    npx = cam["width"] * cam["height"]
    cpu = {"value": round(npx / sec / 1e6, 4), "unit": "Mrays/s",
           "cores": nthreads, "kind": "oracle",
           "sample": (f"one whole frame: all particles splatted (1 thread), the whole grid "
                      f"through Gladstone-Dale (1 thread), every pixel marched ({nthreads} "
                      f"threads); {worked:.1f} s measured"),
           "ms_per_frame": round(sec * 1e3, 1)}
    return cpu, frame_error(r, nthreads)


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
    ap.add_argument("--workload", default="all",
                    choices=["all"] + sorted(WORKLOADS) + ["serve", "theta"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison marches (per-view and FP32 for the multi-view "
                         "workloads, theta_max = 3e-3 for the frame)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
