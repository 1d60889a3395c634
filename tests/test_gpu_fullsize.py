"""Parity at full size, in the launch configuration the benchmark times.

The 262,144-particle plume splatted onto 256^3 and traced at 1920x1080 with
the adaptive Eq. 16 march is checked against the FP64 oracle on the whole
density grid and on a seeded sample of pixels (the oracle computes them one
by one on the GPU's own volume). The 8-view FP16 configuration (1280x720 on a
90 degree arc) is checked the same way, and its precision against the FP64
oracle on the FP32 volume is stated as PSNR.
"""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import (angle, assert_parity_conditioned, assert_parity_plain, export_volume,
                         f32, gpu_trace, ill_conditioned)

pytestmark = pytest.mark.gpu

L = 256
DIMS = (L, L, L)
N_PARTICLES = 262144


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_02048_gb300 import hh

    return hh, torch


@pytest.fixture(scope="module")
def scene(gpu):
    hh, torch = gpu
    parts = hi.plume_particles(N_PARTICLES, L)
    bg = hi.checker_background()
    return parts, torch.from_numpy(parts).cuda(), bg, torch.from_numpy(bg).cuda()


def _sample_pixels(cam, n, seed, flags=None):
    """n seeded pixels; with flags, at least half of them rays that hit."""
    r = np.random.default_rng(seed)
    npx = cam["width"] * cam["height"]
    if flags is None:
        return np.sort(r.choice(npx, n, replace=False))
    hit = np.flatnonzero(flags & 1)
    miss = np.flatnonzero((flags & 1) == 0)
    a = r.choice(hit, min(len(hit), n // 2), replace=False)
    b = r.choice(miss, min(len(miss), n - len(a)), replace=False)
    return np.sort(np.concatenate([a, b]))


def test_fullsize_density_grid(gpu, oracle_lib, scene):
    hh, torch = gpu
    parts, parts_t, _, _ = scene
    rho = torch.empty(L**3, device="cuda")
    hh.hh_splat_density(parts_t, hh.make_grid(DIMS, 2.0), rho)
    torch.cuda.synchronize()
    got = rho.cpu().numpy().astype(np.float64).reshape(L, L, L)
    want = oracle_lib.splat(parts, DIMS, 2.0)
    assert np.abs(got - want).max() <= 1e-5 * want.max()
    assert 1.5 < want.max() < 4.0  # plume-centre density ~ rho0 = 1.2 plus particle noise


@pytest.mark.parametrize("theta", [hi.THETA_CALIBRATED, hi.THETA_PAPER])
def test_fullsize_1080p_adaptive(gpu, oracle_lib, scene, theta):
    hh, torch = gpu
    parts, parts_t, bg, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0), f32(hi.K_GD))
    cam = f32(hi.orbit_camera(DIMS, 0.0, 0.0, 1920, 1080))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=theta))
    got = gpu_trace(hh, torch, vol, [cam], params, bg_t)[0]
    vol4 = export_volume(hh, torch, vol, DIMS)
    pix = _sample_pixels(cam, 4000, seed=5, flags=got["flags"])
    ref = oracle_lib.trace_grid(vol4, cam, params, bg, pixels=pix, nthreads=8)
    # the cap follows this sample's own rate: 10-12 of its 2000 hit rays are ill
    # conditioned at theta 3e-5 (0.50-0.60 %, over five GPU runs), above the
    # whole frame's 0.31 %, which the whole-frame test holds to 0.5 %
    st = assert_parity_conditioned(got, ref, oracle_lib, {"kind": "grid", "vol4": vol4}, DIMS,
                                   cam, params, sel=pix, max_ill_frac=0.008)
    assert st["hits"] >= 1900


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fullsize_1080p_whole_frame(gpu, oracle_lib, scene, storage):
    """Every one of the 2,073,600 pixels of the 1080p frame against the
    oracle (theta_max = 3e-5), with the conditioning rule over the whole
    frame; prints the distribution of the exit-direction error, the rays
    beyond tolerance and those leaving through another face."""
    hh, torch = gpu
    parts, parts_t, bg, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0, storage), f32(hi.K_GD))
    cam = f32(hi.orbit_camera(DIMS, 0.0, 0.0, 1920, 1080))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=hi.THETA_CALIBRATED))
    got = gpu_trace(hh, torch, vol, [cam], params, bg_t)[0]
    vol4 = export_volume(hh, torch, vol, DIMS)
    vol.close()
    ref = oracle_lib.trace_grid(vol4, cam, params, bg, nthreads=16)
    st = assert_parity_conditioned(got, ref, oracle_lib, {"kind": "grid", "vol4": vol4}, DIMS,
                                   cam, params)
    hit = (ref["flags"] & 1) != 0
    ang = angle(got["exit_dir"][hit], ref["exit_dir"][hit])
    q = np.percentile(ang, [50, 99, 99.9, 100])
    print(f"1080p {storage}: {int(hit.sum())} hit rays; exit direction error median {q[0]:.2e}, "
          f"p99 {q[1]:.2e}, p99.9 {q[2]:.2e}, max {q[3]:.2e} rad; {st['n_bad']} rays beyond "
          f"tolerance ({st['n_ill']} ill conditioned); {st['step_mismatch']} with another step "
          f"count; {st['face_mismatch']} through another face (exit points at most "
          f"{st['face_mismatch_pos_max']:.1e} apart); RMSE {st['rmse']:.2e}")
    assert st["hits"] == 876096
    assert st["rmse"] <= 1e-4  # the whole image, excused rays included
    assert q[0] <= 1e-7  # the typical ray is well inside the tolerance


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fullsize_1080p_whole_frame_paper_theta_plain(gpu, oracle_lib, scene, storage):
    """The whole 1080p frame at the paper's theta_max = 3e-3, where Eq. 18
    keeps every step at h_max on this plume: no ray is ill conditioned, so
    every one of the 876,096 hit rays is held to the plain tolerances (exit
    position 1e-3 voxel, exit direction 1e-6 rad) with no excusal."""
    hh, torch = gpu
    parts, parts_t, bg, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0, storage), f32(hi.K_GD))
    cam = f32(hi.orbit_camera(DIMS, 0.0, 0.0, 1920, 1080))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=hi.THETA_PAPER))
    got = gpu_trace(hh, torch, vol, [cam], params, bg_t)[0]
    vol4 = export_volume(hh, torch, vol, DIMS)
    vol.close()
    ref = oracle_lib.trace_grid(vol4, cam, params, bg, nthreads=16)
    st = assert_parity_plain(got, ref, DIMS)
    hit = (ref["flags"] & 1) != 0
    ang = angle(got["exit_dir"][hit], ref["exit_dir"][hit])
    print(f"1080p {storage} theta 3e-3: {st['hits']} hit rays, all within tolerance; exit "
          f"direction error max {ang.max():.2e} rad, position max {st['pos_max']:.2e} voxel; "
          f"{st['step_mismatch']} with another step count; RMSE {st['rmse']:.2e}")
    assert st["hits"] == 876096


def test_fullsize_8view_fp16(gpu, oracle_lib, scene):
    hh, torch = gpu
    parts, parts_t, bg, bg_t = scene
    v16 = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0, "fp16"), f32(hi.K_GD))
    v32 = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0, "fp32"), f32(hi.K_GD))
    cams = f32(hi.arc_cameras(DIMS, n=8, width=1280, height=720))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=hi.THETA_CALIBRATED))
    got = gpu_trace(hh, torch, v16, cams, params, bg_t)
    vol16 = export_volume(hh, torch, v16, DIMS)
    vol32 = export_volume(hh, torch, v32, DIMS)
    for i, (c, g) in enumerate(zip(cams, got)):
        pix = _sample_pixels(c, 4000, seed=100 + i, flags=g["flags"])
        ref = oracle_lib.trace_grid(vol16, c, params, bg, pixels=pix, nthreads=8)
        # the share of ill-conditioned rays depends on how much of the noisy
        # plume core a view's rays cross: 0.15 % to 0.9 % of the sampled hit
        # rays on these views (0.3 % on the whole azimuth-0 frame)
        assert_parity_conditioned(g, ref, oracle_lib, {"kind": "grid", "vol4": vol16}, DIMS, c,
                                  params, sel=pix, max_ill_frac=0.015)
        truth = oracle_lib.trace_grid(vol32, c, params, bg, pixels=pix, nthreads=8)
        mse = np.mean((g["rgb"][pix] - truth["rgb"]) ** 2)
        assert 10 * np.log10(1.0 / max(mse, 1e-30)) >= 50.0


def test_fullsize_8view_fp16_batched_launch_equals_trace(gpu, scene):
    """The precision configuration as the benchmark times it: one persistent
    batched launch (replayed from a CUDA graph) over the 8 views, bit for bit
    the per-view hh_trace result checked above."""
    hh, torch = gpu
    parts, parts_t, bg, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(DIMS, 2.0, "fp16"), f32(hi.K_GD))
    cams = f32(hi.arc_cameras(DIMS, n=8, width=1280, height=720))
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=hi.THETA_CALIBRATED))
    ref = gpu_trace(hh, torch, vol, cams, params, bg_t, want_all=False)
    outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device="cuda")} for c in cams]
    b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
    hh.hh_batch_set_config(b, 256, 0, 32, 4, 1, 0)  # the configuration the autotuner keeps here
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            hh.hh_batch_launch_graph(b, s)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert np.array_equal(o["rgb"].cpu().numpy().reshape(-1, 3), r["rgb"].astype(np.float32))
    b.close()
    vol.close()


def test_fullsize_512_fp16_32_views_batched(gpu, oracle_lib):
    """The batching configuration at full size: 2,097,152 particles -> 512^3
    FP16, 32 views of uneven size in one persistent launch, checked against
    the FP64 oracle on a seeded sample of pixels of every view."""
    hh, torch = gpu
    L5 = 512
    dims = (L5, L5, L5)
    parts_t = torch.from_numpy(hi.plume_particles(2097152, L5)).cuda()
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp16"), f32(hi.K_GD))
    del parts_t
    cams = f32(hi.view_mix(dims, n=32))
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    bg = hi.checker_background()
    bg_t = torch.from_numpy(bg).cuda()
    outs = []
    for c in cams:
        n = c["width"] * c["height"]
        outs.append({"rgb": torch.empty(n * 3, device="cuda"),
                     "exit_pos": torch.empty(n * 3, device="cuda"),
                     "exit_dir": torch.empty(n * 3, device="cuda"),
                     "steps": torch.empty(n, dtype=torch.int32, device="cuda"),
                     "flags": torch.empty(n, dtype=torch.int32, device="cuda")})
    b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
    hh.hh_batch_set_config(b, 128, 0, 32, 4, 1, 1)  # the configuration the autotuner keeps here
    hh.hh_batch_launch(b)
    torch.cuda.synchronize()
    got = [{k: (v.cpu().numpy().reshape(-1, 3).astype(np.float64) if k in ("rgb", "exit_pos",
                                                                          "exit_dir")
                else v.cpu().numpy().view(np.uint32) if k == "flags" else v.cpu().numpy())
            for k, v in o.items()} for o in outs]
    b.close()
    vol4 = export_volume(hh, torch, vol, dims)
    vol.close()
    field = {"kind": "grid", "vol4": vol4}
    hits = ill = pop_ill = 0
    for i, (c, g) in enumerate(zip(cams, got)):
        pix = _sample_pixels(c, 4000, seed=300 + i, flags=g["flags"])
        ref = oracle_lib.trace_grid(vol4, c, params, bg, pixels=pix, nthreads=16)
        # rays about twice as long as at 256^3 (~165 steps): the share of
        # ill-conditioned rays grows with the path (measured 2.6 % of the hit
        # rays beyond tolerance, every one ill conditioned)
        st = assert_parity_conditioned(g, ref, oracle_lib, field, dims, c, params, sel=pix,
                                       max_ill_frac=0.04)
        hits += st["hits"]
        ill += st["n_ill"]
        hit_pix = pix[(ref["flags"] & 1) != 0]
        if len(hit_pix):
            pop_ill += int(ill_conditioned(oracle_lib, field, dims, c, params, hit_pix)[0].sum())
    print(f"512^3 FP16, 32 views: {hits} sampled hit rays; the oracle alone finds {pop_ill} "
          f"ill conditioned; {ill} GPU rays beyond tolerance, all of them ill conditioned")
    assert hits >= 32 * 1500
    # no more rays are excused than the oracle itself finds ill conditioned
    # in the sample
    assert ill <= pop_ill + 2


def test_fullsize_serve_384_fp16(gpu, oracle_lib):
    """The serving configuration at full size: 384^3 FP16 volumes of the
    1,048,576-particle drifting plume, the first requests of the seeded
    Poisson stream (1-16 views up to 3840x2160) in flight together. Every
    served display image is hh_trace's on the same volume, bit for bit; the
    first request is checked against the FP64 oracle on sampled pixels."""
    hh, torch = gpu
    L3 = 384
    dims = (L3, L3, L3)
    base = hi.plume_particles(1048576, L3)
    vols = []
    for t in range(3):
        parts_t = torch.from_numpy(hi.drifting_plume_frame(base, t, L=L3)).cuda()
        vols.append(hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp16"),
                                            f32(hi.K_GD)))
    del parts_t
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    bg = hi.checker_background()
    bg_t = torch.from_numpy(bg).cuda()
    srv = hh.hh_serve_create(8 << 30, 8)
    for t, v in enumerate(vols):
        hh.hh_serve_put_volume(srv, t, v)
    reqs = hi.serving_requests()[:6]
    tickets = []
    for i, r in enumerate(reqs):
        cams = f32([hi.orbit_camera(dims, az, el, w, h) for az, el, w, h in r["views"]])
        outputs = (hh.HH_OUT_RGB | hh.HH_OUT_EXIT | hh.HH_OUT_STEPS | hh.HH_OUT_RGB8) if i == 0 \
            else hh.HH_OUT_RGB8
        # the stream's first requests all fall in sim frame 0: spread them
        # over the three volumes
        tickets.append((hh.hh_serve_submit(srv, i % 3, cams, params, bg_t, outputs), i % 3,
                        cams))
    n_views = 0
    first = None
    for ti, (tk, f, cams) in enumerate(tickets):
        hh.hh_serve_wait(srv, tk, 120000)
        ref = [{"rgb8": torch.empty(c["width"] * c["height"] * 3, dtype=torch.uint8,
                                    device="cuda")} for c in cams]
        hh.hh_trace(vols[f], cams, params, bg_t, ref)
        torch.cuda.synchronize()
        for i, c in enumerate(cams):
            v = hh.hh_serve_view(srv, tk, i, c["width"], c["height"])
            assert torch.equal(v["rgb8"], ref[i]["rgb8"]), (ti, i)
            if ti == 0 and i == 0:
                first = {k: (t.cpu().numpy().reshape(-1, 3).astype(np.float64)
                             if k in ("rgb", "exit_pos", "exit_dir")
                             else t.cpu().numpy().view(np.uint32) if k == "flags"
                             else t.cpu().numpy()) for k, t in v.items() if k != "rgb8"}
            n_views += 1
        hh.hh_serve_release(srv, tk)
    assert n_views >= 12
    srv.close()
    # the first request's first view against the oracle
    _, f, cams = tickets[0]
    vol4 = export_volume(hh, torch, vols[f], dims)
    for v in vols:
        v.close()
    pix = _sample_pixels(cams[0], 4000, seed=500, flags=first["flags"])
    ref = oracle_lib.trace_grid(vol4, cams[0], params, bg, pixels=pix, nthreads=16)
    field = {"kind": "grid", "vol4": vol4}
    # rays 1.5 times as long as at 256^3: no more rays are excused than the
    # oracle alone finds ill conditioned in the sample
    st = assert_parity_conditioned(first, ref, oracle_lib, field, dims, cams[0], params, sel=pix,
                                   max_ill_frac=0.03)
    assert st["hits"] >= 1000
    hit_pix = pix[(ref["flags"] & 1) != 0]
    pop_ill = int(ill_conditioned(oracle_lib, field, dims, cams[0], params, hit_pix)[0].sum())
    assert st["n_ill"] <= pop_ill + 2


def test_fullsize_build_384_binned(gpu, oracle_lib):
    """The serving configuration's build at full size: 1,048,576 plume
    particles on 384^3, whose 226 MB density grid is larger than L2, so the
    particles are binned by cell before the splat; the FP32 volume against the
    oracle's splat and Eqs. 12-13 on every voxel."""
    hh, torch = gpu
    L3 = 384
    dims = (L3, L3, L3)
    parts = hi.drifting_plume_frame(hi.plume_particles(1048576, L3), 5, L=L3)
    K = float(np.float32(hi.K_GD))
    vol = hh.hh_build_index_field(torch.from_numpy(parts).cuda(), hh.make_grid(dims, 2.0), K)
    got = export_volume(hh, torch, vol, dims)
    vol.close()
    want = oracle_lib.index_field(oracle_lib.splat(parts, dims, 2.0), K)
    m = np.abs(want[..., 0]).max()
    assert np.abs(got[..., 0] - want[..., 0]).max() <= 2e-5 * m
    assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 2e-5 * m
