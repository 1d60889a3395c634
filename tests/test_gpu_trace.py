"""GPU parity of the curved-ray march (Eqs. 14-18) against the FP64 oracle,
through the C ABI, on the same volume and the same step schedule."""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import (assert_parity_conditioned, assert_parity_plain, export_volume, f32,
                         gpu_trace)

pytestmark = pytest.mark.gpu

NTHREADS = 8


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
def bg(gpu):
    hh, torch = gpu
    b = hi.checker_background()
    return b, torch.from_numpy(b).cuda()


def _dn_volume(hh, torch, dn, storage="fp32"):
    nz, ny, nx = dn.shape
    return hh.hh_volume_from_dn(torch.from_numpy(np.ascontiguousarray(dn).ravel()).cuda(),
                                hh.make_grid((nx, ny, nz), 2.0, storage))


def _particle_volume(hh, torch, parts, dims, storage="fp32"):
    return hh.hh_build_index_field(torch.from_numpy(parts).cuda(),
                                   hh.make_grid(dims, 2.0, storage), f32(hi.K_GD))


def _check(gpu, oracle_lib, vol, dims, cams, params, bg):
    hh, torch = gpu
    cams, params = f32(cams), f32(params)
    got = gpu_trace(hh, torch, vol, cams, params, bg[1])
    vol4 = export_volume(hh, torch, vol, dims)
    field = {"kind": "grid", "vol4": vol4}
    stats = []
    for c, g in zip(cams, got):
        ref = oracle_lib.trace_grid(vol4, c, params, bg[0], nthreads=NTHREADS)
        stats.append(assert_parity_conditioned(g, ref, oracle_lib, field, dims, c, params))
    return stats


# --------------------------------------------------------------------------- #
# the tiny plain-method scene: 64^3 given dn, 128x128 view, RK4 h = 0.5
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("stepper", ["rk4", "euler"])
def test_plume64_fixed_step(gpu, oracle_lib, bg, stepper):
    hh, torch = gpu
    dims = (64, 64, 64)
    vol = _dn_volume(hh, torch, hi.plume_dn_grid(64))
    cam = hi.orbit_camera(dims, 0.0, 0.0, 128, 128)
    params = hi.params_rk4_fixed(dims, 0.5)
    params["stepper"] = stepper
    cam, params = f32(cam), f32(params)
    got = gpu_trace(hh, torch, vol, [cam], params, bg[1])[0]
    vol4 = export_volume(hh, torch, vol, dims)
    ref = oracle_lib.trace_grid(vol4, cam, params, bg[0], nthreads=NTHREADS)
    # a fixed step is well conditioned: every ray within the plain tolerances,
    # no excusal
    st = assert_parity_plain(got, ref, dims)
    assert st["hits"] > 5000 and st["mean_steps"] > 50 and st["n_bad"] == 0


# --------------------------------------------------------------------------- #
# the plume from particles at reduced size, adaptive Eq. 18
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("theta", [hi.THETA_CALIBRATED, hi.THETA_PAPER, 3e-6])
@pytest.mark.parametrize("stepper", ["euler", "rk4"])
def test_particle_plume_adaptive(gpu, oracle_lib, bg, theta, stepper):
    hh, torch = gpu
    L = 96
    dims = (L, L, L)
    vol = _particle_volume(hh, torch, hi.plume_particles(40000, L), dims)
    cam = hi.orbit_camera(dims, 10.0, 5.0, 160, 90)
    params = hi.params_euler_adaptive(dims, theta_max=theta)
    params["stepper"] = stepper
    st = _check(gpu, oracle_lib, vol, dims, [cam], params, bg)[0]
    assert st["hits"] > 3000


# --------------------------------------------------------------------------- #
# ragged shapes and degenerate cases
# --------------------------------------------------------------------------- #
def test_ragged_grid_and_views_in_one_call(gpu, oracle_lib, bg):
    """Non-cubic grid, image sizes that are not multiples of the 16x8 tile, a
    camera inside the volume and a 1x1 view, all in one hh_trace call."""
    hh, torch = gpu
    dims = (50, 37, 29)
    vol = _dn_volume(hh, torch, hi.plume_dn_grid(dims=dims) * 3.0)
    cams = [hi.orbit_camera(dims, 30.0, 20.0, 37, 23),
            {"eye": [20.0, 18.0, 14.0], "look_at": [40.0, 20.0, 10.0], "up": [0, 0, 1],
             "vfov_deg": 75.0, "width": 33, "height": 17},
            hi.orbit_camera(dims, -60.0, -10.0, 1, 1),
            hi.orbit_camera(dims, 200.0, 0.0, 129, 9)]
    params = hi.params_euler_adaptive(dims, theta_max=1e-5, h_min=0.05, h_max=1.5)
    stats = _check(gpu, oracle_lib, vol, dims, cams, params, bg)
    assert stats[1]["hits"] == 33 * 17  # every ray starts inside


@pytest.mark.parametrize("storage,stepper", [("fp32", "euler"), ("fp32", "rk4"), ("fp16", "euler")])
def test_field_up_to_faces_edges_and_corners(gpu, oracle_lib, bg, storage, stepper):
    """Turbulence of constant strength fills the whole box, faces included, on
    a ragged grid: rays that enter through faces, edges and corners and graze
    the faces sample within half a voxel of them, where the lattice
    coordinate is clamped to the voxel centres (the stored halo), and must
    agree with the oracle's clamped trilinear sample."""
    hh, torch = gpu
    dims = (37, 29, 23)
    dn = hi.homogeneous_turbulence_dn(dims, seed=7, sigma=1.5, std=2e-5)
    assert np.abs(dn[:, :, 0]).max() > 1e-5 and np.abs(dn[-1]).max() > 1e-5
    vol = _dn_volume(hh, torch, dn, storage)
    c = [18.5, 14.5, 11.5]
    cams = [hi.orbit_camera(dims, 45.0, 35.3, 48, 40),  # towards a corner
            hi.orbit_camera(dims, 0.0, 0.0, 61, 33, vfov_deg=50.0),
            # grazing: eyes just outside faces, looking along them
            {"eye": [-0.25, -5.0, 11.5], "look_at": [-0.25, 40.0, 11.0], "up": [0, 0, 1],
             "vfov_deg": 20.0, "width": 24, "height": 24},
            {"eye": [18.5, 14.5, 40.0], "look_at": [18.6, 14.4, 0.0], "up": [0, 1, 0],
             "vfov_deg": 95.0, "width": 32, "height": 32},
            {"eye": c, "look_at": [36.9, 28.9, 22.9], "up": [0, 0, 1],
             "vfov_deg": 120.0, "width": 20, "height": 20}]  # from inside, out through every face
    if stepper == "euler":
        params = hi.params_euler_adaptive(dims, theta_max=1e-5, h_min=0.05, h_max=1.0)
    else:
        params = hi.params_rk4_fixed(dims, 0.35)
    stats = _check(gpu, oracle_lib, vol, dims, cams, params, bg)
    assert stats[0]["hits"] > 500 and stats[4]["hits"] == 400


def test_max_steps_and_misses(gpu, oracle_lib, bg):
    """max_steps cuts rays inside the box (MAXSTEPS flag, exit at the current
    position); a camera looking away from the box sees the background along
    its primary rays; max_steps = 0 stops every hit at its entry point."""
    hh, torch = gpu
    dims = (32, 32, 32)
    vol = _dn_volume(hh, torch, hi.plume_dn_grid(dims=dims))
    cam = hi.orbit_camera(dims, 0.0, 0.0, 40, 32)
    away = dict(cam, look_at=[-200.0, 16.0, 16.0])
    for ms in (7, 0):
        params = dict(hi.params_rk4_fixed(dims, 0.5), max_steps=ms)
        st = _check(gpu, oracle_lib, vol, dims, [cam, away], params, bg)
        assert st[0]["hits"] > 200 and st[1]["hits"] == 0


# --------------------------------------------------------------------------- #
# FP16 storage
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("stepper", ["euler", "rk4"])
def test_fp16_storage_parity(gpu, oracle_lib, bg, stepper):
    """The FP16 march against the oracle on the FP16 volume as dequantised."""
    hh, torch = gpu
    L = 80
    dims = (L, L, L)
    vol = _particle_volume(hh, torch, hi.plume_particles(30000, L), dims, "fp16")
    cam = hi.orbit_camera(dims, -20.0, 0.0, 120, 80)
    params = hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED)
    params["stepper"] = stepper
    _check(gpu, oracle_lib, vol, dims, [cam], params, bg)


def test_fp16_precision_against_fp64_truth(gpu, oracle_lib, bg):
    """Precision of FP16 storage (stated, not a parity bar): the FP16 march
    against the FP64 oracle on the FP32 volume, PSNR >= 50 dB."""
    hh, torch = gpu
    L = 80
    dims = (L, L, L)
    parts = hi.plume_particles(30000, L)
    v32 = _particle_volume(hh, torch, parts, dims, "fp32")
    v16 = _particle_volume(hh, torch, parts, dims, "fp16")
    cams = f32(hi.arc_cameras(dims, n=3, width=96, height=54))
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    truth_vol = export_volume(hh, torch, v32, dims)
    got = gpu_trace(hh, torch, v16, cams, params, bg[1])
    for c, g in zip(cams, got):
        ref = oracle_lib.trace_grid(truth_vol, c, params, bg[0], nthreads=NTHREADS)
        mse = np.mean((g["rgb"] - ref["rgb"]) ** 2)
        psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
        assert psnr >= 50.0, psnr


def test_gpu_adaptive_against_converged_truth(gpu, oracle_lib, bg):
    """The GPU's adaptive march (FP32 and FP16 storage) against the converged
    FP64 truth (RK4 of Eq. 15 at 1/64 voxel on the FP32 volume): the errors
    the schedule and the storage leave, reported next to the oracle's own
    adaptive march on the same rays (tests/test_oracle_method_accuracy.py)."""
    hh, torch = gpu
    dims = (64, 64, 64)
    parts = hi.plume_particles(16384, 64)
    v32 = _particle_volume(hh, torch, parts, dims, "fp32")
    v16 = _particle_volume(hh, torch, parts, dims, "fp16")
    cam = f32(hi.orbit_camera(dims, 0.0, 0.0, 128, 128))
    pix = np.arange(0, 128 * 128, 41)
    vol4 = export_volume(hh, torch, v32, dims)
    truth = oracle_lib.trace_grid(vol4, cam, f32(hi.params_rk4_fixed(dims, 1.0 / 64.0)), bg[0],
                                  pixels=pix, nthreads=NTHREADS)
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    own = oracle_lib.trace_grid(vol4, cam, params, bg[0], pixels=pix, nthreads=NTHREADS)
    hit = (truth["flags"] & 1) != 0
    from parity_util import angle

    err = {"oracle": angle(own["exit_dir"][hit], truth["exit_dir"][hit])}
    for name, v in (("gpu_fp32", v32), ("gpu_fp16", v16)):
        g = gpu_trace(hh, torch, v, [cam], params, bg[1])[0]
        err[name] = angle(g["exit_dir"][pix][hit], truth["exit_dir"][hit])
    for k, a in err.items():
        print(f"{k:9s} exit direction vs truth: median {np.median(a):.2e} "
              f"p99 {np.quantile(a, 0.99):.2e} max {a.max():.2e} rad")
    for k in ("gpu_fp32", "gpu_fp16"):
        assert np.median(err[k]) <= 2 * np.median(err["oracle"]) + 1e-7, k
        assert np.quantile(err[k], 0.99) <= 5e-5 and err[k].max() <= 1e-4, k
    v32.close()
    v16.close()


def test_degenerate_grids_steps_and_eyes(gpu, oracle_lib, bg):
    """Edge cases against the oracle: the smallest grid (2^3), a step longer
    than the box (one step crosses it; RK4 stage points far outside), a single
    step per ray, and eyes on a face and at a corner of the box."""
    hh, torch = gpu
    g = np.random.default_rng(21)
    small = (2, 2, 2)
    vol2 = _dn_volume(hh, torch, g.uniform(-1e-3, 1e-3, size=(2, 2, 2)).astype(np.float32))
    cams2 = [hi.orbit_camera(small, 30.0, 20.0, 24, 16), hi.orbit_camera(small, 200.0, -45.0, 9, 9)]
    for params in (hi.params_rk4_fixed(small, 0.25),
                   hi.params_euler_adaptive(small, theta_max=1e-3, h_min=0.05, h_max=0.5)):
        _check(gpu, oracle_lib, vol2, small, cams2, params, bg)
    vol2.close()
    dims = (24, 20, 16)
    vol = _dn_volume(hh, torch, hi.homogeneous_turbulence_dn(dims, seed=3, sigma=1.5, std=3e-5))
    cams = [hi.orbit_camera(dims, 10.0, 5.0, 32, 24),
            {"eye": [0.0, 10.0, 8.0], "look_at": [24.0, 10.0, 8.0], "up": [0, 0, 1],  # on a face
             "vfov_deg": 80.0, "width": 17, "height": 13},
            {"eye": [24.0, 20.0, 16.0], "look_at": [0.0, 0.0, 0.0], "up": [0, 0, 1],  # at a corner
             "vfov_deg": 60.0, "width": 15, "height": 15}]
    for params in (dict(hi.params_rk4_fixed(dims, 50.0)),
                   dict(hi.params_rk4_fixed(dims, 50.0), stepper="euler"),
                   dict(hi.params_rk4_fixed(dims, 0.5), max_steps=1),
                   dict(hi.params_euler_adaptive(dims, theta_max=1e-5), max_steps=1)):
        st = _check(gpu, oracle_lib, vol, dims, cams, params, bg)
        assert st[1]["hits"] > 0 and st[2]["hits"] > 0
    vol.close()
