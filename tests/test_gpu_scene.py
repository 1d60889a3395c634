"""Scene geometry behind the volume (textured planes) on the GPU: parity with
the FP64 oracle, bit-identity of the batched path, and the depth statistic
of Eq. 19 (angle-of-arrival variance linear in the turbulent path length)."""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import assert_parity_conditioned, export_volume, f32, gpu_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_02048_gb300 import hh

    return hh, torch


def _device_planes(torch, planes):
    return [dict(p, tex=torch.from_numpy(p["tex"]).cuda()) for p in planes]


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_boards_behind_the_plume(gpu, oracle_lib, storage):
    """Two checkerboards at different depths behind the plume volume, seen
    through it and around it: the image now depends on the exit position."""
    hh, torch = gpu
    dims = (80, 80, 80)
    vol = hh.hh_build_index_field(torch.from_numpy(hi.plume_particles(30000, 80)).cuda(),
                                  hh.make_grid(dims, 2.0, storage), f32(hi.K_GD))
    planes = [dict(p, origin=f32(p["origin"]), u=f32(p["u"]), v=f32(p["v"]))
              for p in hi.boards_behind(dims)]
    env = hi.checker_background()
    scene = (torch.from_numpy(env).cuda(), _device_planes(torch, planes))
    cams = f32([hi.orbit_camera(dims, 0.0, 0.0, 160, 120), hi.orbit_camera(dims, 8.0, 4.0, 97, 61)])
    params = f32(hi.params_euler_adaptive(dims, theta_max=hi.THETA_CALIBRATED))
    got = gpu_trace(hh, torch, vol, cams, params, scene)
    vol4 = export_volume(hh, torch, vol, dims)
    for c, g in zip(cams, got):
        ref = oracle_lib.trace_grid(vol4, c, params, env, nthreads=8, planes=planes)
        env_only = oracle_lib.trace_grid(vol4, c, params, env, nthreads=8)
        assert np.abs(ref["rgb"] - env_only["rgb"]).max() > 0.3  # the boards are in view
        assert_parity_conditioned(g, ref, oracle_lib, {"kind": "grid", "vol4": vol4}, dims, c,
                                  params)
    # the batched path sees the same scene, bit for bit
    outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device="cuda")} for c in cams]
    b = hh.hh_batch_create(vol, cams, params, scene, outs)
    hh.hh_batch_set_config(b, 128, 0, 8, 8)
    hh.hh_batch_launch(b)
    torch.cuda.synchronize()
    for o, g in zip(outs, got):
        assert np.array_equal(o["rgb"].cpu().numpy().reshape(-1, 3), g["rgb"].astype(np.float32))
    b.close()


def test_invalid_planes_rejected(gpu):
    hh, torch = gpu
    dims = (16, 16, 16)
    vol = hh.hh_volume_from_dn(torch.zeros(16**3, device="cuda"), hh.make_grid(dims))
    env = torch.from_numpy(hi.checker_background(64, 32)).cuda()
    tex = torch.from_numpy(hi.checker_texture(8, 8)).cuda()
    cam = hi.orbit_camera(dims, 0, 0, 8, 8)
    out = [{"rgb": torch.empty(8 * 8 * 3, device="cuda")}]
    P = hi.params_rk4_fixed(dims)
    good = {"origin": [20.0, 0.0, 0.0], "u": [0.0, 16.0, 0.0], "v": [0.0, 0.0, 16.0], "tex": tex}
    for bad in (dict(good, u=[0.0, 0.0, 0.0]), dict(good, v=[0.0, 1.0, 1.0]),
                dict(good, origin=[float("nan"), 0.0, 0.0]), dict(good, tex=tex[:1])):
        with pytest.raises(hh.HHError):
            hh.hh_trace(vol, [cam], P, (env, [bad]), out)
    with pytest.raises((hh.HHError, ValueError)):  # the binding refuses it first
        hh.hh_trace(vol, [cam], P, (env, [good] * 5), out)
    B = hh.make_background(env, [good])
    B.n_planes = 5  # past the binding: the library refuses it
    with pytest.raises(hh.HHError):
        hh.hh_trace(vol, [cam], P, B, out)
    hh.hh_trace(vol, [cam], P, (env, [good]), out)
    torch.cuda.synchronize()
    vol.close()


def _gpu_slab_variance(hh, torch, Lz, seeds=range(8)):
    """Mean squared exit deflection of near-parallel rays (a far, narrow
    camera below the slab) through homogeneous turbulence of thickness Lz."""
    dims = (64, 64, Lz)
    cam = f32({"eye": [32.0, 32.0, -20000.0], "look_at": [32.0, 32.0, 0.0], "up": [0, 1, 0],
               "vfov_deg": float(np.degrees(2 * np.arctan(31.0 / 20000.0))),
               "width": 32, "height": 32})
    P = f32(hi.params_rk4_fixed(dims, 0.5))
    env = torch.from_numpy(hi.checker_background()).cuda()
    flat = hh.hh_volume_from_dn(torch.zeros(64 * 64 * Lz, device="cuda"), hh.make_grid(dims))
    straight = gpu_trace(hh, torch, flat, [cam], P, env)[0]["exit_dir"]
    d2 = []
    for s in seeds:
        dn = hi.homogeneous_turbulence_dn(dims, seed=100 + s, sigma=2.0)
        vol = hh.hh_volume_from_dn(torch.from_numpy(dn.ravel()).cuda(), hh.make_grid(dims))
        g = gpu_trace(hh, torch, vol, [cam], P, env)[0]
        assert np.all(g["flags"] == 3)
        d2.append(np.sum((g["exit_dir"] - straight) ** 2, axis=1))
        vol.close()
    flat.close()
    return float(np.mean(np.concatenate(d2)))


def test_angle_of_arrival_variance_linear_in_path(gpu):
    """Eq. 19 on the GPU path: the deflection variance doubles with the slab
    thickness, as in the oracle (tests/test_oracle_pins.py)."""
    hh, torch = gpu
    v = [_gpu_slab_variance(hh, torch, L) for L in (24, 48, 96)]
    assert 1.75 < v[1] / v[0] < 2.3 and 1.75 < v[2] / v[1] < 2.3, v
