"""The persistent batched multi-view launch (hh_batch_*): bit-identical to
hh_trace view by view under every launch shape (tile shape, block size,
warp-level compaction threshold, occupancy), through CUDA-graph replays and
after autotuning; and a sample checked against the FP64 oracle."""
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


def _outs(torch, cams):
    outs = []
    for c in cams:
        n = c["width"] * c["height"]
        outs.append({"rgb": torch.full((n * 3,), -1.0, device="cuda"),
                     "exit_pos": torch.full((n * 3,), -1.0, device="cuda"),
                     "exit_dir": torch.full((n * 3,), -1.0, device="cuda"),
                     "steps": torch.full((n,), -1, dtype=torch.int32, device="cuda"),
                     "flags": torch.full((n,), -1, dtype=torch.int32, device="cuda")})
    return outs


def _host(torch, outs):
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


def _mixed_views(dims):
    cams = hi.view_mix(dims, n=6, seed=7, resolutions=((37, 23), (64, 64), (129, 9), (96, 54)))
    cams.append({"eye": [dims[0] / 2 - 3.0, dims[1] / 2, dims[2] / 2],
                 "look_at": [dims[0], dims[1] / 2 + 2.0, dims[2] / 2], "up": [0, 0, 1],
                 "vfov_deg": 70.0, "width": 41, "height": 29})  # starts inside the volume
    cams.append(hi.orbit_camera(dims, 10.0, 0.0, 1, 1))
    return f32(cams)


@pytest.fixture(scope="module")
def scene(gpu):
    hh, torch = gpu
    L = 72
    dims = (L, 64, 80)
    parts = hi.plume_particles(30000, 64)
    parts_t = torch.from_numpy(parts).cuda()
    bg = hi.checker_background()
    return dims, parts_t, bg, torch.from_numpy(bg).cuda()


# (block_threads, blocks_per_sm, refill_min, tile_w, tile_order, tile_group):
# tile-at-a-time and warp refill, every tile shape, views one after the other and
# interleaved, tiles taken by warps and by blocks (a block of 96 threads leaves a
# group of 3 tiles that straddles view boundaries and the last, partial group)
CONFIGS = [(128, 0, 32, 8, 0, 0), (64, 0, 1, 8, 1, 0), (256, 2, 8, 4, 0, 0),
           (96, 1, 16, 16, 1, 0), (32, 3, 31, 8, 0, 0), (128, 0, 32, 8, 1, 0),
           (256, 0, 32, 4, 1, 0), (256, 0, 32, 8, 0, 1), (96, 2, 32, 16, 1, 1),
           (64, 0, 32, 4, 0, 1), (32, 0, 32, 8, 1, 1)]


@pytest.mark.parametrize("storage,stepper,adaptive",
                         [("fp32", "euler", True), ("fp16", "euler", True),
                          ("fp32", "rk4", False), ("fp16", "rk4", True)])
def test_batch_bit_identical_to_trace(gpu, scene, storage, stepper, adaptive):
    hh, torch = gpu
    dims, parts_t, _, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, storage), f32(hi.K_GD))
    cams = _mixed_views(dims)
    params = f32(hi.params_euler_adaptive(dims, theta_max=2e-5) if adaptive
                 else hi.params_rk4_fixed(dims, 0.7))
    params["stepper"] = stepper
    ref_outs = _outs(torch, cams)
    hh.hh_trace(vol, cams, params, bg_t, ref_outs)
    ref = _host(torch, ref_outs)
    assert sum(int((r["flags"] & 1).sum()) for r in ref) > 1000
    for cfg in CONFIGS:
        outs = _outs(torch, cams)
        b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
        hh.hh_batch_set_config(b, *cfg)
        hh.hh_batch_launch(b)
        got = _host(torch, outs)
        for r, g in zip(ref, got):
            for k in r:
                np.testing.assert_array_equal(g[k], r[k], err_msg=f"{cfg} {k}")
        b.close()
    vol.close()


def test_graph_replays_and_autotune(gpu, scene):
    hh, torch = gpu
    dims, parts_t, _, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp16"), f32(hi.K_GD))
    cams = _mixed_views(dims)
    params = f32(hi.params_euler_adaptive(dims, theta_max=2e-5))
    ref_outs = _outs(torch, cams)
    hh.hh_trace(vol, cams, params, bg_t, ref_outs)
    ref = _host(torch, ref_outs)
    outs = _outs(torch, cams)
    b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(3):  # capture, then two replays
            for o in outs:
                for v in o.values():
                    v.fill_(-1)
            hh.hh_batch_launch_graph(b, stream)
            got = _host(torch, outs)
            for r, g in zip(ref, got):
                for k in r:
                    np.testing.assert_array_equal(g[k], r[k])
        best = hh.hh_batch_autotune(b, reps=2, stream=stream)
        assert best["tile_w"] in (4, 8, 16) and 1 <= best["refill_min"] <= 32
        assert hh.hh_batch_get_config(b)["block_threads"] == best["block_threads"]
        assert hh.hh_batch_autotune(b, reps=2, stream=stream) == best  # cached
        hh.hh_batch_launch_graph(b, stream)
        got = _host(torch, outs)
    for r, g in zip(ref, got):
        for k in r:
            np.testing.assert_array_equal(g[k], r[k])
    b.close()
    vol.close()


def test_batch_against_oracle(gpu, scene, oracle_lib):
    hh, torch = gpu
    dims, parts_t, bg, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp32"), f32(hi.K_GD))
    cams = _mixed_views(dims)
    params = f32(hi.params_euler_adaptive(dims, theta_max=2e-5))
    outs = _outs(torch, cams)
    b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
    hh.hh_batch_set_config(b, 128, 0, 8, 8)
    hh.hh_batch_launch(b)
    got = _host(torch, outs)
    vol4 = export_volume(hh, torch, vol, dims)
    for c, g in zip(cams, got):
        g = {"rgb": g["rgb"].reshape(-1, 3).astype(np.float64),
             "exit_pos": g["exit_pos"].reshape(-1, 3).astype(np.float64),
             "exit_dir": g["exit_dir"].reshape(-1, 3).astype(np.float64),
             "steps": g["steps"], "flags": g["flags"].view(np.uint32)}
        ref = oracle_lib.trace_grid(vol4, c, params, bg, nthreads=8)
        assert_parity_conditioned(g, ref, oracle_lib, {"kind": "grid", "vol4": vol4}, dims, c,
                                  params)
    b.close()


def test_batch_rejects_bad_configs(gpu, scene):
    hh, torch = gpu
    dims, parts_t, _, bg_t = scene
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp32"), f32(hi.K_GD))
    cams = _mixed_views(dims)[:2]
    outs = _outs(torch, cams)
    b = hh.hh_batch_create(vol, cams, f32(hi.params_rk4_fixed(dims)), bg_t, outs)
    for cfg in ((0, 0, 32, 8), (100, 0, 32, 8), (128, -1, 32, 8), (128, 0, 0, 8),
                (128, 0, 33, 8), (128, 0, 32, 6), (128, 0, 32, 8, 2), (128, 0, 32, 8, -1),
                (128, 0, 32, 8, 0, 2), (128, 0, 32, 8, 0, -1), (128, 0, 16, 8, 0, 1)):
        with pytest.raises(hh.HHError):
            hh.hh_batch_set_config(b, *cfg)
    with pytest.raises(hh.HHError):
        hh.hh_batch_launch_graph(b, 0)  # the legacy default stream cannot be captured
    b.close()
    vol.close()
