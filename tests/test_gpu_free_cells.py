"""The march's free-space skip on fields built to catch a wrong skip.

A volume's free-corner mask marks the voxels (padded lattice indices) that
are the first corner of a trilinear cell whose eight corners are all zero;
the march takes a sample in such a cell as zero without reading the bricks.
Here the field is zero except at single voxels with strong values, placed on
the edges of the 2^3 micro-bricks (padded indices 1-5, 7, 8), at the grid's
faces (whose halo copies are stored too), in the last, partial bricks of
ragged grids and on both sides of the 16-slice runs the mask is built from. A nonzero sample taken for
zero would turn a passing ray by about 1e-3 rad, a thousand times the
tolerance, so every ray is held to the oracle with no excusal (fixed steps,
where the march is well conditioned), from several sides, on FP32 and FP16
volumes, through hh_trace and the batched launch.
"""
import itertools

import numpy as np
import pytest

import hh_inputs as hi
from parity_util import assert_parity_plain, export_volume, f32, gpu_trace

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


def _spikes(dims, seed):
    """Zero dn with single voxels on brick edges, at the faces, in the
    last bricks and at run boundaries: grid index g has padded index g + 1,
    bricks of 2 padded indices, runs of 16 grid slices."""
    nx, ny, nz = dims
    dn = np.zeros((nz, ny, nx))

    def picks(n):
        # grid indices whose padded index g + 1 is 1-5, 7 or 8, the faces and
        # both sides of a run boundary
        return sorted({g for g in (0, 1, 2, 3, 4, 6, 7, 15, 16, n - 2, n - 1) if 0 <= g < n})

    rng = np.random.default_rng(seed)
    for x, y, z in itertools.product(picks(nx), picks(ny), picks(nz)):
        if rng.random() < 0.15:
            dn[z, y, x] = rng.choice([-1.0, 1.0]) * rng.uniform(1e-3, 3e-3)
    return dn


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("dims", [(16, 16, 16), (13, 10, 17), (9, 22, 6), (6, 7, 33)])
def test_isolated_voxels_on_brick_edges(gpu, oracle_lib, dims, storage):
    hh, torch = gpu
    dn = _spikes(dims, seed=sum(dims))
    bg = hi.checker_background()
    bg_t = torch.from_numpy(bg).cuda()
    vol = hh.hh_volume_from_dn(torch.from_numpy(dn.astype(np.float32).ravel()).cuda(),
                               hh.make_grid(dims, 2.0, storage))
    vol4 = export_volume(hh, torch, vol, dims)
    assert np.count_nonzero(vol4[..., 0]) > 4  # the spikes are there
    cams = f32([hi.orbit_camera(dims, az, el, 48, 40, dist_factor=1.2)
                for az, el in ((0.0, 0.0), (90.0, 25.0), (200.0, -40.0), (315.0, 60.0))])
    params = f32(hi.params_euler_adaptive(dims))
    params.update(adaptive=False, h_fixed=0.5, h_min=0.5, h_max=0.5,
                  max_steps=hi.default_max_steps(dims, 0.5))
    got = gpu_trace(hh, torch, vol, cams, params, bg_t)
    # the same views through the batched launch, bit for bit
    outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device="cuda")} for c in cams]
    b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
    hh.hh_batch_set_config(b, 64, 0, 32, 8, 1, 1)
    hh.hh_batch_launch(b)
    torch.cuda.synchronize()
    b.close()
    hits = 0
    for c, g, o in zip(cams, got, outs):
        assert np.array_equal(o["rgb"].cpu().numpy().reshape(-1, 3), g["rgb"].astype(np.float32))
        ref = oracle_lib.trace_grid(vol4, c, params, bg, nthreads=4)
        st = assert_parity_plain(g, ref, dims)
        hits += st["hits"]
        # rays that pass a spike are turned: the field is not skipped wholesale
        assert np.any(g["flags"] & 1)
    assert hits > 500  # of 4 x 1920 pixels (the thin 6 x 7 x 33 grid: ~760)
    vol.close()


def test_rebuild_refreshes_the_free_cells(gpu, oracle_lib):
    """A volume built from a blob in one corner, marched, then rebuilt from a
    blob reaching into the bricks that were free: the march of the rebuilt
    volume must see the new blob (a mask left from the first build would skip
    it and turn the rays that cross it by far more than the tolerance)."""
    hh, torch = gpu
    dims = (48, 48, 48)
    K = float(np.float32(hi.K_GD))
    pa = hi.plume_particles(6000, 24, seed=31)
    pa[:, :3] += 4.0
    pb = hi.plume_particles(6000, 24, seed=32)
    pb[:, :3] += 20.0
    bg = hi.checker_background()
    bg_t = torch.from_numpy(bg).cuda()
    cams = f32([hi.orbit_camera(dims, 20.0, 15.0, 64, 48, dist_factor=1.2)])
    params = f32(hi.params_euler_adaptive(dims))
    params.update(adaptive=False, h_fixed=0.5, h_min=0.5, h_max=0.5,
                  max_steps=hi.default_max_steps(dims, 0.5))
    vol = hh.hh_build_index_field(torch.from_numpy(pa).cuda(), hh.make_grid(dims, 2.0), K)
    first = gpu_trace(hh, torch, vol, cams, params, bg_t)
    hh.hh_volume_rebuild(vol, torch.from_numpy(pb).cuda(), K)
    got = gpu_trace(hh, torch, vol, cams, params, bg_t)
    vol4 = export_volume(hh, torch, vol, dims)
    # the far corner, empty in the first build, holds the second blob
    assert np.abs(vol4[36:44, 36:44, 36:44, 0]).max() > 0.0
    ref = oracle_lib.trace_grid(vol4, cams[0], params, bg, nthreads=4)
    st = assert_parity_plain(got[0], ref, dims)
    assert st["hits"] > 1000
    # and the two builds march differently
    assert not np.array_equal(first[0]["exit_dir"], got[0]["exit_dir"])
    vol.close()
