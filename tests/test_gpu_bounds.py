"""Bounds of the march's volume reads, checked on the device.

The halo layout lets the Eq. 16 march sample without index clamps: every
sample point lies in the box, its lattice coordinate p + 1/2 in
[1/2, n + 1/2], so both trilinear corners lie in the padded axis [0, n + 1].
The bounds-checking build (-DHH_DEBUG_BOUNDS) counts every corner index
outside the padded volume on the device and flags the ray; on tiny grids
(8^3 and ragged ones down to 2^3) and 4x4-pixel views from every side, from
the corners, grazing the faces and from inside, through hh_trace and the
batched launch, with the adaptive and fixed-step Eq. 16 and RK4 marches on
FP32 and FP16 volumes, the count must stay zero. The results are also held
to the oracle, as in the other parity tests.
"""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import assert_parity_conditioned, export_volume, f32, gpu_trace

pytestmark = pytest.mark.gpu

HH_FLAG_CLAMP = 8


@pytest.fixture(scope="module")
def debug_hh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_2603_02048_gb300 import build as hb

    __graft_entry__.build()
    path = hb.build(variant="debug_bounds")
    from paper_2603_02048_gb300 import hh

    # the normal build has no check
    with pytest.raises(hh.HHError):
        hh.hh_debug_bounds_violations()
    return hh, torch, path


def _cameras(dims):
    nx, ny, nz = dims
    c = [nx / 2.0, ny / 2.0, nz / 2.0]
    cams = [hi.orbit_camera(dims, az, el, 4, 4, vfov_deg=70.0)
            for az, el in ((0, 0), (90, 0), (180, 0), (270, 0), (0, 89), (0, -89),
                           (45, 35.3), (225, -35.3), (30, 10))]
    cams += [
        # grazing: eyes just outside a face, looking along it
        {"eye": [-0.01, -3.0, c[2]], "look_at": [-0.01, ny + 3.0, c[2]], "up": [0, 0, 1],
         "vfov_deg": 10.0, "width": 4, "height": 4},
        {"eye": [nx + 0.01, c[1], -3.0], "look_at": [nx + 0.01, c[1], nz + 3.0],
         "up": [0, 1, 0], "vfov_deg": 10.0, "width": 4, "height": 4},
        # along an edge and through a corner
        {"eye": [-3.0, 0.0, 0.0], "look_at": [nx + 3.0, 0.0, 0.0], "up": [0, 0, 1],
         "vfov_deg": 5.0, "width": 4, "height": 4},
        {"eye": [-2.0, -2.0, -2.0], "look_at": [nx, ny, nz], "up": [0, 0, 1],
         "vfov_deg": 5.0, "width": 4, "height": 4},
        # from inside, out through the faces
        {"eye": c, "look_at": [nx, ny, nz], "up": [0, 0, 1], "vfov_deg": 150.0,
         "width": 4, "height": 4},
        # eye on a face
        {"eye": [0.0, c[1], c[2]], "look_at": [nx, c[1], c[2]], "up": [0, 0, 1],
         "vfov_deg": 90.0, "width": 4, "height": 4},
    ]
    return cams


def _schedules(dims):
    return [hi.params_euler_adaptive(dims, theta_max=1e-5, h_min=0.05, h_max=1.0),
            dict(hi.params_euler_adaptive(dims, theta_max=1e-3, h_min=0.05, h_max=3.0)),
            hi.params_rk4_fixed(dims, 0.35),
            dict(hi.params_rk4_fixed(dims, 0.35), stepper="euler"),
            hi.params_rk4_fixed(dims, 20.0)]  # one step crosses the box


@pytest.mark.parametrize("dims", [(8, 8, 8), (3, 5, 7), (2, 2, 2)])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_no_corner_index_leaves_the_padded_volume(debug_hh, oracle_lib, dims, storage):
    hh, torch, path = debug_hh
    dn = hi.homogeneous_turbulence_dn(dims, seed=3, sigma=1.0, std=3e-4) if min(dims) > 2 \
        else np.random.default_rng(5).uniform(-1e-3, 1e-3, size=dims[::-1]).astype(np.float32)
    bg = hi.checker_background()
    cams = f32(_cameras(dims))
    with hh.library(path):
        bg_t = torch.from_numpy(bg).cuda()
        vol = hh.hh_volume_from_dn(torch.from_numpy(np.ascontiguousarray(dn).ravel()).cuda(),
                                   hh.make_grid(dims, 2.0, storage))
        hh.hh_debug_bounds_violations(reset=True)
        vol4 = export_volume(hh, torch, vol, dims)
        field = {"kind": "grid", "vol4": vol4}
        for params in _schedules(dims):
            params = f32(params)
            got = gpu_trace(hh, torch, vol, cams, params, bg_t)
            # the same views through the persistent batched launch (warp refill,
            # and tiles taken by blocks)
            for cfg in ((64, 0, 8, 4), (96, 0, 32, 8, 1, 1)):
                outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device="cuda")}
                        for c in cams]
                b = hh.hh_batch_create(vol, cams, params, bg_t, outs)
                hh.hh_batch_set_config(b, *cfg)
                hh.hh_batch_launch(b)
                torch.cuda.synchronize()
                b.close()
                assert hh.hh_debug_bounds_violations(reset=True) == 0, (params, cfg)
                for g, o in zip(got, outs):
                    assert np.array_equal(o["rgb"].cpu().numpy().reshape(-1, 3),
                                          g["rgb"].astype(np.float32))
            for c, g in zip(cams, got):
                assert not np.any(g["flags"] & HH_FLAG_CLAMP)
                ref = oracle_lib.trace_grid(vol4, c, params, bg, nthreads=4)
                assert_parity_conditioned(g, ref, oracle_lib, field, dims, c, params)
        vol.close()
