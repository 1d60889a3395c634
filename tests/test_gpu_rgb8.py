"""The display image (rgb8): exactly round-to-nearest-even of 255 times the
float image clamped to [0, 1], whether the float image is written too or not,
through hh_trace, the batched launch and the render server (integer output:
bit-exact)."""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import f32

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


def _expected_u8(rgb):
    v = np.clip(rgb.astype(np.float32), np.float32(0.0), np.float32(1.0)) * np.float32(255.0)
    return np.rint(v).astype(np.uint8)


def test_rgb8_is_the_quantised_float_image(gpu):
    hh, torch = gpu
    dims = (48, 40, 44)
    vol = hh.hh_build_index_field(torch.from_numpy(hi.plume_particles(20000, 40)).cuda(),
                                  hh.make_grid(dims, 2.0, "fp16"), f32(hi.K_GD))
    cams = f32([hi.orbit_camera(dims, 15.0, 10.0, 61, 37), hi.orbit_camera(dims, 200.0, -20.0, 32, 9)])
    params = f32(hi.params_euler_adaptive(dims, theta_max=1e-5))
    bg = torch.from_numpy(hi.checker_background()).cuda()
    npx = [c["width"] * c["height"] for c in cams]
    both = [{"rgb": torch.empty(n * 3, device="cuda"),
             "rgb8": torch.empty(n * 3, dtype=torch.uint8, device="cuda")} for n in npx]
    hh.hh_trace(vol, cams, params, bg, both)
    only8 = [{"rgb8": torch.empty(n * 3, dtype=torch.uint8, device="cuda")} for n in npx]
    hh.hh_trace(vol, cams, params, bg, only8)
    torch.cuda.synchronize()
    for b, o in zip(both, only8):
        want = _expected_u8(b["rgb"].cpu().numpy())
        assert np.array_equal(b["rgb8"].cpu().numpy(), want)
        assert np.array_equal(o["rgb8"].cpu().numpy(), want)
        assert 0 < want.min() or want.max() > 0  # a real image
    # the batched launch, display image only
    bo = [{"rgb8": torch.empty(n * 3, dtype=torch.uint8, device="cuda")} for n in npx]
    batch = hh.hh_batch_create(vol, cams, params, bg, bo)
    hh.hh_batch_launch(batch)
    torch.cuda.synchronize()
    for b, o in zip(both, bo):
        assert np.array_equal(o["rgb8"].cpu().numpy(), b["rgb8"].cpu().numpy())
    batch.close()
    # the render server, display image only
    srv = hh.hh_serve_create(16 << 20, 2)
    hh.hh_serve_put_volume(srv, 0, vol)
    t = hh.hh_serve_submit(srv, 0, cams, params, bg, hh.HH_OUT_RGB8)
    hh.hh_serve_wait(srv, t, 20000)
    for i, (c, b) in enumerate(zip(cams, both)):
        v = hh.hh_serve_view(srv, t, i, c["width"], c["height"])
        assert "rgb" not in v
        assert np.array_equal(v["rgb8"].cpu().numpy(), b["rgb8"].cpu().numpy())
    hh.hh_serve_release(srv, t)
    srv.close()
    # neither image: refused
    with pytest.raises(hh.HHError):
        hh.hh_trace(vol, cams[:1], params, bg, [{"steps": torch.empty(npx[0], dtype=torch.int32,
                                                                        device="cuda")}])
    vol.close()
