"""Invalid arguments come back as HH_ERR_INVALID_ARG with a message; nothing
is launched and the context stays usable."""
import numpy as np
import pytest

import hh_inputs as hi

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


def test_invalid_arguments(gpu):
    hh, torch = gpu
    dims = (16, 16, 16)
    dn = torch.zeros(16**3, device="cuda")
    bad_grids = [hh.make_grid((1, 16, 16)), hh.make_grid((16, 16, 16), 2.0, "fp32")]
    bad_grids[1].storage = 7
    for g in bad_grids:
        with pytest.raises(hh.HHError) as e:
            hh.hh_volume_from_dn(dn, g)
        assert e.value.status == 1
    vol = hh.hh_volume_from_dn(dn, hh.make_grid(dims))
    bg = torch.from_numpy(hi.checker_background()).cuda()
    cam = hi.orbit_camera(dims, 0, 0, 8, 8)
    out = [{"rgb": torch.empty(8 * 8 * 3, device="cuda")}]
    good = hi.params_rk4_fixed(dims)
    before = hh.hh_kernel_launch_count()
    for p in (dict(good, h_fixed=0.0), dict(good, max_steps=-1),
              dict(hi.params_euler_adaptive(dims), eps=0.0),
              dict(hi.params_euler_adaptive(dims), h_min=3.0, h_max=1.0)):
        with pytest.raises(hh.HHError) as e:
            hh.hh_trace(vol, [cam], p, bg, out)
        assert e.value.status == 1 and hh.hh_last_error()
    for c in (dict(cam, width=0), dict(cam, vfov_deg=180.0), dict(cam, look_at=cam["eye"]),
              dict(cam, up=[1.0, 0.0, 0.0])):
        with pytest.raises(hh.HHError):
            hh.hh_trace(vol, [c], good, bg, out)
    with pytest.raises(hh.HHError):
        hh.hh_trace(vol, [cam], good, bg[:1], out)  # background one row high
    assert hh.hh_kernel_launch_count() == before
    # the context is still fine
    hh.hh_trace(vol, [cam], good, bg, out)
    torch.cuda.synchronize()
    assert np.isfinite(out[0]["rgb"].cpu().numpy()).all()
    vol.close()
