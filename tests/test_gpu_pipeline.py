"""The real-time frame pipeline (hh_pipeline_*): host particles in, host
display images out, two frames in flight. Each frame's images are
hh_trace's on the pipeline's own volume (bit for bit, integer output), for
one view (hh_trace launches) and several (one batched launch); frames run
with two in flight give the same images; empty frames and bad calls."""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import f32

pytestmark = pytest.mark.gpu

DIMS = (40, 36, 44)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_02048_gb300 import hh

    return hh, torch


def _frames(n_frames, n_particles):
    """A drifting plume: the base particles moved up by 0.5 voxel per frame."""
    base = hi.plume_particles(n_particles, 36)
    out = []
    for t in range(n_frames):
        p = base.copy()
        p[:, 2] += 0.5 * t
        out.append(p)
    return out


def _pinned(torch, a):
    return torch.from_numpy(a).pin_memory()


def _trace_rgb8(hh, torch, vol, cams, params, bg_t):
    outs = [{"rgb8": torch.empty(c["width"] * c["height"] * 3, dtype=torch.uint8,
                                 device="cuda")} for c in cams]
    hh.hh_trace(vol, cams, params, bg_t, outs)
    torch.cuda.synchronize()
    return [o["rgb8"].cpu().numpy() for o in outs]


@pytest.mark.parametrize("batched", [False, True])
def test_pipeline_frames_equal_trace(gpu, batched):
    hh, torch = gpu
    cams = f32([hi.orbit_camera(DIMS, 20.0, 10.0, 64, 40)] if not batched else
               [hi.orbit_camera(DIMS, a, e, w, h)
                for a, e, w, h in ((20.0, 10.0, 64, 40), (140.0, -15.0, 33, 17),
                                   (260.0, 25.0, 48, 48))])
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=1e-5))
    bg_t = torch.from_numpy(hi.checker_background()).cuda()
    frames = _frames(4, 6000)
    cfg = {"block_threads": 128, "blocks_per_sm": 0, "refill_min": 32, "tile_w": 8}
    pipe = hh.hh_pipeline_create(hh.make_grid(DIMS, 2.0, "fp16"), f32(hi.K_GD), 6000, cams,
                                 params, bg_t, cfg if batched else None)
    # one frame at a time: each image against hh_trace on the frame's volume
    # (the two slots' volumes alternate)
    serial = []
    vols = set()
    for t, parts in enumerate(frames):
        imgs = [_pinned(torch, np.zeros(c["width"] * c["height"] * 3, np.uint8)) for c in cams]
        f = hh.hh_pipeline_submit(pipe, _pinned(torch, parts), imgs)
        assert f == t
        hh.hh_pipeline_wait(pipe, f)
        vol = hh.hh_pipeline_volume(pipe)
        vols.add(vol.handle.value)
        want = _trace_rgb8(hh, torch, vol, cams, params, bg_t)
        for a, b in zip(imgs, want):
            assert np.array_equal(a.numpy(), b)
        serial.append([a.numpy().copy() for a in imgs])
    assert any(not np.array_equal(serial[0][0], s[0]) for s in serial[1:])  # frames differ
    assert len(vols) == 2  # one volume per slot
    # two frames in flight: the same images (the FP32 atomics of the splat may
    # change a last bit of the volume between builds: at most one display level)
    imgs = [[_pinned(torch, np.zeros(c["width"] * c["height"] * 3, np.uint8)) for c in cams]
            for _ in frames]
    ids = []
    for t, parts in enumerate(frames):
        ids.append(hh.hh_pipeline_submit(pipe, _pinned(torch, parts), imgs[t]))
        if t >= 1:
            hh.hh_pipeline_wait(pipe, ids[t - 1])
    hh.hh_pipeline_wait(pipe, ids[-1])
    assert ids == [4, 5, 6, 7]
    for t in range(len(frames)):
        for a, b in zip(imgs[t], serial[t]):
            d = np.abs(a.numpy().astype(int) - b.astype(int))
            assert d.max() <= 1 and np.count_nonzero(d) <= 0.001 * d.size
    hh.hh_pipeline_wait(pipe, 0)  # long done
    pipe.close()


def test_pipeline_empty_frame_and_errors(gpu):
    hh, torch = gpu
    cams = f32([hi.orbit_camera(DIMS, 75.0, 5.0, 24, 20)])
    params = f32(hi.params_euler_adaptive(DIMS, theta_max=1e-5))
    bg_t = torch.from_numpy(hi.checker_background()).cuda()
    pipe = hh.hh_pipeline_create(hh.make_grid(DIMS, 2.0, "fp32"), f32(hi.K_GD), 100, cams,
                                 params, bg_t)
    img = [np.zeros(24 * 20 * 3, np.uint8)]  # pageable host memory works too
    f = hh.hh_pipeline_submit(pipe, np.zeros((0, 4), np.float32), img)
    hh.hh_pipeline_wait(pipe, f)
    want = _trace_rgb8(hh, torch, hh.hh_pipeline_volume(pipe), cams, params, bg_t)
    assert np.array_equal(img[0], want[0]) and img[0].max() > 0
    with pytest.raises(hh.HHError) as e:
        hh.hh_pipeline_submit(pipe, np.zeros((101, 4), np.float32), img)  # over max_particles
    assert e.value.status == hh.HH_ERR_INVALID_ARG
    with pytest.raises(hh.HHError) as e:
        hh.hh_pipeline_wait(pipe, 5)  # not submitted
    assert e.value.status == hh.HH_ERR_NOT_FOUND
    with pytest.raises(ValueError):
        hh.hh_pipeline_submit(pipe, np.zeros((1, 4), np.float32), img + img)
    pipe.close()
    with pytest.raises(hh.HHError) as e:
        hh.hh_pipeline_create(hh.make_grid(DIMS, 2.0, "fp32"), f32(hi.K_GD), 10, [], params,
                              bg_t)
    assert e.value.status == hh.HH_ERR_INVALID_ARG
