"""The allocation-free volume build, for callers that cannot allocate device
memory (a host that owns the whole device-memory budget, or a real-time frame
loop that must not pay cudaMalloc's synchronisation and latency).

It is called through the C ABI and must give the same volume as the
allocating entry point (hh_build_index_field, read back with
hh_volume_export), within the build tolerance the other tests use, on two
calls in a row (the second call reuses the fixed device array the first one
filled). This file is collected last so that a failure here never hides the
other tests, and it passes both alone in a fresh process and after them.
"""
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


def _reference(hh, torch, parts_t, dims, K):
    vol = hh.hh_build_index_field(parts_t, hh.make_grid(dims, 2.0, "fp32"), K)
    out = torch.empty(dims[0] * dims[1] * dims[2] * 4, device="cuda")
    hh.hh_volume_export(vol, out)
    torch.cuda.synchronize()
    vol.close()
    return out.cpu().numpy().reshape(dims[2], dims[1], dims[0], 4).astype(np.float64)


def test_noalloc_build_matches_allocating_build_twice(gpu):
    hh, torch = gpu
    K = float(np.float32(hi.K_GD))
    # two different scenes in a row: the second call must not see the first's density
    for dims, n, L in (((128, 128, 128), 60000, 128), ((70, 64, 90), 20000, 64)):
        parts_t = torch.from_numpy(hi.plume_particles(n, L, seed=n)).cuda()
        want = _reference(hh, torch, parts_t, dims, K)
        vol4 = torch.full((dims[0] * dims[1] * dims[2] * 4,), float("nan"), device="cuda")
        hh.hh_build_index_field_noalloc(parts_t, hh.make_grid(dims, 2.0, "fp32"), K, vol4)
        torch.cuda.synchronize()
        got = vol4.cpu().numpy().reshape(dims[2], dims[1], dims[0], 4).astype(np.float64)
        m = np.abs(want[..., 0]).max()
        assert m > 0
        # FP32 atomics accumulate in a different order in each build
        assert np.abs(got[..., 0] - want[..., 0]).max() <= 2e-5 * m
        assert np.abs(got[..., 1:] - want[..., 1:]).max() <= 2e-5 * m


def test_noalloc_rejects_grids_beyond_its_array(gpu):
    hh, torch = gpu
    parts_t = torch.from_numpy(hi.plume_particles(100, 64)).cuda()
    vol4 = torch.empty(4 * 16, device="cuda")
    with pytest.raises(hh.HHError) as e:
        hh.hh_build_index_field_noalloc(parts_t, hh.make_grid((129, 128, 128), 2.0, "fp32"),
                                        1.0, vol4)
    assert e.value.status == 1 and "at most 2097152" in str(e.value)
    with pytest.raises(hh.HHError):
        hh.hh_build_index_field_noalloc(parts_t, hh.make_grid((16, 16, 16), 2.0, "fp16"), 1.0,
                                        vol4)


def test_noalloc_call_allocates_no_device_memory(gpu):
    """What the entry point is for: after a first call (which looks up the
    array's address), further calls leave the device's free memory unchanged."""
    hh, torch = gpu
    K = float(np.float32(hi.K_GD))
    dims = (96, 80, 72)
    parts_t = torch.from_numpy(hi.plume_particles(30000, 72, seed=5)).cuda()
    vol4 = torch.empty(dims[0] * dims[1] * dims[2] * 4, device="cuda")
    grid = hh.make_grid(dims, 2.0, "fp32")
    hh.hh_build_index_field_noalloc(parts_t, grid, K, vol4)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        hh.hh_build_index_field_noalloc(parts_t, grid, K, vol4)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_null_particles(gpu):
    """n > 0 with a NULL particle array is refused before any launch."""
    import ctypes

    hh, torch = gpu
    vol4 = torch.empty(16 * 16 * 16 * 4, device="cuda")
    parts = hh.hh_particles(None, 100)
    grid = hh.make_grid((16, 16, 16), 2.0, "fp32")
    st = hh.load().hh_build_index_field_noalloc(ctypes.byref(parts), ctypes.byref(grid), 1.0,
                                                ctypes.c_void_p(vol4.data_ptr()), None)
    assert st == 1  # HH_ERR_INVALID_ARG
    assert "particles" in hh.hh_last_error()
