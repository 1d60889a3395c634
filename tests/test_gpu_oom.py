"""Out-of-memory paths of every entry point that allocates, driven on demand.

HH_FAIL_ALLOC_AT=k makes the library's k-th device or pinned-host allocation
fail as cudaErrorMemoryAllocation (nothing is allocated). For k = 1, 2, ...
each creator must return HH_ERR_OOM and give back everything it had taken
(hh_live_allocations() returns to its value before the call), until k passes
the number of allocations the call makes and it succeeds. The library stays
usable after every failure. No GPU memory is actually exhausted.
"""
import os

import numpy as np
import pytest

import hh_inputs as hi

pytestmark = pytest.mark.gpu

HH_ERR_OOM = 2


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
def inputs(gpu):
    hh, torch = gpu
    dims = (40, 36, 32)
    parts = hi.plume_particles(5000, 32)
    cams = [hi.orbit_camera(dims, 10.0, 5.0, 24, 16), hi.orbit_camera(dims, 100.0, 0.0, 17, 9)]
    params = hi.params_euler_adaptive(dims, theta_max=1e-5)
    bg = torch.from_numpy(hi.checker_background()).cuda()
    return dims, parts, torch.from_numpy(parts).cuda(), cams, params, bg


def _creators(hh, torch, inputs):
    dims, parts, parts_t, cams, params, bg = inputs
    K = float(np.float32(hi.K_GD))
    grid = hh.make_grid(dims, 2.0, "fp16")

    def build():
        return hh.hh_build_index_field(parts_t, grid, K)

    def batch():
        vol = hh.hh_build_index_field(parts_t, grid, K)
        outs = [{"rgb": torch.empty(c["width"] * c["height"] * 3, device="cuda")} for c in cams]
        try:
            os.environ["HH_FAIL_ALLOC_AT"] = os.environ.pop("HH_FAIL_ALLOC_AT_NEXT")
            return _Pair(hh.hh_batch_create(vol, cams, params, bg, outs), vol)
        except BaseException:
            os.environ.pop("HH_FAIL_ALLOC_AT", None)
            vol.close()
            raise

    def pipeline():
        return hh.hh_pipeline_create(grid, K, len(parts), cams, params, bg)

    def serve():
        return hh.hh_serve_create(1 << 20, 3)

    return {"build": build, "batch": batch, "pipeline": pipeline, "serve": serve}


class _Pair:
    def __init__(self, a, b):
        self.a, self.b = a, b

    def close(self):
        self.a.close()
        self.b.close()


@pytest.mark.parametrize("what,sort", [("build", "0"), ("build", "1"), ("batch", "0"),
                                       ("pipeline", "0"), ("serve", "0")])
def test_every_allocation_failure_returns_oom_and_leaks_nothing(gpu, inputs, what, sort):
    hh, torch = gpu
    os.environ["HH_SPLAT_SORT"] = sort  # "1": the binned splat's scratch is allocated too
    create = _creators(hh, torch, inputs)[what]
    failures = 0
    try:
        for k in range(1, 64):
            live = hh.hh_live_allocations()
            if what == "batch":  # armed after the volume it needs is built
                os.environ["HH_FAIL_ALLOC_AT_NEXT"] = str(k)
            else:
                os.environ["HH_FAIL_ALLOC_AT"] = str(k)
            try:
                obj = create()
            except hh.HHError as e:
                assert e.status == HH_ERR_OOM, (k, str(e))
                assert hh.hh_live_allocations() == live, (k, "leaked")
                failures += 1
                continue
            finally:
                os.environ.pop("HH_FAIL_ALLOC_AT", None)
                os.environ.pop("HH_FAIL_ALLOC_AT_NEXT", None)
            # k is past the call's allocations: it succeeded and still works
            assert hh.hh_live_allocations() > live
            obj.close()
            torch.cuda.synchronize()
            assert hh.hh_live_allocations() == live
            break
        else:
            pytest.fail("the call never succeeded")
    finally:
        os.environ.pop("HH_SPLAT_SORT", None)
    # every allocation of the call was failed once
    assert failures == k - 1 and failures >= {"build": 4, "batch": 2, "pipeline": 6,
                                              "serve": 10}[what] + (2 if sort == "1" else 0)
