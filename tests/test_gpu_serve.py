"""The render server (hh_serve_*): continuous batching over slot streams.

Each request's result is the same alone and in a mix of concurrent requests
(bit for bit, and equal to hh_trace); admission respects the memory budget;
requests wait for their frame's volume (bounded waits time out); cancel,
release and invalid calls return statuses. No test faults or hangs a GPU:
every failure here is made on the host."""
import time

import numpy as np
import pytest

import hh_inputs as hi
from parity_util import f32

pytestmark = pytest.mark.gpu

OUTS_ALL = 1 | 2 | 4


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
def frames(gpu):
    hh, torch = gpu
    dims = (64, 64, 64)
    base = hi.plume_particles(40000, 64)
    vols = []
    for t in range(3):
        parts = hi.drifting_plume_frame(base, t, L=64)
        vols.append(hh.hh_build_index_field(torch.from_numpy(parts).cuda(),
                                            hh.make_grid(dims, 2.0, "fp16"), f32(hi.K_GD)))
    torch.cuda.synchronize()
    bg = torch.from_numpy(hi.checker_background()).cuda()
    params = f32(hi.params_euler_adaptive(dims, theta_max=2e-5))
    return dims, vols, bg, params


def _request_views(dims, seed, n):
    return f32(hi.view_mix(dims, n=n, seed=seed,
                           resolutions=((48, 32), (64, 64), (97, 41), (128, 72))))


def _trace_ref(hh, torch, vol, cams, params, bg):
    outs = []
    for c in cams:
        n = c["width"] * c["height"]
        outs.append({"rgb": torch.empty(n * 3, device="cuda"),
                     "exit_pos": torch.empty(n * 3, device="cuda"),
                     "exit_dir": torch.empty(n * 3, device="cuda"),
                     "steps": torch.empty(n, dtype=torch.int32, device="cuda"),
                     "flags": torch.empty(n, dtype=torch.int32, device="cuda")})
    hh.hh_trace(vol, cams, params, bg, outs)
    torch.cuda.synchronize()
    return outs


def _fetch(hh, srv, ticket, cams):
    return [hh.hh_serve_view(srv, ticket, i, c["width"], c["height"]) for i, c in enumerate(cams)]


def _equal(a, b):
    for x, y in zip(a, b):
        for k in ("rgb", "exit_pos", "exit_dir", "steps", "flags"):
            assert bool((x[k] == y[k]).all()), k


def test_alone_equals_in_the_mix(gpu, frames):
    hh, torch = gpu
    dims, vols, bg, params = frames
    srv = hh.hh_serve_create(256 << 20, 4)
    for f, v in enumerate(vols):
        hh.hh_serve_put_volume(srv, f, v)
    probe = _request_views(dims, 11, 3)
    # alone
    t = hh.hh_serve_submit(srv, 1, probe, params, bg, OUTS_ALL)
    hh.hh_serve_wait(srv, t, 20000)
    alone = _fetch(hh, srv, t, probe)
    hh.hh_serve_release(srv, t)
    _equal(alone, _trace_ref(hh, torch, vols[1], probe, params, bg))
    # the same request in a mix of 24 concurrent requests over three frames
    tickets = []
    for i in range(24):
        cams = _request_views(dims, 100 + i, 1 + i % 7)
        tickets.append((hh.hh_serve_submit(srv, i % 3, cams, params, bg, OUTS_ALL), i % 3, cams))
        if i == 11:
            tp = hh.hh_serve_submit(srv, 1, probe, params, bg, OUTS_ALL)
    lat = hh.hh_serve_wait(srv, tp, 20000)
    assert lat > 0
    _equal(alone, _fetch(hh, srv, tp, probe))
    hh.hh_serve_release(srv, tp)
    for t, f, cams in tickets:
        hh.hh_serve_wait(srv, t, 20000)
        _equal(_fetch(hh, srv, t, cams), _trace_ref(hh, torch, vols[f], cams, params, bg))
        hh.hh_serve_release(srv, t)
    st = hh.hh_serve_get_stats(srv)
    assert st["completed"] == 26 and st["pending"] == 0 and st["running"] == 0
    assert st["pool_used"] == 0
    srv.close()


def test_admission_by_memory(gpu, frames):
    """A budget that holds two requests' outputs: every request still
    completes as earlier ones are released (a finished request keeps its
    outputs until released); a request larger than the budget is refused at
    submission."""
    hh, torch = gpu
    dims, vols, bg, params = frames
    cams = f32([hi.orbit_camera(dims, 30.0 * i, 0.0, 128, 128) for i in range(2)])
    one = sum(((c["width"] * c["height"] * 12 + 255) // 256) * 256 for c in cams)
    srv = hh.hh_serve_create(2 * one + 512, 8)
    hh.hh_serve_put_volume(srv, 0, vols[0])
    tickets = [hh.hh_serve_submit(srv, 0, cams, params, bg) for _ in range(7)]
    for t in tickets:
        hh.hh_serve_wait(srv, t, 20000)
        st = hh.hh_serve_get_stats(srv)
        assert st["pool_used"] <= st["pool_capacity"]
        assert st["running"] + st["completed"] - st["admitted"] <= 2
        assert st["admitted"] - (tickets.index(t)) <= 2  # memory, not the 8 slots, limits it
        hh.hh_serve_release(srv, t)
    big = f32([hi.orbit_camera(dims, 0.0, 0.0, 512, 512)])
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_submit(srv, 0, big, params, bg)
    assert e.value.status == 2
    assert hh.hh_serve_get_stats(srv)["rejected"] == 1
    srv.close()


def test_wait_for_frame_timeout_cancel_release(gpu, frames):
    hh, torch = gpu
    dims, vols, bg, params = frames
    srv = hh.hh_serve_create(64 << 20, 2)
    cams = _request_views(dims, 5, 2)
    t = hh.hh_serve_submit(srv, 42, cams, params, bg)  # frame 42 is not there yet
    t0 = time.time()
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_wait(srv, t, 60)
    assert e.value.status == 4 and time.time() - t0 < 5.0  # HH_ERR_TIMEOUT, bounded
    assert hh.hh_serve_poll(srv, t)[0] == 5  # HH_ERR_BUSY: still waiting
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_release(srv, t)  # not finished
    assert e.value.status == 5
    hh.hh_serve_put_volume(srv, 42, vols[2])
    hh.hh_serve_wait(srv, t, 20000)
    hh.hh_serve_release(srv, t)
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_wait(srv, t, 10)
    assert e.value.status == 7  # released: not found
    # cancel a waiting request
    t2 = hh.hh_serve_submit(srv, 99, cams, params, bg)
    hh.hh_serve_cancel(srv, t2)
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_wait(srv, t2, 1000)
    assert e.value.status == 6
    hh.hh_serve_release(srv, t2)
    # a frame in use cannot be replaced; an idle one can be removed
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_remove_volume(srv, 7)
    assert e.value.status == 7
    hh.hh_serve_remove_volume(srv, 42)
    st = hh.hh_serve_get_stats(srv)
    assert st["cancelled"] == 1 and st["completed"] == 1 and st["pool_used"] == 0
    srv.close()


def test_invalid_calls_and_budget_failure(gpu, frames):
    hh, torch = gpu
    dims, vols, bg, params = frames
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_create(1 << 52, 2)  # 4 PiB: the device cannot provide it
    assert e.value.status == 2
    for slots in (0, 65):
        with pytest.raises(hh.HHError):
            hh.hh_serve_create(1 << 20, slots)
    srv = hh.hh_serve_create(1 << 20, 1)
    cams = _request_views(dims, 3, 1)
    with pytest.raises(hh.HHError):
        hh.hh_serve_submit(srv, 0, cams, dict(params, eps=0.0), bg)
    with pytest.raises(hh.HHError):
        hh.hh_serve_submit(srv, 0, [dict(cams[0], width=0)], params, bg)
    with pytest.raises(hh.HHError):
        hh.hh_serve_set_config(srv, 128, 0, 0, 8)
    assert hh.hh_serve_poll(srv, 12345)[0] == 7
    srv.close()


def test_worker_leaves_when_idle_and_comes_back(gpu, frames):
    """The persistent worker's wait for work is bounded: with the queue empty
    its warps leave after about 2 ms (an idle exit), and the next request
    launches it again; results stay hh_trace's."""
    hh, torch = gpu
    dims, vols, bg, params = frames
    srv = hh.hh_serve_create(64 << 20, 4)
    hh.hh_serve_put_volume(srv, 0, vols[0])
    cams = _request_views(dims, 21, 2)
    ref = _trace_ref(hh, torch, vols[0], cams, params, bg)
    for round_ in range(2):
        t = hh.hh_serve_submit(srv, 0, cams, params, bg, OUTS_ALL)
        hh.hh_serve_wait(srv, t, 20000)
        _equal(_fetch(hh, srv, t, cams), ref)
        hh.hh_serve_release(srv, t)
        deadline = time.time() + 5.0
        while hh.hh_serve_get_stats(srv)["worker_idle_exits"] < round_ + 1:
            assert time.time() < deadline, "the worker did not leave its empty queue"
            time.sleep(0.005)
    st = hh.hh_serve_get_stats(srv)
    assert st["worker_launches"] == 2 and st["worker_idle_exits"] == 2
    assert st["completed"] == 2 and st["entry_timeouts"] == 0
    srv.close()


def test_missing_queue_entry_times_out_on_the_device(gpu, frames, monkeypatch):
    """A request whose queue entry never reaches the device (the host drops
    its copy: HH_SERVE_DROP_ENTRY) is failed by the worker's bounded wait with
    HH_ERR_TIMEOUT; the requests before and after it are served as usual."""
    hh, torch = gpu
    dims, vols, bg, params = frames
    srv = hh.hh_serve_create(64 << 20, 4)
    hh.hh_serve_put_volume(srv, 0, vols[0])
    cams = _request_views(dims, 22, 2)
    ref = _trace_ref(hh, torch, vols[0], cams, params, bg)
    monkeypatch.setenv("HH_SERVE_DROP_ENTRY", "2")  # the second job this server publishes
    t1 = hh.hh_serve_submit(srv, 0, cams, params, bg, OUTS_ALL)
    hh.hh_serve_wait(srv, t1, 20000)
    t2 = hh.hh_serve_submit(srv, 0, cams, params, bg, OUTS_ALL)
    t0 = time.time()
    with pytest.raises(hh.HHError) as e:
        hh.hh_serve_wait(srv, t2, 20000)
    assert e.value.status == 4 and time.time() - t0 < 5.0  # HH_ERR_TIMEOUT from the device
    monkeypatch.delenv("HH_SERVE_DROP_ENTRY")
    t3 = hh.hh_serve_submit(srv, 0, cams, params, bg, OUTS_ALL)
    hh.hh_serve_wait(srv, t3, 20000)
    for t in (t1, t3):
        _equal(_fetch(hh, srv, t, cams), ref)
        hh.hh_serve_release(srv, t)
    hh.hh_serve_release(srv, t2)
    st = hh.hh_serve_get_stats(srv)
    assert st["entry_timeouts"] == 1 and st["failed"] == 1 and st["completed"] == 2
    deadline = time.time() + 5.0
    while hh.hh_serve_get_stats(srv)["pool_used"] != 0:  # the failed one's memory comes back
        assert time.time() < deadline
        time.sleep(0.005)
    srv.close()
