"""Thin ctypes binding of the C ABI in include/hh.h, with the same names.

Only argument marshalling happens here: torch tensors are used as device
buffers (their data pointers are passed through), the current torch CUDA
stream is passed as the cudaStream_t, and every status is turned into an
exception. All computation runs in the CUDA kernels of libhh.so. There is no
CPU fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhh.so")

HH_OK = 0
HH_ERR_INVALID_ARG = 1
HH_ERR_OOM = 2
HH_ERR_CUDA = 3
HH_ERR_TIMEOUT = 4
HH_ERR_BUSY = 5
HH_ERR_CANCELLED = 6
HH_ERR_NOT_FOUND = 7
STATUS_NAMES = {0: "HH_OK", 1: "HH_ERR_INVALID_ARG", 2: "HH_ERR_OOM", 3: "HH_ERR_CUDA",
                4: "HH_ERR_TIMEOUT", 5: "HH_ERR_BUSY", 6: "HH_ERR_CANCELLED",
                7: "HH_ERR_NOT_FOUND"}
HH_STORE_FP32 = 0
HH_STORE_FP16_SCALED = 1
HH_STEP_EULER_PAPER = 0
HH_STEP_RK4 = 1
HH_FLAG_HIT = 1
HH_FLAG_EXITED = 2
HH_FLAG_MAXSTEPS = 4

STORAGES = {"fp32": HH_STORE_FP32, "fp16": HH_STORE_FP16_SCALED}
STEPPERS = {"euler": HH_STEP_EULER_PAPER, "rk4": HH_STEP_RK4}


class HHError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class hh_particles(ctypes.Structure):
    _fields_ = [("xyzm_dev", ctypes.c_void_p), ("n", ctypes.c_int64)]


class hh_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h_kernel", ctypes.c_float), ("storage", ctypes.c_int)]


class hh_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("look_at", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("vfov_deg", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class hh_step_params(ctypes.Structure):
    _fields_ = [("stepper", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("h_fixed", ctypes.c_float), ("h_min", ctypes.c_float),
                ("h_max", ctypes.c_float), ("theta_max", ctypes.c_float),
                ("eps", ctypes.c_float), ("max_steps", ctypes.c_int)]


class hh_plane(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("u", ctypes.c_float * 3),
                ("v", ctypes.c_float * 3), ("rgb8_dev", ctypes.c_void_p),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


HH_MAX_PLANES = 4


class hh_background(ctypes.Structure):
    _fields_ = [("rgb8_dev", ctypes.c_void_p), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("n_planes", ctypes.c_int),
                ("planes", hh_plane * HH_MAX_PLANES)]


class hh_view_out(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("exit_pos", ctypes.c_void_p),
                ("exit_dir", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("rgb8", ctypes.c_void_p)]


class hh_batch_config(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("refill_min", ctypes.c_int), ("tile_w", ctypes.c_int),
                ("tile_order", ctypes.c_int), ("tile_group", ctypes.c_int)]


class hh_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("running", ctypes.c_uint64),
                ("rays_completed", ctypes.c_uint64), ("pool_used", ctypes.c_size_t),
                ("pool_capacity", ctypes.c_size_t), ("worker_launches", ctypes.c_uint64),
                ("worker_idle_exits", ctypes.c_uint64), ("entry_timeouts", ctypes.c_uint64)]


HH_OUT_RGB = 1
HH_OUT_EXIT = 2
HH_OUT_STEPS = 4
HH_OUT_RGB8 = 8


# Every symbol include/hh.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
SIGNATURES = {
    "hh_splat_density": (ctypes.c_int, [ctypes.POINTER(hh_particles), ctypes.POINTER(hh_grid),
                                        _P, _P]),
    "hh_volume_from_density": (ctypes.c_int, [_P, ctypes.POINTER(hh_grid), ctypes.c_float, _P,
                                              ctypes.POINTER(_P)]),
    "hh_volume_from_dn": (ctypes.c_int, [_P, ctypes.POINTER(hh_grid), _P, ctypes.POINTER(_P)]),
    "hh_build_index_field": (ctypes.c_int, [ctypes.POINTER(hh_particles),
                                            ctypes.POINTER(hh_grid), ctypes.c_float, _P,
                                            ctypes.POINTER(_P)]),
    "hh_volume_rebuild": (ctypes.c_int, [_P, ctypes.POINTER(hh_particles), ctypes.c_float, _P]),
    "hh_build_index_field_noalloc": (ctypes.c_int, [ctypes.POINTER(hh_particles),
                                                    ctypes.POINTER(hh_grid), ctypes.c_float, _P,
                                                    _P]),
    "hh_volume_export": (ctypes.c_int, [_P, _P, _P]),
    "hh_volume_info": (ctypes.c_int, [_P, ctypes.POINTER(hh_grid),
                                      ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_size_t), _P]),
    "hh_volume_scales": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float)]),
    "hh_volume_free": (ctypes.c_int, [_P]),
    "hh_trace": (ctypes.c_int, [_P, ctypes.POINTER(hh_camera), ctypes.c_int,
                                ctypes.POINTER(hh_step_params), ctypes.POINTER(hh_background),
                                ctypes.POINTER(hh_view_out), _P]),
    "hh_batch_create": (ctypes.c_int, [_P, ctypes.POINTER(hh_camera), ctypes.c_int,
                                       ctypes.POINTER(hh_step_params),
                                       ctypes.POINTER(hh_background), ctypes.POINTER(hh_view_out),
                                       ctypes.POINTER(_P)]),
    "hh_batch_set_config": (ctypes.c_int, [_P, ctypes.POINTER(hh_batch_config)]),
    "hh_batch_get_config": (ctypes.c_int, [_P, ctypes.POINTER(hh_batch_config)]),
    "hh_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(hh_batch_config)]),
    "hh_batch_launch": (ctypes.c_int, [_P, _P]),
    "hh_batch_launch_graph": (ctypes.c_int, [_P, _P]),
    "hh_batch_free": (ctypes.c_int, [_P]),
    "hh_pipeline_create": (ctypes.c_int, [ctypes.POINTER(hh_grid), ctypes.c_float, ctypes.c_int64,
                                          ctypes.POINTER(hh_camera), ctypes.c_int,
                                          ctypes.POINTER(hh_step_params),
                                          ctypes.POINTER(hh_background),
                                          ctypes.POINTER(hh_batch_config), ctypes.POINTER(_P)]),
    "hh_pipeline_submit": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(_P),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "hh_pipeline_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int]),
    "hh_pipeline_volume": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "hh_pipeline_free": (ctypes.c_int, [_P]),
    "hh_serve_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_P)]),
    "hh_serve_set_config": (ctypes.c_int, [_P, ctypes.POINTER(hh_batch_config)]),
    "hh_serve_put_volume": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    "hh_serve_remove_volume": (ctypes.c_int, [_P, ctypes.c_int64]),
    "hh_serve_submit": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(hh_camera), ctypes.c_int,
                                       ctypes.POINTER(hh_step_params),
                                       ctypes.POINTER(hh_background), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "hh_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "hh_serve_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]),
    "hh_serve_view": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.POINTER(hh_view_out)]),
    "hh_serve_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "hh_serve_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "hh_serve_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(hh_serve_stats)]),
    "hh_serve_destroy": (ctypes.c_int, [_P]),
    "hh_last_error": (ctypes.c_char_p, []),
    "hh_kernel_launch_count": (ctypes.c_uint64, []),
    "hh_live_allocations": (ctypes.c_int64, []),
    "hh_debug_bounds_violations": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libhh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with "
                               "python -m paper_2603_02048_gb300.build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != HH_OK:
        raise HHError(status, load().hh_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------- #
# marshalling helpers
# --------------------------------------------------------------------------- #
def make_grid(dims, h_kernel: float = 2.0, storage: str = "fp32") -> hh_grid:
    nx, ny, nz = (int(d) for d in dims)
    return hh_grid(nx, ny, nz, float(h_kernel), STORAGES[storage])


def make_camera(cam: dict) -> hh_camera:
    c = hh_camera()
    c.eye[:] = [float(v) for v in cam["eye"]]
    c.look_at[:] = [float(v) for v in cam["look_at"]]
    c.up[:] = [float(v) for v in cam["up"]]
    c.vfov_deg = float(cam["vfov_deg"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def make_params(p: dict) -> hh_step_params:
    return hh_step_params(STEPPERS[p.get("stepper", "euler")], int(bool(p.get("adaptive"))),
                          float(p.get("h_fixed", 0.5)), float(p.get("h_min", 0.125)),
                          float(p.get("h_max", 2.0)), float(p.get("theta_max", 3e-3)),
                          float(p.get("eps", 1e-6)), int(p["max_steps"]))


def make_background(bg, planes=None) -> hh_background:
    """bg: (H, W, 3) uint8 CUDA tensor (environment map); planes: list of
    dicts {origin, u, v, tex ((h, w, 3) uint8 CUDA tensor)}."""
    B = hh_background()
    B.rgb8_dev = _ptr(bg).value
    B.width, B.height = int(bg.shape[1]), int(bg.shape[0])
    planes = list(planes or [])
    if len(planes) > HH_MAX_PLANES:
        raise ValueError("too many planes")
    B.n_planes = len(planes)
    for k, pl in enumerate(planes):
        P = B.planes[k]
        P.origin[:] = [float(x) for x in pl["origin"]]
        P.u[:] = [float(x) for x in pl["u"]]
        P.v[:] = [float(x) for x in pl["v"]]
        P.rgb8_dev = _ptr(pl["tex"]).value
        P.height, P.width = int(pl["tex"].shape[0]), int(pl["tex"].shape[1])
    return B


def _background(bg) -> hh_background:
    """A ready hh_background, a (map, planes) pair, or a map tensor alone."""
    if isinstance(bg, hh_background):
        return bg
    if isinstance(bg, tuple):
        return make_background(*bg)
    return make_background(bg)


class Volume:
    """Owns an hh_volume handle; freed on close() or garbage collection."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(load().hh_volume_free(self.handle))
        self.handle = None

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                load().hh_volume_free(self.handle)
        except Exception:
            pass


# --------------------------------------------------------------------------- #
# the C-ABI calls, same names
# --------------------------------------------------------------------------- #
def hh_splat_density(xyzm, grid: hh_grid, rho, stream=None):
    """Splat particles (n, 4) float32 CUDA tensor into rho (nz*ny*nx floats)."""
    parts = hh_particles(_ptr(xyzm), int(xyzm.shape[0]))
    _check(load().hh_splat_density(ctypes.byref(parts), ctypes.byref(grid), _ptr(rho),
                                   _stream(stream)))


def hh_volume_from_density(rho, grid: hh_grid, K_gd: float, stream=None) -> Volume:
    out = ctypes.c_void_p()
    _check(load().hh_volume_from_density(_ptr(rho), ctypes.byref(grid), float(K_gd),
                                         _stream(stream), ctypes.byref(out)))
    return Volume(out)


def hh_volume_from_dn(dn, grid: hh_grid, stream=None) -> Volume:
    out = ctypes.c_void_p()
    _check(load().hh_volume_from_dn(_ptr(dn), ctypes.byref(grid), _stream(stream),
                                    ctypes.byref(out)))
    return Volume(out)


def hh_build_index_field(xyzm, grid: hh_grid, K_gd: float, stream=None) -> Volume:
    parts = hh_particles(_ptr(xyzm), int(xyzm.shape[0]))
    out = ctypes.c_void_p()
    _check(load().hh_build_index_field(ctypes.byref(parts), ctypes.byref(grid), float(K_gd),
                                       _stream(stream), ctypes.byref(out)))
    return Volume(out)


def hh_volume_rebuild(vol: Volume, xyzm, K_gd: float, stream=None):
    parts = hh_particles(_ptr(xyzm), int(xyzm.shape[0]))
    _check(load().hh_volume_rebuild(vol.handle, ctypes.byref(parts), float(K_gd),
                                    _stream(stream)))


def hh_build_index_field_noalloc(xyzm, grid: hh_grid, K_gd: float, vol4, stream=None):
    """Allocation-free FP32 build into the caller's vol4 (nz*ny*nx*4 floats)."""
    parts = hh_particles(_ptr(xyzm), int(xyzm.shape[0]))
    _check(load().hh_build_index_field_noalloc(ctypes.byref(parts), ctypes.byref(grid),
                                               float(K_gd), _ptr(vol4), _stream(stream)))


def hh_volume_export(vol: Volume, dst, stream=None):
    _check(load().hh_volume_export(vol.handle, _ptr(dst), _stream(stream)))


def hh_volume_scales(vol: Volume):
    """(s_n, s_g) of the volume (1, 1 for FP32 storage)."""
    s_n, s_g = ctypes.c_float(), ctypes.c_float()
    _check(load().hh_volume_scales(vol.handle, ctypes.byref(s_n), ctypes.byref(s_g)))
    return s_n.value, s_g.value


def hh_volume_info(vol: Volume, stream=None) -> dict:
    g = hh_grid()
    s_n = ctypes.c_float()
    s_g = ctypes.c_float()
    nbytes = ctypes.c_size_t()
    _check(load().hh_volume_info(vol.handle, ctypes.byref(g), ctypes.byref(s_n),
                                 ctypes.byref(s_g), ctypes.byref(nbytes), _stream(stream)))
    return {"dims": (g.nx, g.ny, g.nz), "h_kernel": g.h_kernel, "storage": g.storage,
            "s_n": s_n.value, "s_g": s_g.value, "bytes": nbytes.value}


def hh_volume_free(vol: Volume):
    vol.close()


def hh_trace(vol: Volume, cams, params, bg, outs, stream=None):
    """cams: list of camera dicts or hh_camera; params: dict or hh_step_params;
    bg: (H, W, 3) uint8 CUDA tensor, (map, planes) or an hh_background (the
    tensors must stay alive until the work is done); outs: list of dicts with CUDA tensors
    'rgb' (required) and optional 'exit_pos', 'exit_dir', 'steps', 'flags'."""
    n = len(cams)
    c_cams = (hh_camera * max(n, 1))(*[c if isinstance(c, hh_camera) else make_camera(c)
                                       for c in cams])
    c_outs = (hh_view_out * max(n, 1))(*[
        _view_out(o) for o in outs])
    P = params if isinstance(params, hh_step_params) else make_params(params)
    B = _background(bg)
    _check(load().hh_trace(vol.handle, c_cams, n, ctypes.byref(P), ctypes.byref(B), c_outs,
                           _stream(stream)))


class Batch:
    """Owns an hh_batch handle and keeps its views' buffers alive."""

    def __init__(self, handle: ctypes.c_void_p, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(load().hh_batch_free(self.handle))
        self.handle = None

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                load().hh_batch_free(self.handle)
        except Exception:
            pass


def _views(cams, outs):
    n = len(cams)
    c_cams = (hh_camera * max(n, 1))(*[c if isinstance(c, hh_camera) else make_camera(c)
                                       for c in cams])
    c_outs = (hh_view_out * max(n, 1))(*[
        _view_out(o) for o in outs])
    return n, c_cams, c_outs


def _view_out(o: dict) -> hh_view_out:
    """hh_view_out of a dict of CUDA tensors: rgb (float32) and/or rgb8
    (uint8), and optional exit_pos, exit_dir, steps, flags."""
    return hh_view_out(_ptr(o.get("rgb")), _ptr(o.get("exit_pos")), _ptr(o.get("exit_dir")),
                       _ptr(o.get("steps")), _ptr(o.get("flags")), _ptr(o.get("rgb8")))


def hh_batch_create(vol: Volume, cams, params, bg, outs) -> Batch:
    n, c_cams, c_outs = _views(cams, outs)
    P = params if isinstance(params, hh_step_params) else make_params(params)
    B = _background(bg)
    out = ctypes.c_void_p()
    _check(load().hh_batch_create(vol.handle, c_cams, n, ctypes.byref(P), ctypes.byref(B),
                                  c_outs, ctypes.byref(out)))
    return Batch(out, (vol, bg, outs))


def hh_batch_set_config(b: Batch, block_threads=128, blocks_per_sm=0, refill_min=32, tile_w=8,
                        tile_order=0, tile_group=0):
    c = hh_batch_config(int(block_threads), int(blocks_per_sm), int(refill_min), int(tile_w),
                        int(tile_order), int(tile_group))
    _check(load().hh_batch_set_config(b.handle, ctypes.byref(c)))


def hh_batch_get_config(b: Batch) -> dict:
    c = hh_batch_config()
    _check(load().hh_batch_get_config(b.handle, ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in hh_batch_config._fields_}


def hh_batch_autotune(b: Batch, reps: int = 3, stream=None) -> dict:
    c = hh_batch_config()
    _check(load().hh_batch_autotune(b.handle, int(reps), _stream(stream), ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in hh_batch_config._fields_}


def hh_batch_launch(b: Batch, stream=None):
    _check(load().hh_batch_launch(b.handle, _stream(stream)))


def hh_batch_launch_graph(b: Batch, stream=None):
    _check(load().hh_batch_launch_graph(b.handle, _stream(stream)))


def hh_batch_free(b: Batch):
    b.close()


class Pipeline:
    """Owns an hh_pipeline handle; keeps the background alive, and each
    frame's host buffers until the frame has been waited for."""

    def __init__(self, handle: ctypes.c_void_p, n_views: int, keep):
        self.handle = handle
        self.n_views = n_views
        self._keep = keep
        self._frames = {}  # frame -> its host buffers

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(load().hh_pipeline_free(self.handle))
        self.handle = None
        self._frames.clear()

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                load().hh_pipeline_free(self.handle)
        except Exception:
            pass


def _host_ptr(a):
    """Address of a contiguous host array: a CPU torch tensor (pinned for
    asynchronous copies) or a numpy array."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous host (CPU) tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return ctypes.c_void_p(a.ctypes.data)


def hh_pipeline_create(grid: hh_grid, K_gd: float, max_particles: int, cams, params, bg,
                       cfg=None) -> Pipeline:
    """cfg: None (one hh_trace launch per view) or a dict of hh_batch_config
    fields (the views as one batched launch)."""
    n, c_cams, _ = _views(cams, [{} for _ in cams])
    P = params if isinstance(params, hh_step_params) else make_params(params)
    B = _background(bg)
    C = None if cfg is None else ctypes.byref(hh_batch_config(
        int(cfg["block_threads"]), int(cfg["blocks_per_sm"]), int(cfg["refill_min"]),
        int(cfg["tile_w"]), int(cfg.get("tile_order", 0)), int(cfg.get("tile_group", 0))))
    out = ctypes.c_void_p()
    _check(load().hh_pipeline_create(ctypes.byref(grid), float(K_gd), int(max_particles), c_cams,
                                     n, ctypes.byref(P), ctypes.byref(B), C, ctypes.byref(out)))
    return Pipeline(out, n, (bg, B))


def hh_pipeline_submit(p: Pipeline, xyzm_host, rgb8_host) -> int:
    """xyzm_host: (n, 4) float32 host array; rgb8_host: one host uint8 array
    of H*W*3 bytes per view. Returns the frame number."""
    if len(rgb8_host) != p.n_views:
        raise ValueError(f"expected {p.n_views} image buffers")
    n = int(xyzm_host.shape[0]) if len(xyzm_host.shape) else 0
    imgs = (ctypes.c_void_p * p.n_views)(*[_host_ptr(a) for a in rgb8_host])
    frame = ctypes.c_uint64()
    _check(load().hh_pipeline_submit(p.handle, _host_ptr(xyzm_host) if n else None, n, imgs,
                                     ctypes.byref(frame)))
    p._frames[frame.value] = (xyzm_host, rgb8_host)
    return frame.value


def hh_pipeline_wait(p: Pipeline, frame: int, timeout_ms: int = 60000):
    _check(load().hh_pipeline_wait(p.handle, int(frame), int(timeout_ms)))
    for f in [f for f in p._frames if f <= frame]:
        del p._frames[f]


def hh_pipeline_volume(p: Pipeline) -> Volume:
    """The pipeline's own volume (not owned: do not close it)."""
    out = ctypes.c_void_p()
    _check(load().hh_pipeline_volume(p.handle, ctypes.byref(out)))
    return _BorrowedVolume(out)


class _BorrowedVolume(Volume):
    """A volume handle owned by someone else (close() and collection leave it)."""

    def close(self):
        self.handle = None

    def __del__(self):
        pass


def hh_pipeline_free(p: Pipeline):
    p.close()


class Server:
    """Owns an hh_server handle."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle
        self._frames = {}  # frame id -> the volume the server borrows
        self._bgs = {}     # ticket -> the background its request reads

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(load().hh_serve_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                load().hh_serve_destroy(self.handle)
        except Exception:
            pass


def hh_serve_create(mem_budget_bytes: int, max_slots: int) -> Server:
    out = ctypes.c_void_p()
    _check(load().hh_serve_create(int(mem_budget_bytes), int(max_slots), ctypes.byref(out)))
    return Server(out)


def hh_serve_set_config(s: Server, block_threads=128, blocks_per_sm=0, refill_min=32, tile_w=8,
                        tile_order=0, tile_group=0):
    c = hh_batch_config(int(block_threads), int(blocks_per_sm), int(refill_min), int(tile_w),
                        int(tile_order), int(tile_group))
    _check(load().hh_serve_set_config(s.handle, ctypes.byref(c)))


def hh_serve_put_volume(s: Server, frame_id: int, vol: Volume):
    _check(load().hh_serve_put_volume(s.handle, int(frame_id), vol.handle))
    s._frames[int(frame_id)] = vol


def hh_serve_remove_volume(s: Server, frame_id: int):
    _check(load().hh_serve_remove_volume(s.handle, int(frame_id)))
    s._frames.pop(int(frame_id), None)


def hh_serve_submit(s: Server, frame_id: int, cams, params, bg, outputs: int = HH_OUT_RGB) -> int:
    n = len(cams)
    c_cams = (hh_camera * max(n, 1))(*[c if isinstance(c, hh_camera) else make_camera(c)
                                       for c in cams])
    P = params if isinstance(params, hh_step_params) else make_params(params)
    B = _background(bg)
    t = ctypes.c_uint64()
    _check(load().hh_serve_submit(s.handle, int(frame_id), c_cams, n, ctypes.byref(P),
                                  ctypes.byref(B), int(outputs), ctypes.byref(t)))
    s._bgs[int(t.value)] = bg
    return int(t.value)


def hh_serve_poll(s: Server, ticket: int):
    """Returns (status, latency_ms); status HH_OK, HH_ERR_BUSY, ... (no raise
    for BUSY)."""
    lat = ctypes.c_double(0.0)
    st = load().hh_serve_poll(s.handle, ctypes.c_uint64(ticket), ctypes.byref(lat))
    return st, lat.value


def hh_serve_wait(s: Server, ticket: int, timeout_ms: int = 10000) -> float:
    lat = ctypes.c_double(0.0)
    _check(load().hh_serve_wait(s.handle, ctypes.c_uint64(ticket), int(timeout_ms),
                                ctypes.byref(lat)))
    return lat.value


class _DeviceArray:
    """A __cuda_array_interface__ view of device memory owned elsewhere."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": None}


def hh_serve_view(s: Server, ticket: int, view: int, width: int, height: int) -> dict:
    """Copies of a done request's view outputs as torch CUDA tensors."""
    import torch

    o = hh_view_out()
    _check(load().hh_serve_view(s.handle, ctypes.c_uint64(ticket), int(view), ctypes.byref(o)))
    npx = int(width) * int(height)
    out = {}
    for name, n, ts in (("rgb", npx * 3, "<f4"), ("exit_pos", npx * 3, "<f4"),
                        ("exit_dir", npx * 3, "<f4"), ("steps", npx, "<i4"),
                        ("flags", npx, "<i4"), ("rgb8", npx * 3, "|u1")):
        ptr = getattr(o, name)
        if ptr:
            out[name] = torch.as_tensor(_DeviceArray(ptr, (n,), ts), device="cuda").clone()
    return out


def hh_serve_release(s: Server, ticket: int):
    _check(load().hh_serve_release(s.handle, ctypes.c_uint64(ticket)))
    s._bgs.pop(int(ticket), None)


def hh_serve_cancel(s: Server, ticket: int):
    _check(load().hh_serve_cancel(s.handle, ctypes.c_uint64(ticket)))


def hh_serve_get_stats(s: Server) -> dict:
    st = hh_serve_stats()
    _check(load().hh_serve_get_stats(s.handle, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in hh_serve_stats._fields_}


def hh_serve_destroy(s: Server):
    s.close()


def hh_last_error() -> str:
    return load().hh_last_error().decode()


def hh_kernel_launch_count() -> int:
    return int(load().hh_kernel_launch_count())


def hh_live_allocations() -> int:
    return int(load().hh_live_allocations())


def hh_debug_bounds_violations(reset: bool = True) -> int:
    """Corner indices outside the padded volume counted by a bounds-checking
    build (raises HHError NOT_FOUND on the normal build)."""
    c = ctypes.c_uint64(0)
    _check(load().hh_debug_bounds_violations(ctypes.byref(c), int(bool(reset))))
    return int(c.value)


@contextlib.contextmanager
def library(path: str):
    """Runs the block with the binding on another build of the library (e.g.
    the bounds-checking variant); objects made inside must be freed inside."""
    global _lib
    saved = _lib
    _lib = None
    load(path)
    try:
        yield _lib
    finally:
        _lib = saved
