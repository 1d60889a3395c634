"""FP64 CPU oracle for the curved-ray heat-haze hot path (arXiv 2603.02048, Sec. 3.3).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The CUDA
library (``paper_2603_02048_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``hh_oracle.c`` (plain C, double precision); this module
compiles it with gcc into ``liboracle.so`` and wraps it with ctypes + numpy.
Array conventions: grids are numpy arrays of shape (nz, ny, nx) (x fastest in
memory), volumes (nz, ny, nx, 4) with channels {dn, gx, gy, gz}; images
(H, W, 3); positions in voxel units.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

FLAG_HIT = 1
FLAG_EXITED = 2
FLAG_MAXSTEPS = 4

FIELD_KINDS = {"grid": 0, "constant": 1, "stratified": 2, "spherical": 3, "luneburg": 4}
STEPPERS = {"euler": 0, "rk4": 1}


def build(force: bool = False) -> str:
    """Compiles hh_oracle.c into liboracle.so (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB_PATH)
    except subprocess.CalledProcessError as e:  # pragma: no cover - build failure path
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed:\n{e.stderr}") from e
    return _LIB_PATH


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dims", ctypes.c_int * 3),
                ("vol4", ctypes.POINTER(ctypes.c_double)),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("sigma", ctypes.c_double), ("radius", ctypes.c_double),
                ("center", ctypes.c_double * 3)]


class _Params(ctypes.Structure):
    _fields_ = [("stepper", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("h_fixed", ctypes.c_double), ("h_min", ctypes.c_double),
                ("h_max", ctypes.c_double), ("theta_max", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_steps", ctypes.c_int)]


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("look_at", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("vfov_deg", ctypes.c_double),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class _Plane(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("u", ctypes.c_double * 3),
                ("v", ctypes.c_double * 3), ("rgb8", ctypes.POINTER(ctypes.c_uint8)),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class _Scene(ctypes.Structure):
    _fields_ = [("rgb8", ctypes.POINTER(ctypes.c_uint8)), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("n_planes", ctypes.c_int),
                ("planes", _Plane * 4)]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.hho_kernel_m4.restype = ctypes.c_double
        lib.hho_kernel_m4.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.hho_splat.argtypes = [_F, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, _D]
        lib.hho_index_field.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _D]
        lib.hho_trilinear4.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        lib.hho_march_ray.restype = ctypes.c_int
        lib.hho_march_ray.argtypes = [ctypes.POINTER(_Field), _D, _D, _D, ctypes.POINTER(_Params),
                                      _D, _D, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_uint32), _D, ctypes.c_int]
        lib.hho_camera_ray.argtypes = [ctypes.POINTER(_Camera), ctypes.c_int, ctypes.c_int, _D]
        lib.hho_slab.restype = ctypes.c_int
        lib.hho_slab.argtypes = [_D, _D, _D, _D, _D]
        lib.hho_background.argtypes = [ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                       ctypes.c_int, _D, _D]
        lib.hho_scene_color.argtypes = [ctypes.POINTER(_Scene), _D, _D, _D]
        trace_args = [ctypes.POINTER(_Camera), ctypes.POINTER(_Params), ctypes.POINTER(_Scene),
                      ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _D, _D, _D,
                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32),
                      ctypes.c_int]
        lib.hho_trace_field.argtypes = [ctypes.POINTER(_Field), _D] + trace_args
        lib.hho_trace_grid.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int] + trace_args
        lib.hho_march_rays.argtypes = [ctypes.POINTER(_Field), _D, _D, _D, ctypes.c_int64,
                                       ctypes.POINTER(_Params), _D, _D,
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _vec3(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


# --------------------------------------------------------------------------- #
# wrappers
# --------------------------------------------------------------------------- #
def kernel_m4(r: float, h: float) -> float:
    """M4 cubic spline W(r, h) (Sec. 3.3.1 splat kernel)."""
    return _load().hho_kernel_m4(float(r), float(h))


def splat(xyzm: np.ndarray, dims, h: float) -> np.ndarray:
    """rho at voxel centres from particles xyzm (N, 4) float32 {x, y, z, m}."""
    xyzm = np.ascontiguousarray(xyzm, dtype=np.float32).reshape(-1, 4)
    nx, ny, nz = (int(d) for d in dims)
    rho = np.zeros((nz, ny, nx), dtype=np.float64)
    _load().hho_splat(_ptr(xyzm, ctypes.c_float), xyzm.shape[0], nx, ny, nz, float(h),
                      _ptr(rho, ctypes.c_double))
    return rho


def index_field(rho: np.ndarray, K: float) -> np.ndarray:
    """{dn, gx, gy, gz} per voxel from rho (nz, ny, nx): Eqs. 12-13."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    vol4 = np.zeros((nz, ny, nx, 4), dtype=np.float64)
    _load().hho_index_field(_ptr(rho, ctypes.c_double), nx, ny, nz, float(K),
                            _ptr(vol4, ctypes.c_double))
    return vol4


def trilinear4(vol4: np.ndarray, p) -> np.ndarray:
    vol4 = np.ascontiguousarray(vol4, dtype=np.float64)
    nz, ny, nx, _ = vol4.shape
    out = np.zeros(4)
    p = _vec3(p)
    _load().hho_trilinear4(_ptr(vol4, ctypes.c_double), nx, ny, nz, _ptr(p, ctypes.c_double),
                           _ptr(out, ctypes.c_double))
    return out


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    for k in ("eye", "look_at", "up"):
        getattr(c, k)[:] = [float(x) for x in cam[k]]
    c.vfov_deg = float(cam["vfov_deg"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def _params(p: dict) -> _Params:
    q = _Params()
    q.stepper = STEPPERS[p.get("stepper", "euler")]
    q.adaptive = int(bool(p.get("adaptive", False)))
    q.h_fixed = float(p.get("h_fixed", 0.5))
    q.h_min = float(p.get("h_min", 0.125))
    q.h_max = float(p.get("h_max", 2.0))
    q.theta_max = float(p.get("theta_max", 3e-3))
    q.eps = float(p.get("eps", 1e-6))
    q.max_steps = int(p["max_steps"])
    return q


class _FieldHolder:
    """Keeps the numpy volume alive while the C struct points into it."""

    def __init__(self, spec: dict):
        self.f = _Field()
        kind = spec["kind"]
        self.f.kind = FIELD_KINDS[kind]
        self.vol = None
        if kind == "grid":
            self.vol = np.ascontiguousarray(spec["vol4"], dtype=np.float64)
            nz, ny, nx, _ = self.vol.shape
            self.f.dims[:] = [nx, ny, nz]
            self.f.vol4 = _ptr(self.vol, ctypes.c_double)
        self.f.a = float(spec.get("a", 0.0))
        self.f.b = float(spec.get("b", 0.0))
        self.f.sigma = float(spec.get("sigma", 1.0))
        self.f.radius = float(spec.get("radius", 1.0))
        self.f.center[:] = [float(x) for x in spec.get("center", (0.0, 0.0, 0.0))]


def camera_ray(cam: dict, px: int, py: int) -> np.ndarray:
    d = np.zeros(3)
    c = _camera(cam)
    _load().hho_camera_ray(ctypes.byref(c), int(px), int(py), _ptr(d, ctypes.c_double))
    return d


def slab(o, d, box):
    o, d, box = _vec3(o), _vec3(d), _vec3(box)
    tin = np.zeros(1)
    tout = np.zeros(1)
    hit = _load().hho_slab(_ptr(o, ctypes.c_double), _ptr(d, ctypes.c_double),
                           _ptr(box, ctypes.c_double), _ptr(tin, ctypes.c_double),
                           _ptr(tout, ctypes.c_double))
    return bool(hit), float(tin[0]), float(tout[0])


def background(bg: np.ndarray, d) -> np.ndarray:
    bg = np.ascontiguousarray(bg, dtype=np.uint8)
    H, W, _ = bg.shape
    d = _vec3(d)
    out = np.zeros(3)
    _load().hho_background(_ptr(bg, ctypes.c_uint8), W, H, _ptr(d, ctypes.c_double),
                           _ptr(out, ctypes.c_double))
    return out


def march_ray(field: dict, box, C0, w0, params: dict, path_cap: int = 0) -> dict:
    """One ray from C0 along unit w0 through an analytic or gridded field."""
    holder = _FieldHolder(field)
    box, C0, w0 = _vec3(box), _vec3(C0), _vec3(w0)
    P = _params(params)
    ep = np.zeros(3)
    ed = np.zeros(3)
    steps = ctypes.c_int32(0)
    flags = ctypes.c_uint32(0)
    path = np.zeros((max(path_cap, 1), 7))
    _load().hho_march_ray(ctypes.byref(holder.f), _ptr(box, ctypes.c_double),
                          _ptr(C0, ctypes.c_double), _ptr(w0, ctypes.c_double), ctypes.byref(P),
                          _ptr(ep, ctypes.c_double), _ptr(ed, ctypes.c_double),
                          ctypes.byref(steps), ctypes.byref(flags),
                          _ptr(path, ctypes.c_double) if path_cap > 0 else None, int(path_cap))
    out = {"exit_pos": ep, "exit_dir": ed, "steps": int(steps.value), "flags": int(flags.value)}
    if path_cap > 0:
        out["path"] = path[: min(out["steps"], path_cap)]
    return out


def march_rays(field: dict, box, C0: np.ndarray, w0: np.ndarray, params: dict,
               nthreads: int = 1) -> dict:
    """Marches many rays from given start points C0 (n, 3) and unit directions
    w0 (n, 3); returns exit_pos, exit_dir, steps, flags per ray."""
    holder = _FieldHolder(field)
    box = _vec3(box)
    C0 = np.ascontiguousarray(C0, dtype=np.float64).reshape(-1, 3)
    w0 = np.ascontiguousarray(w0, dtype=np.float64).reshape(-1, 3)
    n = C0.shape[0]
    P = _params(params)
    ep = np.zeros((n, 3))
    ed = np.zeros((n, 3))
    steps = np.zeros(n, dtype=np.int32)
    flags = np.zeros(n, dtype=np.uint32)
    _load().hho_march_rays(ctypes.byref(holder.f), _ptr(box, ctypes.c_double),
                           _ptr(C0, ctypes.c_double), _ptr(w0, ctypes.c_double), n,
                           ctypes.byref(P), _ptr(ep, ctypes.c_double), _ptr(ed, ctypes.c_double),
                           _ptr(steps, ctypes.c_int32), _ptr(flags, ctypes.c_uint32),
                           int(nthreads))
    return {"exit_pos": ep, "exit_dir": ed, "steps": steps, "flags": flags}


class _SceneHolder:
    """A C scene over the environment map and up to 4 textured planes
    (dicts {origin, u, v, tex (H, W, 3) uint8}); keeps the arrays alive."""

    def __init__(self, bg: np.ndarray, planes=None):
        self.arrays = [np.ascontiguousarray(bg, dtype=np.uint8)]
        self.s = _Scene()
        H, W, _ = self.arrays[0].shape
        self.s.rgb8 = _ptr(self.arrays[0], ctypes.c_uint8)
        self.s.width, self.s.height = W, H
        planes = list(planes or [])
        assert len(planes) <= 4
        self.s.n_planes = len(planes)
        for k, pl in enumerate(planes):
            tex = np.ascontiguousarray(pl["tex"], dtype=np.uint8)
            self.arrays.append(tex)
            p = self.s.planes[k]
            p.origin[:] = [float(x) for x in pl["origin"]]
            p.u[:] = [float(x) for x in pl["u"]]
            p.v[:] = [float(x) for x in pl["v"]]
            p.rgb8 = _ptr(tex, ctypes.c_uint8)
            p.height, p.width = tex.shape[0], tex.shape[1]


def scene_color(bg: np.ndarray, P, d, planes=None) -> np.ndarray:
    """What the straight ray P + t d (t > 0) sees: nearest plane, else the map."""
    sc = _SceneHolder(bg, planes)
    P, d = _vec3(P), _vec3(d)
    out = np.zeros(3)
    _load().hho_scene_color(ctypes.byref(sc.s), _ptr(P, ctypes.c_double),
                            _ptr(d, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def _trace(fn, lead_args, cam, params, bg, pixels, nthreads, planes=None):
    c = _camera(cam)
    P = _params(params)
    sc = _SceneHolder(bg, planes)
    if pixels is None:
        n = int(cam["width"]) * int(cam["height"])
        pix_ptr = None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        n = pixels.shape[0]
        pix_ptr = _ptr(pixels, ctypes.c_int64)
    rgb = np.zeros((n, 3))
    ep = np.zeros((n, 3))
    ed = np.zeros((n, 3))
    steps = np.zeros(n, dtype=np.int32)
    flags = np.zeros(n, dtype=np.uint32)
    fn(*lead_args, ctypes.byref(c), ctypes.byref(P), ctypes.byref(sc.s),
       pix_ptr, n, _ptr(rgb, ctypes.c_double), _ptr(ep, ctypes.c_double),
       _ptr(ed, ctypes.c_double), _ptr(steps, ctypes.c_int32), _ptr(flags, ctypes.c_uint32),
       int(nthreads))
    return {"rgb": rgb, "exit_pos": ep, "exit_dir": ed, "steps": steps, "flags": flags}


def trace_grid(vol4: np.ndarray, cam: dict, params: dict, bg: np.ndarray, pixels=None,
               nthreads: int = 1, planes=None) -> dict:
    """Traces camera pixels through a gridded {dn, g} volume (nz, ny, nx, 4).

    Returns per-pixel arrays rgb (n,3), exit_pos (n,3), exit_dir (n,3),
    steps (n,), flags (n,), in row-major pixel order or the order of ``pixels``.
    """
    vol4 = np.ascontiguousarray(vol4, dtype=np.float64)
    nz, ny, nx, _ = vol4.shape
    return _trace(_load().hho_trace_grid, (_ptr(vol4, ctypes.c_double), nx, ny, nz), cam,
                  params, bg, pixels, nthreads, planes)


def trace_field(field: dict, box, cam: dict, params: dict, bg: np.ndarray, pixels=None,
                nthreads: int = 1, planes=None) -> dict:
    """Traces camera pixels through an analytic (or gridded) field in box [0, box]."""
    holder = _FieldHolder(field)
    box = _vec3(box)
    out = _trace(_load().hho_trace_field, (ctypes.byref(holder.f), _ptr(box, ctypes.c_double)),
                 cam, params, bg, pixels, nthreads, planes)
    del holder
    return out
