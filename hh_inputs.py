"""Seeded synthetic inputs for the curved-ray heat-haze path.

This module holds no arithmetic of the method: it only draws the inputs that
both the CUDA library and the FP64 oracle consume (particle sets, a given dn
grid, backgrounds, cameras, request streams) and the step-parameter presets.
Everything is numpy PCG64 with fixed seeds: scene 0, background 1, view mix 2,
request arrivals 3.

Units are voxels. A grid of R^3 voxels spans the box [0, R]^3 and voxel
(i, j, k) has its centre at (i + 1/2, j + 1/2, k + 1/2). Grids are returned as
(nz, ny, nx) arrays (x fastest in memory). Cameras are plain dicts
{eye, look_at, up, vfov_deg, width, height}.
"""
from __future__ import annotations

import math

import numpy as np

SEED_SCENE = 0
SEED_BACKGROUND = 1
SEED_VIEWS = 2
SEED_ARRIVALS = 3

# Gladstone-Dale constant (m^3/kg) used with rho in kg/m^3 (air, rho0 ~ 1.2).
K_GD = 2.26e-4

# Resolutions of the uneven multi-view batch and of the serving requests.
BATCH_RESOLUTIONS = ((256, 256), (640, 480), (1280, 720), (1920, 1080))
SERVE_RESOLUTIONS = ((320, 240), (1280, 720), (1920, 1080), (3840, 2160))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def voxel_centres(dims):
    """Broadcastable (z, y, x) coordinate arrays of the voxel centres."""
    nx, ny, nz = dims
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    return z[:, None, None], y[None, :, None], x[None, None, :]


# --------------------------------------------------------------------------- #
# scenes
# --------------------------------------------------------------------------- #
def plume_dn_grid(R: int = 64, seed: int = SEED_SCENE, dims=None) -> np.ndarray:
    """Tiny plain-method scene: a given FP32 dn = n - 1 grid.

    dn = -3e-5 exp(-|x - c|^2 / (2 * 12^2)) plus 8 seeded Gaussian blobs with
    amplitude U[-2e-5, 2e-5], sigma U[3, 8] voxels and centres U[8, 56]^3 (for
    R = 64; the centre range and plume width scale with the grid).
    """
    if dims is None:
        dims = (R, R, R)
    nx, ny, nz = dims
    s = np.array([nx, ny, nz], dtype=np.float64) / 64.0
    g = rng(seed)
    z, y, x = voxel_centres(dims)
    c = np.array([nx, ny, nz], dtype=np.float64) / 2.0
    sig = 12.0 * float(np.mean(s))
    dn = -3e-5 * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * sig**2))
    amp = g.uniform(-2e-5, 2e-5, size=8)
    sigma = g.uniform(3.0, 8.0, size=8) * float(np.mean(s))
    centres = g.uniform(8.0, 56.0, size=(8, 3)) * s
    for a, sg, cc in zip(amp, sigma, centres):
        dn = dn + a * np.exp(-((x - cc[0]) ** 2 + (y - cc[1]) ** 2 + (z - cc[2]) ** 2)
                             / (2 * sg**2))
    return np.ascontiguousarray(dn, dtype=np.float32)


def plume_particles(n: int, L: int, seed: int = SEED_SCENE, sigma_frac: float = 0.15,
                    rho0: float = 1.2, h: float = 2.0) -> np.ndarray:
    """SPH particles of a hot plume, (n, 4) float32 {x, y, z, m} in voxel units.

    Positions ~ N(centre, (sigma_frac L)^2) per axis with the z mean raised by
    sigma_frac L / 2 (upward bias). Particles within 2h of a face are redrawn,
    so n is exact and no kernel support crosses the grid boundary. Masses are
    equal, m = rho0 (2 pi)^{3/2} sigma^3 / n, so the plume-centre density is
    about rho0 (kg/m^3 with voxel volume 1).
    """
    g = rng(seed)
    sigma = sigma_frac * L
    mean = np.array([L / 2.0, L / 2.0, L / 2.0 + 0.5 * sigma])
    lo, hi = 2.0 * h, L - 2.0 * h
    pos = np.empty((0, 3))
    while pos.shape[0] < n:
        draw = g.normal(mean, sigma, size=(max(2 * (n - pos.shape[0]), 1024), 3))
        keep = np.all((draw >= lo) & (draw <= hi), axis=1)
        pos = np.concatenate([pos, draw[keep]], axis=0)
    pos = pos[:n]
    m = rho0 * (2 * math.pi) ** 1.5 * sigma**3 / n
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = pos
    out[:, 3] = m
    return out


def drifting_plume_frame(base: np.ndarray, t: int, seed: int = SEED_SCENE,
                         L: int = 384, h: float = 2.0) -> np.ndarray:
    """Frame t of a drifting plume: base + (0, 0, 0.5 t) + N(0, 0.25^2) jitter
    per frame (accumulated), wrapped back into [2h, L - 2h] on z."""
    g = rng(seed * 1000 + 17 + t)
    out = base.copy()
    jitter = g.normal(0.0, 0.25 * math.sqrt(max(t, 1)), size=(base.shape[0], 3))
    out[:, 0] = base[:, 0] + jitter[:, 0]
    out[:, 1] = base[:, 1] + jitter[:, 1]
    out[:, 2] = base[:, 2] + 0.5 * t + jitter[:, 2]
    lo, hi = 2.0 * h, L - 2.0 * h
    span = hi - lo
    for a in range(3):
        out[:, a] = lo + np.mod(out[:, a] - lo, span)
    return np.ascontiguousarray(out, dtype=np.float32)


def sample_field_dn(fn, dims) -> np.ndarray:
    """FP32 grid of dn = fn(x, y, z) evaluated at voxel centres."""
    z, y, x = voxel_centres(dims)
    return np.ascontiguousarray(np.broadcast_to(fn(x, y, z), (dims[2], dims[1], dims[0])),
                                dtype=np.float32)


def random_particles(n: int, dims, seed: int = SEED_SCENE, margin: float = 0.0,
                     mass_range=(0.5, 2.0)) -> np.ndarray:
    """Uniform particles in [margin, dims - margin], masses U[mass_range]."""
    g = rng(seed)
    out = np.empty((n, 4), dtype=np.float32)
    for a in range(3):
        out[:, a] = g.uniform(margin, dims[a] - margin, size=n)
    out[:, 3] = g.uniform(*mass_range, size=n)
    return out


# --------------------------------------------------------------------------- #
# backgrounds
# --------------------------------------------------------------------------- #
def checker_background(W: int = 512, H: int = 512, seed: int = SEED_BACKGROUND,
                       squares: int = 16) -> np.ndarray:
    """RGB8 equirect map: squares x squares checker (levels 0.2 / 0.8) plus
    U[-0.1, 0.1] noise per channel, clipped to [0, 1]."""
    g = rng(seed)
    j = np.arange(H)[:, None]
    i = np.arange(W)[None, :]
    base = np.where(((i * squares // W) + (j * squares // H)) % 2 == 0, 0.2, 0.8)
    img = base[:, :, None] + g.uniform(-0.1, 0.1, size=(H, W, 3))
    return np.ascontiguousarray(np.clip(np.rint(img * 255.0), 0, 255), dtype=np.uint8)


# --------------------------------------------------------------------------- #
# cameras
# --------------------------------------------------------------------------- #
def orbit_camera(dims, azimuth_deg: float, elevation_deg: float, width: int, height: int,
                 dist_factor: float = 1.5, vfov_deg: float = 60.0) -> dict:
    """Camera dist_factor grid widths from the grid centre, looking at it,
    up = +z. Azimuth 0 puts the eye on the -x side looking along +x."""
    nx, ny, nz = dims
    c = np.array([nx, ny, nz], dtype=np.float64) / 2.0
    dist = dist_factor * max(nx, ny, nz)
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    d = np.array([math.cos(az) * math.cos(el), math.sin(az) * math.cos(el), math.sin(el)])
    eye = c - dist * d
    return {"eye": [float(v) for v in eye], "look_at": [float(v) for v in c],
            "up": [0.0, 0.0, 1.0], "vfov_deg": float(vfov_deg),
            "width": int(width), "height": int(height)}


def arc_cameras(dims, n: int = 8, span_deg=(-45.0, 45.0), width: int = 1280,
                height: int = 720) -> list:
    """n views evenly spaced in azimuth over span_deg (a 90 degree arc)."""
    az = np.linspace(span_deg[0], span_deg[1], n)
    return [orbit_camera(dims, float(a), 0.0, width, height) for a in az]


def view_mix(dims, n: int = 32, seed: int = SEED_VIEWS, resolutions=BATCH_RESOLUTIONS) -> list:
    """n views of uneven resolution: resolution uniform over `resolutions`,
    eyes on a sphere of 1.5 grid widths, azimuth U[0, 360), elevation U[-30, 30]."""
    g = rng(seed)
    cams = []
    for _ in range(n):
        w, h = resolutions[int(g.integers(0, len(resolutions)))]
        cams.append(orbit_camera(dims, float(g.uniform(0.0, 360.0)),
                                 float(g.uniform(-30.0, 30.0)), w, h))
    return cams


def serving_requests(rate_hz: float = 200.0, duration_s: float = 2.0, n_frames: int = 60,
                     seed: int = SEED_ARRIVALS, resolutions=SERVE_RESOLUTIONS,
                     max_views: int = 16) -> list:
    """Poisson request stream against a sim clock of n_frames over duration_s.

    Each request: {t, frame, views: [(azimuth, elevation, w, h), ...]} with
    1..max_views views (uniform) at resolutions drawn from `resolutions`."""
    g = rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += float(g.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        frame = min(int(t / duration_s * n_frames), n_frames - 1)
        nv = int(g.integers(1, max_views + 1))
        views = []
        for _ in range(nv):
            w, h = resolutions[int(g.integers(0, len(resolutions)))]
            views.append((float(g.uniform(0.0, 360.0)), float(g.uniform(-30.0, 30.0)), w, h))
        reqs.append({"t": t, "frame": frame, "views": views})
    return reqs


# --------------------------------------------------------------------------- #
# step-parameter presets (voxel units)
# --------------------------------------------------------------------------- #
def default_max_steps(dims, h_min: float) -> int:
    """Three times the box diagonal over the smallest step."""
    diag = math.sqrt(sum(float(d) ** 2 for d in dims))
    return int(math.ceil(3.0 * diag / h_min))


def params_rk4_fixed(dims, h: float = 0.5) -> dict:
    return {"stepper": "rk4", "adaptive": False, "h_fixed": h, "h_min": h, "h_max": h,
            "theta_max": 0.0, "eps": 1e-6, "max_steps": default_max_steps(dims, h)}


def params_euler_adaptive(dims, theta_max: float = 3e-5, h_min: float = 0.125,
                          h_max: float = 2.0, eps: float = 1e-6) -> dict:
    return {"stepper": "euler", "adaptive": True, "h_fixed": h_max, "h_min": h_min,
            "h_max": h_max, "theta_max": theta_max, "eps": eps,
            "max_steps": default_max_steps(dims, h_min)}


# Adaptive tolerances: the paper's value (Sec. 4.1 tolerance sweep) and one
# calibrated to the 256^3 plume so that Eq. 18 actually varies the step.
THETA_PAPER = 3e-3
THETA_CALIBRATED = 3e-5


# --------------------------------------------------------------------------- #
# scene geometry and homogeneous turbulence
# --------------------------------------------------------------------------- #
def checker_texture(W: int = 256, H: int = 256, squares: int = 8, seed: int = SEED_BACKGROUND,
                    tint=(1.0, 1.0, 1.0)) -> np.ndarray:
    """RGB8 checkerboard texture (levels 0.15 / 0.85, U[-0.05, 0.05] noise)."""
    g = rng(seed + 101)
    j = np.arange(H)[:, None]
    i = np.arange(W)[None, :]
    base = np.where(((i * squares // W) + (j * squares // H)) % 2 == 0, 0.15, 0.85)
    img = base[:, :, None] * np.asarray(tint)[None, None, :] + g.uniform(-0.05, 0.05, (H, W, 3))
    return np.ascontiguousarray(np.clip(np.rint(img * 255.0), 0, 255), dtype=np.uint8)


def boards_behind(dims, depths=(0.5, 1.5), size=1.2) -> list:
    """Checkerboard planes facing a camera on the -x side, at x = nx +
    depth * nx, centred on the grid axis, size * nx wide: the 'two boards at
    different distances' of the paper's depth experiment (Sec. 4.2)."""
    nx, ny, nz = dims
    out = []
    for k, dpt in enumerate(depths):
        half = 0.5 * size * nx * (1.0 + dpt)
        out.append({"origin": [nx + dpt * nx, ny / 2 - half, nz / 2 - half],
                    "u": [0.0, 2 * half, 0.0], "v": [0.0, 0.0, 2 * half],
                    "tex": checker_texture(256, 256, squares=8 + 4 * k, seed=10 + k,
                                           tint=(1.0, 0.9 - 0.2 * k, 0.8))})
    return out


def homogeneous_turbulence_dn(dims, seed: int = SEED_SCENE, sigma: float = 2.0,
                              std: float = 1e-5) -> np.ndarray:
    """Statistically homogeneous dn field: white noise filtered by a Gaussian
    of width sigma voxels in Fourier space (periodic, so homogeneous up to the
    faces), scaled to standard deviation `std`. FP32, (nz, ny, nx)."""
    g = rng(seed)
    nx, ny, nz = dims
    noise = g.standard_normal((nz, ny, nx))
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    filt = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    field = np.fft.irfftn(np.fft.rfftn(noise) * filt, s=(nz, ny, nx), axes=(0, 1, 2))
    field *= std / field.std()
    return np.ascontiguousarray(field, dtype=np.float32)
