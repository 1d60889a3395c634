"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks a closed form, an
invariant of the ray equation (Eqs. 14-15), a convergence order, a property
the paper states (Eq. 18 bounds the turning angle per step), or brute force on
tiny inputs. A dropped term, a wrong sign, index or factor anywhere in the
oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import hh_inputs as hi

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# --------------------------------------------------------------------------- #
# Splat kernel and splat (Sec. 3.3.1)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("h", [0.7, 2.0, 3.5])
def test_kernel_normalised_and_compact(oracle_lib, h):
    """Any SPH density kernel integrates to one over space and vanishes at its
    support radius; W(0) of the M4 spline is 1/(pi h^3)."""
    o = oracle_lib
    total, err = integrate.quad(lambda r: o.kernel_m4(r, h) * 4 * math.pi * r * r, 0, 2 * h,
                                points=[h], epsabs=1e-13, epsrel=1e-13)
    assert abs(total - 1.0) < 1e-10
    assert o.kernel_m4(2 * h, h) == 0.0
    assert o.kernel_m4(2 * h + 1e-9, h) == 0.0
    assert o.kernel_m4(0.0, h) == pytest.approx(1.0 / (math.pi * h**3), rel=1e-15)


def test_kernel_smooth_at_piece_joins(oracle_lib):
    """The M4 spline is C2: value and slope agree on both sides of q = 1 and
    the value goes to zero like (2 - q)^3 at q = 2."""
    o = oracle_lib
    h = 2.0
    d = 1e-4
    W = [o.kernel_m4(h + k * d, h) for k in range(-3, 4)]  # W[3] at q = 1
    # one-sided quotients use only points of one piece each
    v_l = 3 * W[2] - 3 * W[1] + W[0]  # quadratic extrapolation to q = 1
    v_r = 3 * W[4] - 3 * W[5] + W[6]
    assert abs(v_l - W[3]) < 1e-10 and abs(v_r - W[3]) < 1e-10
    s_l = (W[2] - W[1]) / d
    s_r = (W[5] - W[4]) / d
    c_l = (W[2] - 2 * W[1] + W[0]) / d**2
    c_r = (W[6] - 2 * W[5] + W[4]) / d**2
    assert abs(s_l - s_r) < 3 * d * max(abs(c_l), abs(c_r)) + 1e-9
    assert abs(c_l - c_r) < 1e-3 * max(abs(c_l), abs(c_r)) + 1e-6
    near = o.kernel_m4(2 * h - 1e-2, h) / (1e-2 / h) ** 3
    assert near == pytest.approx(0.25 / (math.pi * h**3), rel=2e-2)


def test_splat_brute_force_all_voxels(oracle_lib):
    """Bounding-box restricted splat == brute force over every voxel and
    particle (non-cubic grid, particles near faces and outside the grid)."""
    o = oracle_lib
    dims = (11, 7, 9)
    parts = hi.random_particles(25, dims, seed=5, margin=-2.0)
    h = 1.3
    rho = o.splat(parts, dims, h)
    nx, ny, nz = dims
    ref = np.zeros((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = 0.0
                for x, y, z, m in parts.astype(np.float64):
                    r = math.sqrt((i + 0.5 - x) ** 2 + (j + 0.5 - y) ** 2 + (k + 0.5 - z) ** 2)
                    s += m * o.kernel_m4(r, h)
                ref[k, j, i] = s
    np.testing.assert_allclose(rho, ref, rtol=1e-13, atol=1e-15)


def test_splat_mass_conservation(oracle_lib):
    """For particles away from the faces, sum(rho) * voxel volume ~ sum(m):
    the unit-lattice sum of a kernel with support 4 voxels is 1 to ~1e-3."""
    o = oracle_lib
    dims = (40, 40, 40)
    parts = hi.random_particles(300, dims, seed=7, margin=5.0)
    rho = o.splat(parts, dims, 2.0)
    assert abs(rho.sum() / parts[:, 3].astype(np.float64).sum() - 1.0) < 1e-3


def test_splat_axis_permutation(oracle_lib):
    """Swapping the x and y coordinates of every particle transposes rho."""
    o = oracle_lib
    dims = (13, 9, 6)
    parts = hi.random_particles(40, dims, seed=9)
    rho = o.splat(parts, dims, 1.5)
    sw = parts.copy()
    sw[:, [0, 1]] = parts[:, [1, 0]]
    rho_sw = o.splat(sw, (9, 13, 6), 1.5)
    np.testing.assert_allclose(rho_sw, rho.transpose(0, 2, 1), rtol=1e-14, atol=1e-16)


# --------------------------------------------------------------------------- #
# Gladstone-Dale + finite differences (Eqs. 12-13)
# --------------------------------------------------------------------------- #
def test_index_field_linear_exact(oracle_lib):
    """dn = K rho; for a linear rho every difference (central and one-sided at
    the faces) is exact: g = K (beta, gamma, delta) everywhere."""
    dims = (7, 5, 4)
    K = 2.26e-4
    z, y, x = hi.voxel_centres(dims)
    rho = 1.2 + 0.3 * x - 0.7 * y + 0.11 * z + 0 * x * y * z
    vol = oracle_lib.index_field(rho, K)
    np.testing.assert_allclose(vol[..., 0], K * rho, rtol=1e-15)
    for c, slope in zip((1, 2, 3), (0.3, -0.7, 0.11)):
        np.testing.assert_allclose(vol[..., c], K * slope, rtol=1e-11)


def test_index_field_quadratic(oracle_lib):
    """rho = x^2 + 2 y^2 - z^2: central differences are exact for a quadratic;
    a one-sided difference equals the derivative half a voxel inward."""
    dims = (6, 5, 7)
    z, y, x = hi.voxel_centres(dims)
    rho = x**2 + 2 * y**2 - z**2
    vol = oracle_lib.index_field(rho, 1.0)
    gx = np.broadcast_to(2 * x, rho.shape).copy()
    gy = np.broadcast_to(4 * y, rho.shape).copy()
    gz = np.broadcast_to(-2 * z, rho.shape).copy()
    gx[:, :, 0] = 2 * 1.0
    gx[:, :, -1] = 2 * (dims[0] - 1.0)
    gy[:, 0, :] = 4 * 1.0
    gy[:, -1, :] = 4 * (dims[1] - 1.0)
    gz[0] = -2 * 1.0
    gz[-1] = -2 * (dims[2] - 1.0)
    np.testing.assert_allclose(vol[..., 1], gx, atol=1e-12)
    np.testing.assert_allclose(vol[..., 2], gy, atol=1e-12)
    np.testing.assert_allclose(vol[..., 3], gz, atol=1e-12)


def test_index_field_second_order(oracle_lib):
    """Inside the grid the central difference of a Gaussian converges to the
    analytic derivative as dx^2 (ratio 4 when the voxel is halved)."""
    errs = []
    for scale in (1, 2):
        n = 24 * scale
        dims = (n, n, n)
        z, y, x = hi.voxel_centres(dims)
        s = 5.0 * scale
        c = n / 2
        f = np.exp(-((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) / (2 * s * s))
        vol = oracle_lib.index_field(f, 1.0)
        # derivative in units of the coarse voxel: d/dx (scaled) * scale
        gx_true = -(x - c) / (s * s) * f
        sl = slice(2 * scale, n - 2 * scale)
        errs.append(np.abs(vol[sl, sl, sl, 1] - gx_true[sl, sl, sl]).max() * scale)
    assert 3.6 < errs[0] / errs[1] < 4.4


# --------------------------------------------------------------------------- #
# Trilinear sampling (Sec. 3.3.1)
# --------------------------------------------------------------------------- #
def test_trilinear_reproduces_multilinear(oracle_lib):
    """Trilinear interpolation over voxel centres is exact for any function
    a + bx + cy + dz + exy + fyz + gxz + hxyz, per channel (non-cubic grid)."""
    dims = (6, 4, 5)
    z, y, x = hi.voxel_centres(dims)
    coef = np.array([[0.3, 1.1, -0.4, 0.2, 0.05, -0.02, 0.03, 0.01],
                     [1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0],
                     [0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                     [0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]])

    def ml(c, x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z
                + c[6] * x * z + c[7] * x * y * z)

    vol = np.stack([np.broadcast_to(ml(c, x, y, z), (5, 4, 6)) for c in coef], axis=-1)
    r = np.random.default_rng(3)
    for _ in range(50):
        p = r.uniform([0.5, 0.5, 0.5], [5.5, 3.5, 4.5])
        got = oracle_lib.trilinear4(vol, p)
        want = [ml(c, *p) for c in coef]
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # outside the centres the lattice coordinate is clamped to the edge
    got = oracle_lib.trilinear4(vol, [0.1, 3.9, -2.0])
    want = [ml(c, 0.5, 3.5, 0.5) for c in coef]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------- #
# Camera, entry, background
# --------------------------------------------------------------------------- #
def test_camera_pinhole_geometry(oracle_lib):
    """Rays are unit; projected onto the image plane (d / (d.f) - f) they form
    a square-pixel lattice of pitch 2 tan(vfov/2) / H centred on the axis;
    row 0 is up (+z) and the first column is on the left (+y when looking
    along +x with z up)."""
    cam = {"eye": [-10.0, 2.0, 3.0], "look_at": [5.0, 2.0, 3.0], "up": [0, 0, 1],
           "vfov_deg": 50.0, "width": 7, "height": 4}
    t = math.tan(math.radians(25.0))
    pitch = 2 * t / 4
    f = np.array([1.0, 0, 0])
    for py in range(4):
        for px in range(7):
            d = oracle_lib.camera_ray(cam, px, py)
            assert abs(np.linalg.norm(d) - 1) < 1e-15
            q = d / d.dot(f) - f
            # right = f x up = -y, screen-up = +z
            assert q[1] == pytest.approx(-(px + 0.5 - 3.5) * pitch, abs=1e-14)
            assert q[2] == pytest.approx(-(py + 0.5 - 2.0) * pitch, abs=1e-14)
    one = dict(cam, width=1, height=1)
    np.testing.assert_allclose(oracle_lib.camera_ray(one, 0, 0), f, atol=1e-15)


def test_slab_entry_exit(oracle_lib):
    box = [10.0, 6.0, 4.0]
    hit, tin, tout = oracle_lib.slab([-5, 3, 2], [1, 0, 0], box)
    assert hit and tin == 5.0 and tout == 15.0
    hit, tin, tout = oracle_lib.slab([5, 3, 2], [0, -1, 0], box)
    assert hit and tin == -3.0 and tout == 3.0
    assert not oracle_lib.slab([-5, 7, 2], [1, 0, 0], box)[0]  # parallel, outside
    assert not oracle_lib.slab([-5, 3, 2], [-1, 0, 0], box)[0]  # behind the eye
    d = np.array([10.0, 6.0, 4.0]) / np.linalg.norm([10, 6, 4])
    hit, tin, tout = oracle_lib.slab([0, 0, 0], d, box)
    assert hit and tin == pytest.approx(0) and tout == pytest.approx(math.sqrt(152))


def test_background_conventions(oracle_lib):
    """A ramp map returns its own bilinear texel coordinates: the red channel
    encodes the column, green the row. Fixes phi = atan2(y, x) on u,
    polar angle from +z on v, the half-texel centres, the clamp in v and the
    wrap in u."""
    W, H = 256, 128
    bg = np.zeros((H, W, 3), dtype=np.uint8)
    bg[..., 0] = np.arange(W)[None, :]
    bg[..., 1] = np.arange(H)[:, None] * 2
    B = oracle_lib.background
    c = B(bg, [1, 0, 0]) * 255
    assert c[0] == pytest.approx(W / 2 - 0.5) and c[1] == pytest.approx(2 * (H / 2 - 0.5))
    c = B(bg, [0, 1, 0]) * 255
    assert c[0] == pytest.approx(3 * W / 4 - 0.5)
    c = B(bg, [0, -1, 0]) * 255
    assert c[0] == pytest.approx(W / 4 - 0.5)
    assert B(bg, [0, 0, 1])[1] == 0.0  # pole: clamped to row 0
    assert B(bg, [0, 0, -1])[1] * 255 == pytest.approx(2 * (H - 1))
    c = B(bg, [math.cos(0.3), 0, math.sin(0.3)]) * 255  # 0.3 rad above the horizon
    assert c[1] == pytest.approx(2 * (((math.pi / 2 - 0.3) / math.pi) * H - 0.5))
    # seam: phi = pi lands half-way between the last column and column 0
    c = B(bg, [-1, 0, 0]) * 255
    assert c[0] == pytest.approx(0.5 * (W - 1))
    flat = np.full((8, 16, 3), 77, dtype=np.uint8)
    r = np.random.default_rng(1)
    for _ in range(10):
        np.testing.assert_allclose(B(flat, r.normal(size=3)), 77 / 255, atol=1e-15)


# --------------------------------------------------------------------------- #
# The march (Eqs. 14-18)
# --------------------------------------------------------------------------- #
BOX = [64.0, 64.0, 64.0]


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("stepper", ["euler", "rk4"])
def test_constant_index_straight_chord(oracle_lib, stepper):
    """Constant n: the ray is the straight chord; it exits at the slab exit
    point with its direction unchanged after ceil(chord / h) steps."""
    w0 = _unit([1.0, 0.37, -0.21])
    C0 = np.array([0.0, 20.0, 40.0])
    hit, tin, tout = oracle_lib.slab(C0, w0, BOX)
    for adaptive, h in ((False, 0.7), (True, 2.0)):
        P = {"stepper": stepper, "adaptive": adaptive, "h_fixed": h, "h_min": 0.1, "h_max": h,
             "theta_max": 3e-3, "eps": 1e-6, "max_steps": 10000}
        r = oracle_lib.march_ray({"kind": "constant", "a": 0.02}, BOX, C0, w0, P)
        np.testing.assert_allclose(r["exit_pos"], C0 + tout * w0, atol=1e-11)
        np.testing.assert_allclose(r["exit_dir"], w0, atol=1e-15)
        assert r["steps"] == math.ceil(tout / h)
        assert r["flags"] == oracle_lib.FLAG_EXITED


def _invariant_drift(oracle_lib, field, inv, C0, w0, stepper, h, n_steps):
    P = {"stepper": stepper, "adaptive": False, "h_fixed": h, "max_steps": 100000}
    r = oracle_lib.march_ray(field, BOX, C0, w0, P, path_cap=n_steps + 1)
    path = r["path"]
    assert path.shape[0] > n_steps, "ray left the box before the comparison point"
    return abs(inv(path[n_steps, :3], path[n_steps, 3:6]) - inv(path[0, :3], path[0, 3:6]))


def _snell(field):
    a, b = field["a"], field["b"]
    return lambda C, w: (1 + a + b * C[2]) * math.hypot(w[0], w[1])


def _bouguer(field):
    c = np.array(field["center"])

    def inv(C, w):
        r = C - c
        n = 1 + field["a"] * math.exp(-r.dot(r) / (2 * field["sigma"] ** 2))
        return n * np.linalg.norm(np.cross(r, w))
    return inv


STRAT = {"kind": "stratified", "a": 0.0, "b": 0.5 / 64}
SPH = {"kind": "spherical", "a": 0.3, "sigma": 9.0, "center": [32.0, 32.0, 32.0]}


@pytest.mark.parametrize("field,inv,C0,w0", [
    (STRAT, _snell(STRAT), [0.0, 10.0, 5.0], _unit([1.0, 0.3, 0.6])),
    (SPH, _bouguer(SPH), [0.0, 36.0, 30.0], _unit([1.0, 0.0, 0.05])),
])
def test_invariants_converge_euler_first_order(oracle_lib, field, inv, C0, w0):
    """Snell's n |w_xy| (stratified n) and Bouguer's n |r x w| (spherical n)
    are conserved by Eq. 14; Eq. 16 conserves them to O(h)."""
    L = 48.0
    d = [_invariant_drift(oracle_lib, field, inv, C0, w0, "euler", h, int(L / h))
         for h in (0.5, 0.25, 0.125)]
    assert d[0] > 1e-6
    assert 1.7 < d[0] / d[1] < 2.3 and 1.7 < d[1] / d[2] < 2.3


@pytest.mark.parametrize("field,inv,C0,w0", [
    (STRAT, _snell(STRAT), [0.0, 10.0, 5.0], _unit([1.0, 0.3, 0.6])),
    (SPH, _bouguer(SPH), [0.0, 36.0, 30.0], _unit([1.0, 0.0, 0.05])),
])
def test_invariants_converge_rk4_fourth_order(oracle_lib, field, inv, C0, w0):
    L = 48.0
    d = [_invariant_drift(oracle_lib, field, inv, C0, w0, "rk4", h, int(L / h))
         for h in (4.0, 2.0)]
    assert d[1] > 1e-12
    assert 11.0 < d[0] / d[1] < 22.0


def _luneburg_exit(b, R=20.0, c=32.0, box=64.0):
    """Closed form: a ray entering a Luneburg lens parallel to +x at impact
    parameter b (units of the radius) leaves the sphere at the far focus
    c + (R, 0, 0) with direction (sqrt(1-b^2), -b, 0), then runs straight."""
    wx, wy = math.sqrt(1 - b * b), -b
    t = (box - (c + R)) / wx
    return np.array([box, c + t * wy, c]), np.array([wx, wy, 0.0])


LUNE = {"kind": "luneburg", "radius": 20.0, "center": [32.0, 32.0, 32.0]}


def _luneburg_energy_drift(oracle_lib, b, stepper, h, L=20.0):
    """Inside a Luneburg lens, in the optical parameter dtau = ds / n, the ray
    equation (Eq. 14) becomes d^2 r / dtau^2 = -r (radius units): each axis
    is a harmonic oscillator and E_a = (n w_a)^2 + r_a^2 is conserved. A ray
    entering at the surface along +x at impact parameter b has
    E_x = 2 - b^2 and E_y = b^2. Returns the drift after arc length L."""
    R, c = 20.0, np.array([32.0, 32.0, 32.0])
    C0 = c + R * (1 - 1e-12) * np.array([-math.sqrt(1 - b * b), b, 0.0])
    n_steps = int(round(L / h))
    P = {"stepper": stepper, "adaptive": False, "h_fixed": h, "max_steps": 1000000}
    r = oracle_lib.march_ray(LUNE, BOX, C0, [1.0, 0, 0], P, path_cap=n_steps + 1)
    p = r["path"][n_steps]
    x = (p[:3] - c) / R
    n = math.sqrt(2 - x.dot(x))
    assert x.dot(x) < 1.0
    return max(abs((n * p[3]) ** 2 + x[0] ** 2 - (2 - b * b)),
               abs((n * p[4]) ** 2 + x[1] ** 2 - b * b))


@pytest.mark.parametrize("b", [0.3, 0.7])
def test_luneburg_oscillator_energies(oracle_lib, b):
    """Eq. 16 conserves the Luneburg oscillator energies to O(h), RK4 to
    O(h^4); an n misplaced in the update (w + ds n g) breaks both."""
    e = [_luneburg_energy_drift(oracle_lib, b, "euler", h) for h in (0.4, 0.2, 0.1)]
    assert e[0] > 1e-4
    assert 1.8 < e[0] / e[1] < 2.2 and 1.8 < e[1] / e[2] < 2.2
    r = [_luneburg_energy_drift(oracle_lib, b, "rk4", h) for h in (2.0, 1.0, 0.5)]
    assert r[0] > 1e-8
    assert 13.0 < r[0] / r[1] < 19.0 and 13.0 < r[1] / r[2] < 19.0


def _luneburg_exit(b, R=20.0, c=32.0, box=64.0):
    """Closed form: a ray entering a Luneburg lens parallel to +x at impact
    parameter b (units of the radius) leaves the sphere at the far focus
    c + (R, 0, 0) with direction (sqrt(1-b^2), -b, 0), then runs straight."""
    wx, wy = math.sqrt(1 - b * b), -b
    t = (box - (c + R)) / wx
    return np.array([box, c + t * wy, c]), np.array([wx, wy, 0.0])


@pytest.mark.parametrize("b", [0.2, 0.55, 0.8])
def test_luneburg_focus(oracle_lib, b):
    """Both steppers focus a ray entering from the box face onto the far
    focus of the lens. The gradient jumps at the lens surface, so the error
    is first order with an erratic phase: the tolerance is loose but a wrong
    ray equation misses by order one."""
    C0 = [0.0, 32.0 + 20.0 * b, 32.0]
    want_p, want_d = _luneburg_exit(b)
    for stepper in ("rk4", "euler"):
        P = {"stepper": stepper, "adaptive": False, "h_fixed": 0.0125, "max_steps": 100000}
        r = oracle_lib.march_ray(LUNE, BOX, C0, [1.0, 0, 0], P)
        assert r["flags"] == oracle_lib.FLAG_EXITED
        assert np.linalg.norm(r["exit_pos"] - want_p) < 2e-2
        assert np.linalg.norm(r["exit_dir"] - want_d) < 3e-4


def test_euler_update_structure(oracle_lib):
    """Eq. 16: every position increment is ds_k times the NEW direction
    w_{k+1}, and every direction is unit length."""
    field = {"kind": "luneburg", "radius": 20.0, "center": [32.0, 32.0, 32.0]}
    P = {"stepper": "euler", "adaptive": False, "h_fixed": 0.9, "max_steps": 1000}
    r = oracle_lib.march_ray(field, BOX, [0, 41.0, 30.0], _unit([1, 0, 0.1]), P, path_cap=1000)
    path = r["path"]
    np.testing.assert_allclose(np.linalg.norm(path[:, 3:6], axis=1), 1.0, atol=1e-14)
    inc = path[1:, :3] - path[:-1, :3]
    np.testing.assert_allclose(inc, path[:-1, 6:7] * path[1:, 3:6], atol=1e-12)
    # and not the old one (the field does bend the ray here)
    assert np.abs(inc - path[:-1, 6:7] * path[:-1, 3:6]).max() > 1e-4


def test_exit_clip_on_last_segment(oracle_lib):
    """The ray leaves along the last Eq. 16 segment: the exit point lies on a
    box face, on the segment from the last position along the new direction
    w_{k+1}, and the reported exit direction is w_{k+1} (the stratified field
    still bends the ray at the face)."""
    P = {"stepper": "euler", "adaptive": False, "h_fixed": 1.7, "max_steps": 1000}
    w0 = _unit([1.0, 0.2, 0.9])
    r = oracle_lib.march_ray(STRAT, BOX, [0.0, 10.0, 2.0], w0, P, path_cap=1000)
    last = r["path"][-1]
    seg = r["exit_pos"] - last[:3]
    t = np.linalg.norm(seg)
    assert 0 < t <= last[6]
    np.testing.assert_allclose(seg / t, r["exit_dir"], atol=1e-12)
    on_face = np.isclose(r["exit_pos"], 0.0, atol=1e-12) | np.isclose(r["exit_pos"], 64.0,
                                                                        atol=1e-12)
    assert on_face.any()
    # the last step did turn the ray, so w_k and w_{k+1} are distinguishable
    assert np.linalg.norm(r["exit_dir"] - last[3:6]) > 1e-4


def test_adaptive_step_bounds_turning_angle(oracle_lib):
    """Eq. 18 bounds the turning angle per step by theta_max; unclamped steps
    (|g_perp| >> eps) turn by atan(theta_max) ~ theta_max, with n ~ 1.1-1.4
    inside a Luneburg lens so a misplaced n would show."""
    field = {"kind": "luneburg", "radius": 20.0, "center": [32.0, 32.0, 32.0]}
    theta = 0.01
    P = {"stepper": "euler", "adaptive": True, "h_min": 1e-4, "h_max": 1.0,
         "theta_max": theta, "eps": 1e-12, "max_steps": 100000}
    r = oracle_lib.march_ray(field, BOX, [0, 40.0, 33.0], [1.0, 0, 0], P, path_cap=100000)
    path = r["path"]
    w = path[:, 3:6]
    ang = np.arctan2(np.linalg.norm(np.cross(w[:-1], w[1:]), axis=1),
                     np.einsum("ij,ij->i", w[:-1], w[1:]))
    assert ang.max() <= theta * (1 + 1e-12)
    ds = path[:-1, 6]
    unclamped = (ds > 1e-4) & (ds < 1.0)
    assert unclamped.sum() > 20
    np.testing.assert_allclose(ang[unclamped], math.atan(theta), rtol=1e-6)
    # outside the lens g = 0, so the step is the upper clamp
    outside = np.linalg.norm(path[:, :3] - 32.0, axis=1) > 20.5
    assert outside.sum() > 10 and np.all(path[outside, 6] == 1.0)


def test_adaptive_along_gradient_takes_max_step(oracle_lib):
    """A ray travelling along grad n has g_perp = 0 and is not bent: every
    adaptive step is the upper clamp."""
    P = {"stepper": "euler", "adaptive": True, "h_min": 0.01, "h_max": 1.5,
         "theta_max": 1e-3, "eps": 1e-9, "max_steps": 1000}
    r = oracle_lib.march_ray(STRAT, BOX, [10.0, 10.0, 0.0], [0, 0, 1.0], P, path_cap=1000)
    assert np.all(r["path"][:, 6] == 1.5)
    np.testing.assert_allclose(r["exit_pos"], [10, 10, 64], atol=1e-12)


def test_max_steps_stops_inside(oracle_lib):
    P = {"stepper": "euler", "adaptive": False, "h_fixed": 1.0, "max_steps": 3}
    r = oracle_lib.march_ray({"kind": "constant", "a": 0.0}, BOX, [0, 5, 5], [1.0, 0, 0], P)
    assert r["steps"] == 3 and r["flags"] == oracle_lib.FLAG_MAXSTEPS
    np.testing.assert_allclose(r["exit_pos"], [3, 5, 5], atol=1e-15)


def test_gridded_luneburg_converges_to_closed_form(oracle_lib):
    """The whole grid path (sampled dn, finite-difference gradient, trilinear
    fetch) converges to the analytic Luneburg exit as the grid is refined."""
    b = 0.45
    errs = []
    for scale in (1, 2):
        n = 64 * scale
        dims = (n, n, n)
        R, c = 20.0 * scale, n / 2.0
        dn = hi.sample_field_dn(
            lambda x, y, z: np.where((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 < R * R,
                                     np.sqrt(np.maximum(2 - ((x - c) ** 2 + (y - c) ** 2
                                                             + (z - c) ** 2) / (R * R), 1.0))
                                     - 1.0, 0.0), dims)
        vol = oracle_lib.index_field(dn.astype(np.float64), 1.0)
        P = {"stepper": "rk4", "adaptive": False, "h_fixed": 0.1 * scale, "max_steps": 100000}
        r = oracle_lib.march_ray({"kind": "grid", "vol4": vol}, [n, n, n], [0, c + R * b, c + 0.5],
                                 [1.0, 0, 0], P)
        want_p, want_d = _luneburg_exit(b, R=R, c=c, box=float(n))
        errs.append(np.linalg.norm(r["exit_dir"] - want_d))
    assert errs[1] < errs[0] and errs[1] < 0.02


# --------------------------------------------------------------------------- #
# Whole pixels
# --------------------------------------------------------------------------- #
def test_trace_identity_field_is_direct_lookup(oracle_lib):
    """dn = 0 everywhere: every pixel shows the background at its primary ray
    direction, hits exit at the slab exit point, misses report the eye."""
    dims = (16, 12, 10)
    vol = np.zeros((10, 12, 16, 4))
    cam = hi.orbit_camera(dims, 20.0, 10.0, 24, 18)
    bg = hi.checker_background(64, 32)
    P = hi.params_euler_adaptive(dims, theta_max=3e-3)
    out = oracle_lib.trace_grid(vol, cam, P, bg, nthreads=4)
    box = np.array(dims, dtype=np.float64)
    for pix in range(24 * 18):
        d = oracle_lib.camera_ray(cam, pix % 24, pix // 24)
        np.testing.assert_allclose(out["rgb"][pix], oracle_lib.background(bg, d), atol=1e-14)
        np.testing.assert_allclose(out["exit_dir"][pix], d, atol=1e-14)
        hit, tin, tout = oracle_lib.slab(cam["eye"], d, box)
        if hit:
            assert out["flags"][pix] == oracle_lib.FLAG_HIT | oracle_lib.FLAG_EXITED
            np.testing.assert_allclose(out["exit_pos"][pix], np.array(cam["eye"]) + tout * d,
                                       atol=1e-9)
        else:
            assert out["flags"][pix] == 0 and out["steps"][pix] == 0
            np.testing.assert_allclose(out["exit_pos"][pix], cam["eye"], atol=0)
    assert (out["flags"] != 0).sum() > 50 and (out["flags"] == 0).sum() > 50


def test_trace_pixel_subset_and_threads_agree(oracle_lib):
    dims = (32, 32, 32)
    vol = oracle_lib.index_field(hi.plume_dn_grid(dims=dims).astype(np.float64), 1.0)
    cam = hi.orbit_camera(dims, 0.0, 0.0, 20, 16)
    bg = hi.checker_background()
    P = hi.params_rk4_fixed(dims)
    full = oracle_lib.trace_grid(vol, cam, P, bg, nthreads=1)
    sub = np.array([5, 170, 171, 319, 0, 160])
    part = oracle_lib.trace_grid(vol, cam, P, bg, pixels=sub, nthreads=3)
    for k in ("rgb", "exit_pos", "exit_dir", "steps", "flags"):
        np.testing.assert_array_equal(part[k], full[k][sub])


def test_march_rays_equals_single_rays(oracle_lib):
    """The batched march is the single-ray march, ray by ray."""
    r = np.random.default_rng(4)
    C0 = np.c_[np.zeros(7), r.uniform(10, 54, size=(7, 2))]
    w0 = np.c_[np.ones(7), r.uniform(-0.3, 0.3, size=(7, 2))]
    w0 /= np.linalg.norm(w0, axis=1, keepdims=True)
    P = {"stepper": "rk4", "adaptive": True, "h_min": 0.05, "h_max": 1.0, "theta_max": 1e-3,
         "eps": 1e-6, "max_steps": 100000}
    many = oracle_lib.march_rays(LUNE, BOX, C0, w0, P, nthreads=3)
    for i in range(7):
        one = oracle_lib.march_ray(LUNE, BOX, C0[i], w0[i], P)
        np.testing.assert_array_equal(many["exit_pos"][i], one["exit_pos"])
        np.testing.assert_array_equal(many["exit_dir"][i], one["exit_dir"])
        assert many["steps"][i] == one["steps"] and many["flags"][i] == one["flags"]


# --------------------------------------------------------------------------- #
# Scene planes (the analytic scene geometry behind the volume)
# --------------------------------------------------------------------------- #
def _ramp_texture(W=64, H=32):
    t = np.zeros((H, W, 3), dtype=np.uint8)
    t[..., 0] = np.arange(W)[None, :] * 4
    t[..., 1] = np.arange(H)[:, None] * 8
    t[..., 2] = 200
    return t


def test_plane_hit_texture_coordinates(oracle_lib):
    """A ramp texture returns its bilinear texel coordinates: the hit point
    (solved here as a 3x3 linear system P + t d = o + a u + b v) maps to
    (a W - 1/2, b H - 1/2), clamped to the texel centres."""
    W, H = 64, 32
    tex = _ramp_texture(W, H)
    plane = {"origin": [10.0, -20.0, 5.0], "u": [0.0, 40.0, 0.0], "v": [0.0, 0.0, 20.0],
             "tex": tex}
    env = np.full((8, 16, 3), 9, dtype=np.uint8)
    r = np.random.default_rng(2)
    for _ in range(40):
        P = r.uniform(-50, 0, size=3)
        X = np.array(plane["origin"]) + r.uniform(0.02, 0.98) * np.array(plane["u"]) \
            + r.uniform(0.02, 0.98) * np.array(plane["v"])
        d = (X - P) / np.linalg.norm(X - P)
        A = np.column_stack([d, -np.array(plane["u"]), -np.array(plane["v"])])
        t, a, b = np.linalg.solve(A, np.array(plane["origin"]) - P)
        c = oracle_lib.scene_color(env, P, d, [plane]) * 255
        s = min(max(a * W - 0.5, 0), W - 1)
        q = min(max(b * H - 0.5, 0), H - 1)
        assert c[0] == pytest.approx(4 * s, abs=1e-9) and c[1] == pytest.approx(8 * q, abs=1e-9)
        assert c[2] == pytest.approx(200, abs=1e-9)


def test_plane_nearest_front_and_misses(oracle_lib):
    env = np.full((8, 16, 3), 9, dtype=np.uint8)
    red = np.zeros((4, 4, 3), np.uint8)
    red[..., 0] = 255
    green = np.zeros((4, 4, 3), np.uint8)
    green[..., 1] = 255
    near = {"origin": [10.0, -5.0, -5.0], "u": [0.0, 10.0, 0.0], "v": [0.0, 0.0, 10.0],
            "tex": red}
    far = {"origin": [20.0, -5.0, -5.0], "u": [0.0, 10.0, 0.0], "v": [0.0, 0.0, 10.0],
           "tex": green}
    sc = oracle_lib.scene_color
    np.testing.assert_allclose(sc(env, [0, 0, 0], [1, 0, 0], [far, near]), [1, 0, 0])
    np.testing.assert_allclose(sc(env, [15, 0, 0], [1, 0, 0], [far, near]), [0, 1, 0])
    np.testing.assert_allclose(sc(env, [0, 0, 0], [-1, 0, 0], [far, near]), 9 / 255)  # behind
    np.testing.assert_allclose(sc(env, [0, 0, 0], [0, 1, 0], [far, near]), 9 / 255)  # parallel
    np.testing.assert_allclose(sc(env, [0, 6, 0], [1, 0, 0], [far, near]), 9 / 255)  # beside


def _slab_variance(oracle_lib, Lz, seeds=range(8), n_side=32):
    """Mean squared exit deflection of parallel rays crossing a slab of
    homogeneous turbulence (FFT-filtered noise, correlation 2 voxels) of
    thickness Lz along +z."""
    dims = (64, 64, Lz)
    defl = []
    for s in seeds:
        dn = hi.homogeneous_turbulence_dn(dims, seed=100 + s, sigma=2.0)
        vol = oracle_lib.index_field(dn.astype(np.float64), 1.0)
        xs = np.linspace(1.0, 63.0, n_side)
        X, Y = np.meshgrid(xs, xs)
        C0 = np.c_[X.ravel(), Y.ravel(), np.zeros(X.size)]
        w0 = np.tile([0.0, 0.0, 1.0], (X.size, 1))
        P = {"stepper": "rk4", "adaptive": False, "h_fixed": 0.5, "max_steps": 10 * Lz}
        out = oracle_lib.march_rays({"kind": "grid", "vol4": vol}, dims, C0, w0, P, nthreads=8)
        assert np.all(out["flags"] == oracle_lib.FLAG_EXITED)
        defl.append(out["exit_dir"][:, :2])
    d = np.concatenate(defl)
    return float(np.mean(np.sum(d * d, axis=1)))


def test_angle_of_arrival_variance_grows_linearly_with_path(oracle_lib):
    """Eq. 19: under constant turbulence strength the angle-of-arrival
    variance grows linearly with the path length L (<alpha^2> = 3/8 K_n^2 L).
    The marched deflection of parallel rays through homogeneous turbulence
    doubles when the slab thickness doubles."""
    v = [_slab_variance(oracle_lib, L) for L in (24, 48, 96)]
    assert v[0] > 0
    assert 1.75 < v[1] / v[0] < 2.3 and 1.75 < v[2] / v[1] < 2.3, v
