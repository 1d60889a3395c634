"""The parity rule itself (tests/parity_util.py), on the CPU: it accepts the
oracle's own answer rounded to FP32, rejects mistakes planted on well- and on
ill-conditioned rays, and its rounding model vanishes where the march has
nothing to amplify."""
import numpy as np
import pytest

import hh_inputs as hi
from parity_util import (DIR_TOL, angle, assert_parity_conditioned, f32, ill_conditioned,
                         step_turns,
                         path_spread, perturbation_spread, start_states)

D = (64, 64, 64)


@pytest.fixture(scope="module")
def plume(oracle_lib):
    parts = hi.plume_particles(16384, 64)
    rho = oracle_lib.splat(parts, D, 2.0)
    vol4 = oracle_lib.index_field(rho.astype(np.float32).astype(np.float64),
                                  float(np.float32(hi.K_GD)))
    cam = f32(hi.orbit_camera(D, 0.0, 0.0, 128, 128))
    params = f32(hi.params_euler_adaptive(D, theta_max=hi.THETA_CALIBRATED))
    ref = oracle_lib.trace_grid(vol4, cam, params, hi.checker_background(), nthreads=8)
    return {"kind": "grid", "vol4": vol4}, cam, params, ref


def _as_fp32(ref):
    return {k: (v.astype(np.float32).astype(np.float64) if v.dtype == np.float64 else v.copy())
            for k, v in ref.items()}


def _turned(v, a, seed):
    """v turned by the angle a about a seeded axis perpendicular to it."""
    p = np.random.default_rng(seed).normal(size=3)
    p -= np.dot(p, v) * v
    p /= np.linalg.norm(p)
    return np.cos(a) * v + np.sin(a) * p


def test_accepts_the_oracle_rounded_to_fp32(oracle_lib, plume):
    field, cam, params, ref = plume
    st = assert_parity_conditioned(_as_fp32(ref), ref, oracle_lib, field, D, cam, params)
    assert st["hits"] > 2000 and st["n_bad"] == 0


def test_rejects_a_turned_well_conditioned_ray(oracle_lib, plume):
    field, cam, params, ref = plume
    hit = np.flatnonzero((ref["flags"] & 1) != 0)
    C0, w0 = start_states(oracle_lib, cam, D, hit[:200])
    s_dir, _, s_steps = perturbation_spread(oracle_lib, field, D, C0, w0, params)
    # the direction perturbation alone moves the exit by 2^-23 rad
    k = hit[:200][np.flatnonzero((s_dir < DIR_TOL / 4) & ~s_steps)[0]]
    got = _as_fp32(ref)
    got["exit_dir"][k] = _turned(ref["exit_dir"][k], 3 * DIR_TOL, seed=1)
    assert angle(got["exit_dir"][k], ref["exit_dir"][k]) > 2 * DIR_TOL
    with pytest.raises(AssertionError):
        assert_parity_conditioned(got, ref, oracle_lib, field, D, cam, params)


def test_rejects_an_ill_conditioned_ray_turned_far_beyond_its_spread(oracle_lib, plume):
    field, cam, params, ref = plume
    hit = np.flatnonzero((ref["flags"] & 1) != 0)
    ill, s_dir, _, _ = ill_conditioned(oracle_lib, field, D, cam, params, hit)
    if not ill.any():
        pytest.skip("no ill-conditioned ray in this view")
    i = int(np.argmax(s_dir))
    C0, w0 = start_states(oracle_lib, cam, D, hit[i:i + 1])
    p_dir, _, _ = path_spread(oracle_lib, field, D, C0, w0, params)
    far = 100 * max(s_dir[i], p_dir[0]) + 1e-4  # beyond any one-step turn as well
    got = _as_fp32(ref)
    got["exit_dir"][hit[i]] = _turned(ref["exit_dir"][hit[i]], far, seed=2)
    with pytest.raises(AssertionError):
        assert_parity_conditioned(got, ref, oracle_lib, field, D, cam, params)


def test_path_spread_vanishes_in_a_constant_field(oracle_lib, plume):
    """With dn constant and g = 0 nothing bends the ray: the direction is
    insensitive to rounding at every step, and the exit point moves only by
    the position errors themselves. A start moved by e slides the straight
    ray's exit point on its exit face (normal n) by e - (e.n / w.n) w, so half
    an ulp along each axis gives a known response, the same at every step of
    the straight path: the model must return sqrt(K) times its sum."""
    _, cam, params, ref = plume
    vol4 = np.zeros(D[::-1] + (4,))
    vol4[..., 0] = 1e-4
    const = {"kind": "grid", "vol4": vol4}
    # rays across the middle of the view, which leave through one face, away
    # from its edges (where the exit face is ambiguous)
    W = cam["width"]
    hit = [p for p in np.flatnonzero((ref["flags"] & 1) != 0)
           if abs(p % W - W // 2) < 16 and abs(p // W - W // 2) < 16][::37][:8]
    C0, w0 = start_states(oracle_lib, cam, D, hit)
    p_dir, p_pos, p_steps = path_spread(oracle_lib, const, D, C0, w0, params)
    assert np.all(p_dir == 0.0)
    eps = 2.0**-24 * max(D)
    box = np.asarray(D, dtype=np.float64)
    for i in range(len(hit)):
        m = oracle_lib.march_ray(const, D, C0[i], w0[i], params)
        x, w = m["exit_pos"], m["exit_dir"]
        dist = np.minimum(np.abs(x), np.abs(box - x))
        a = int(np.argmin(dist))
        assert np.sort(dist)[1] > 1.0 and m["steps"] > 10
        s = sum(np.abs(eps * e - (eps * e[a] / w[a]) * w).max() for e in np.eye(3))
        assert p_pos[i] == pytest.approx(np.sqrt(m["steps"]) * s, rel=1e-3)


def test_one_step_allowance_is_the_rays_own_step_not_theta(oracle_lib, plume):
    """A ray whose GPU step count differs from the oracle's by one gets the
    turn of the step one side took and the other did not, read off the
    oracle's own path. Near the box faces, where such rays end, that turn is
    tiny: a plant of theta_max / 10 on such a ray (which a theta_max
    allowance would excuse) is rejected, while the ray with the step added
    and its direction within its spreads is accepted."""
    field, cam, params, ref = plume
    hit = np.flatnonzero((ref["flags"] & 1) != 0)
    ill, s_dir, _, s_steps = ill_conditioned(oracle_lib, field, D, cam, params, hit)
    cand = np.flatnonzero(s_steps)
    if not len(cand):
        pytest.skip("no ray in this view changes its step count under perturbation")
    i = int(cand[0])
    k = hit[i]
    C0, w0 = start_states(oracle_lib, cam, D, hit[i:i + 1])
    last, nxt = step_turns(oracle_lib, field, D, C0, w0, params)
    assert nxt[0] < params["theta_max"] / 100  # the field is ~0 at the faces
    got = _as_fp32(ref)
    got["steps"][k] += 1
    # within tolerance: the extra step alone is not a failure
    assert_parity_conditioned(got, ref, oracle_lib, field, D, cam, params)
    got["exit_dir"][k] = _turned(ref["exit_dir"][k], params["theta_max"] / 10, seed=3)
    with pytest.raises(AssertionError):
        assert_parity_conditioned(got, ref, oracle_lib, field, D, cam, params)


def test_rmse_counts_excused_rays(oracle_lib, plume):
    """The image RMSE bound holds over every compared ray: a colour error
    planted on one ray of the view, large enough to lift the RMSE of the
    whole view past 1e-4, is rejected although the ray's exit matches."""
    field, cam, params, ref = plume
    hit = np.flatnonzero((ref["flags"] & 1) != 0)
    got = _as_fp32(ref)
    n = got["rgb"].size
    got["rgb"][hit[0]] += 2e-4 * np.sqrt(n / 3.0)
    with pytest.raises(AssertionError):
        assert_parity_conditioned(got, ref, oracle_lib, field, D, cam, params)
