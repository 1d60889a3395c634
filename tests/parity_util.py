"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same inputs, and compare them.

Tolerances (FP32 march against the FP64 oracle on the same volume and the
same step schedule): exit position <= 1e-3 voxel, exit direction <= 1e-6 rad
(angle = atan2(|a x b|, a.b) in FP64), float-image RMSE <= 1e-4.

Conditioning. Where the Eq. 18 step varies on the scale of itself (noisy
plume cores), the discrete march amplifies tiny changes of the start state:
the oracle's own exit direction moves by up to ~2e-5 rad when its start point
moves by 1e-6 voxel. No FP32 implementation can be held to 1e-6 rad on such
rays, because rounding the inputs to FP32 already moves the FP64 answer by
more than that. So every ray must meet the tolerance, except rays whose
oracle answer itself moves by more than half the tolerance when the start
state is perturbed at FP32 rounding scale (one ulp of the entry point, 2^-23
rad of direction) or whose step count changes under that perturbation. Those
ill-conditioned rays are counted against a per-test cap (close to the rate
measured on that workload), and their GPU result must lie within five times
the oracle's own perturbation spread (plus the tolerance). Only a ray whose
GPU step count differs from the oracle's by exactly one (its last step lands
within rounding of a box face) gets one more allowance: the turn of the step
that one side took and the other did not, read off the oracle's own path
(the turn of its last step, or of one more step from its exit point along its
exit direction), never a bound from theta_max. The image RMSE bound applies
to every compared ray, excused ones included.

With HH_PARITY_LOG set to a file name, every check appends one JSON line of
its statistics (hits, rays beyond tolerance, ill-conditioned rays, the worst
excess over the tolerance) to that file.
"""
from __future__ import annotations

import numpy as np

POS_TOL = 1e-3
DIR_TOL = 1e-6
RMSE_TOL = 1e-4


def f32(x):
    """Rounds a scalar, list or dict of them to FP32 values (as Python floats),
    so that the oracle sees exactly the numbers the device sees."""
    if isinstance(x, dict):
        return {k: f32(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [f32(v) for v in x]
    if isinstance(x, float):
        return float(np.float32(x))
    return x


def gpu_trace(hh, torch, vol, cams, params, bg_t, want_all=True):
    """Traces cams through vol on the GPU; returns a list of numpy dicts.
    bg_t: the environment map tensor, or (map, planes)."""
    dev = (bg_t[0] if isinstance(bg_t, tuple) else bg_t).device
    outs = []
    for c in cams:
        n = c["width"] * c["height"]
        o = {"rgb": torch.empty(n * 3, device=dev)}
        if want_all:
            o.update({"exit_pos": torch.empty(n * 3, device=dev),
                      "exit_dir": torch.empty(n * 3, device=dev),
                      "steps": torch.empty(n, dtype=torch.int32, device=dev),
                      "flags": torch.empty(n, dtype=torch.int32, device=dev)})
        outs.append(o)
    hh.hh_trace(vol, cams, params, bg_t, outs)
    torch.cuda.synchronize()
    res = []
    for o in outs:
        r = {"rgb": o["rgb"].cpu().numpy().reshape(-1, 3).astype(np.float64)}
        if want_all:
            r["exit_pos"] = o["exit_pos"].cpu().numpy().reshape(-1, 3).astype(np.float64)
            r["exit_dir"] = o["exit_dir"].cpu().numpy().reshape(-1, 3).astype(np.float64)
            r["steps"] = o["steps"].cpu().numpy()
            r["flags"] = o["flags"].cpu().numpy().view(np.uint32)
        res.append(r)
    return res


def export_volume(hh, torch, vol, dims):
    """The volume exactly as the march reads it, widened to FP64 (nz,ny,nx,4)."""
    nx, ny, nz = dims
    t = torch.empty(nx * ny * nz * 4, device="cuda")
    hh.hh_volume_export(vol, t)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64).reshape(nz, ny, nx, 4)


def angle(a, b):
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.einsum("...i,...i->...", a, b))


def exit_face(p, box):
    """Face of the box [0, box] that each exit point lies on: 0/1/2 for the
    x/y/z = 0 faces, 3/4/5 for x/y/z = box (the nearest face)."""
    p = np.asarray(p, dtype=np.float64)
    d = np.concatenate([np.abs(p), np.abs(np.asarray(box, dtype=np.float64) - p)], axis=1)
    return np.argmin(d, axis=1)


def compare(gpu: dict, ref: dict, sel=None, box=None) -> dict:
    """Statistics of the GPU result against the oracle (optionally on the
    pixel subset `sel` of the GPU arrays, matching ref's order). With box,
    also the number of rays that leave through different faces."""
    g = {k: (v if sel is None else v[sel]) for k, v in gpu.items()}
    st = {"rmse": float(np.sqrt(np.mean((g["rgb"] - ref["rgb"]) ** 2))),
          "rgb_max": float(np.abs(g["rgb"] - ref["rgb"]).max())}
    if "exit_dir" in g:
        hit_g = (g["flags"] & 1) != 0
        hit_r = (ref["flags"] & 1) != 0
        same_hit = hit_g == hit_r
        same_steps = (g["steps"] == ref["steps"]) & same_hit
        ang = angle(g["exit_dir"], ref["exit_dir"])
        pos = np.abs(g["exit_pos"] - ref["exit_pos"]).max(axis=1)
        st.update({
            "n": int(len(ang)),
            "hits": int(hit_r.sum()),
            "hit_mismatch": int((~same_hit).sum()),
            "step_mismatch": int((~same_steps).sum()),
            "dir_max": float(ang.max()) if len(ang) else 0.0,
            "dir_max_same_steps": float(ang[same_steps].max()) if same_steps.any() else 0.0,
            "pos_max_same_steps": float(pos[same_steps].max()) if same_steps.any() else 0.0,
            "pos_max": float(pos[same_hit].max()) if same_hit.any() else 0.0,
            "flags_equal_same_steps": bool(np.all(g["flags"][same_steps]
                                                  == ref["flags"][same_steps])),
            "mean_steps": float(ref["steps"][hit_r].mean()) if hit_r.any() else 0.0,
        })
        if box is not None:
            # a ray that leaves within rounding of an edge may be put on either
            # face: counted, with the largest position difference among them
            both = ((g["flags"] & 2) != 0) & ((ref["flags"] & 2) != 0)
            other = np.zeros_like(both)
            other[both] = (exit_face(g["exit_pos"][both], box)
                           != exit_face(ref["exit_pos"][both], box))
            st["face_mismatch"] = int(other.sum())
            st["face_mismatch_pos_max"] = float(pos[other].max()) if other.any() else 0.0
    return st


def start_states(oracle, cam, box, pix):
    """FP64 entry point and primary direction of each pixel (hits only)."""
    eye = np.asarray(cam["eye"], dtype=np.float64)
    C0 = np.zeros((len(pix), 3))
    w0 = np.zeros((len(pix), 3))
    for i, p in enumerate(pix):
        d = oracle.camera_ray(cam, int(p) % cam["width"], int(p) // cam["width"])
        hit, tin, _ = oracle.slab(eye, d, box)
        assert hit
        C0[i] = eye + max(tin, 0.0) * d
        w0[i] = d
    return C0, w0


def perturbation_spread(oracle, field, box, C0, w0, params, n_pert=6, seed=0, nthreads=8):
    """Largest change of the oracle's exit direction / position, and whether
    its step count changed, when the start state moves at FP32 rounding scale."""
    r = np.random.default_rng(seed)
    base = oracle.march_rays(field, box, C0, w0, params, nthreads=nthreads)
    pos_eps = 2.0**-23 * max(float(np.abs(C0).max()), float(max(box)))
    dir_eps = 2.0**-23
    s_dir = np.zeros(len(C0))
    s_pos = np.zeros(len(C0))
    s_steps = np.zeros(len(C0), dtype=bool)
    for _ in range(n_pert):
        dc = r.normal(size=C0.shape)
        dc *= pos_eps / np.linalg.norm(dc, axis=1, keepdims=True)
        dw = r.normal(size=w0.shape)
        dw -= np.einsum("ij,ij->i", dw, w0)[:, None] * w0
        dw *= dir_eps / np.linalg.norm(dw, axis=1, keepdims=True)
        w = w0 + dw
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        q = oracle.march_rays(field, box, C0 + dc, w, params, nthreads=nthreads)
        s_dir = np.maximum(s_dir, angle(q["exit_dir"], base["exit_dir"]))
        s_pos = np.maximum(s_pos, np.abs(q["exit_pos"] - base["exit_pos"]).max(axis=1))
        s_steps |= q["steps"] != base["steps"]
    return s_dir, s_pos, s_steps


def path_spread(oracle, field, box, C0, w0, params, nthreads=8):
    """Accumulated sensitivity to rounding at every step. An FP32 march rounds
    at each of its K steps, not only at the start: its sample position is the
    position rounded to FP32, each coordinate on its own by up to half an ulp
    of the box extent (2^-24 of it), while the direction (carried as a small
    deflection of the primary direction) and the compensated position carry
    far smaller errors. The oracle's march depends only on the current state
    (C_k, w_k), so restarting it from each recorded state with the position
    moved by that half ulp along x, along y and along z gives the exit's
    response to each coordinate's rounding at step k; their sum s_k is the
    first-order change for the worst signs of the three roundings, and
    independent steps add as sqrt(sum_k s_k^2). Returns that for the exit
    direction and position, and whether some restart changed the step count."""
    pos_eps = 2.0**-24 * float(max(box))
    out_dir = np.zeros(len(C0))
    out_pos = np.zeros(len(C0))
    out_steps = np.zeros(len(C0), dtype=bool)
    axes = pos_eps * np.eye(3)
    for i in range(len(C0)):
        m = oracle.march_ray(field, box, C0[i], w0[i], params, path_cap=int(params["max_steps"]))
        path = m["path"]
        K = len(path)
        if K == 0:
            continue
        Ck = (path[:, None, 0:3] + axes[None]).reshape(-1, 3)
        wk = np.repeat(path[:, 3:6], 3, axis=0)
        q = oracle.march_rays(field, box, Ck, wk, params, nthreads=nthreads)
        sd = angle(q["exit_dir"], m["exit_dir"]).reshape(K, 3).sum(axis=1)
        sp = np.abs(q["exit_pos"] - m["exit_pos"]).max(axis=1).reshape(K, 3).sum(axis=1)
        remaining = m["steps"] - np.arange(K)
        out_dir[i] = np.sqrt(np.sum(sd**2))
        out_pos[i] = np.sqrt(np.sum(sp**2))
        out_steps[i] = bool(np.any(q["steps"].reshape(K, 3) != remaining[:, None]))
    return out_dir, out_pos, out_steps


def ill_conditioned(oracle, field, box, cam, params, pix, n_pert=6, seed=0):
    """Which of the pixels pix (rays that hit) the oracle alone finds ill
    conditioned: its exit direction or position moves by more than half a
    tolerance, or its step count changes, under start-state perturbations at
    FP32 rounding scale. Also returns the spreads."""
    C0, w0 = start_states(oracle, cam, box, pix)
    s_dir, s_pos, s_steps = perturbation_spread(oracle, field, box, C0, w0, params,
                                                n_pert=n_pert, seed=seed)
    ill = (s_dir > DIR_TOL / 2) | (s_pos > POS_TOL / 2) | s_steps
    return ill, s_dir, s_pos, s_steps


def step_turns(oracle, field, box, C0, w0, params):
    """For each ray from (C0, w0): the turn of the oracle's last step (the
    angle between the direction before and after it) and the turn of one more
    step from its exit point along its exit direction. They bound the
    difference a step count one higher or one lower makes: the step that one
    side took and the other did not, at the same place to within rounding."""
    last = np.zeros(len(C0))
    nxt = np.zeros(len(C0))
    one = dict(params, max_steps=1)
    for i in range(len(C0)):
        m = oracle.march_ray(field, box, C0[i], w0[i], params, path_cap=int(params["max_steps"]))
        if m["steps"] > 0:
            last[i] = float(angle(m["path"][-1, 3:6], m["exit_dir"]))
        q = oracle.march_ray(field, box, m["exit_pos"], m["exit_dir"], one)
        nxt[i] = float(angle(m["exit_dir"], q["exit_dir"]))
    return last, nxt


def _log(st: dict, label):
    import json
    import os

    path = os.environ.get("HH_PARITY_LOG")
    if not path:
        return
    rec = {"test": label or os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]}
    rec.update({k: v for k, v in st.items() if isinstance(v, (int, float, bool, str))})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def assert_parity_conditioned(gpu: dict, ref: dict, oracle, field, box, cam, params, sel=None,
                              max_ill_frac: float = 0.005, label=None) -> dict:
    """Parity with the conditioning rule above. gpu holds the whole view (or
    `sel` picks the pixels that ref holds, in ref's order). At most
    max_ill_frac of the hit rays (plus two) may be excused as ill conditioned.
    Returns the statistics (also appended to HH_PARITY_LOG when set)."""
    st = compare(gpu, ref, sel, box=box)
    g = {k: (v if sel is None else v[sel]) for k, v in gpu.items()}
    pix = np.arange(len(g["steps"])) if sel is None else np.asarray(sel)
    hit_g = (g["flags"] & 1) != 0
    hit_r = (ref["flags"] & 1) != 0
    assert st["hit_mismatch"] == 0, st
    ang = angle(g["exit_dir"], ref["exit_dir"])
    pos = np.abs(g["exit_pos"] - ref["exit_pos"]).max(axis=1)
    bad = (ang > DIR_TOL) | (pos > POS_TOL) | (g["flags"] != ref["flags"])
    assert not np.any(bad & ~hit_r), "a ray that misses the volume differs"
    idx = np.flatnonzero(bad)
    st["n_bad"] = int(len(idx))
    st["n_ill"] = 0
    st["n_turn"] = 0
    # worst excess over the plain tolerance, as a multiple of it
    st["worst_dir_over_tol"] = float(ang.max() / DIR_TOL) if len(ang) else 0.0
    st["worst_pos_over_tol"] = float(pos[hit_r].max() / POS_TOL) if hit_r.any() else 0.0
    if len(idx):
        ill, s_dir, s_pos, s_steps = ill_conditioned(oracle, field, box, cam, params, pix[idx])
        if not np.all(ill):
            # the spread is a maximum over random perturbations: rays that six
            # of them leave below the threshold get 64 more
            j = np.flatnonzero(~ill)
            ill2, d2, p2, st2 = ill_conditioned(oracle, field, box, cam, params, pix[idx][j],
                                                n_pert=64, seed=1)
            ill[j] = ill2
            s_dir[j] = np.maximum(s_dir[j], d2)
            s_pos[j] = np.maximum(s_pos[j], p2)
            s_steps[j] |= st2
        st["n_ill"] = int(ill.sum())
        show = np.concatenate([np.flatnonzero(~ill), np.arange(len(idx))])[:5]
        worst = {"pixels": pix[idx][show].tolist(), "dir": ang[idx][show].tolist(),
                 "pos": pos[idx][show].tolist(), "spread_dir": s_dir[show].tolist(),
                 "spread_pos": s_pos[show].tolist(), "steps_changed": s_steps[show].tolist(),
                 "ill": ill[show].tolist()}
        assert np.all(ill), dict(st, **worst)
        # the one-step allowance: only where the step counts differ by one
        dk = g["steps"][idx].astype(np.int64) - ref["steps"][idx].astype(np.int64)
        turn = np.zeros(len(idx))
        k1 = np.flatnonzero(np.abs(dk) == 1)
        if len(k1):
            C0, w0 = start_states(oracle, cam, box, pix[idx][k1])
            last, nxt = step_turns(oracle, field, box, C0, w0, params)
            turn[k1] = np.where(dk[k1] < 0, last, nxt)
        st["n_turn"] = int(len(k1))

        def over_of():
            return (ang[idx] > DIR_TOL + 5 * s_dir + turn) | (pos[idx] > POS_TOL + 5 * s_pos)

        over = over_of()
        if over.any():
            # beyond what one rounding at the start explains: measure the
            # rounding made at every step along the ray (path_spread)
            j = np.flatnonzero(over)
            C0, w0 = start_states(oracle, cam, box, pix[idx][j])
            p_dir, p_pos, _ = path_spread(oracle, field, box, C0, w0, params)
            s_dir[j] = np.maximum(s_dir[j], p_dir)
            s_pos[j] = np.maximum(s_pos[j], p_pos)
            over = over_of()
            st["n_path"] = int(len(j))
            # how close the rays measured along their path come to that bound
            st["worst_path_over_bound"] = float(max(
                (ang[idx][j] / (DIR_TOL + 5 * s_dir[j] + turn[j])).max(),
                (pos[idx][j] / (POS_TOL + 5 * s_pos[j])).max()))
        excess = ang[idx] / (DIR_TOL + 5 * s_dir + turn)
        st["worst_over_bound"] = float(excess.max())
        if over.any():
            k = np.flatnonzero(over)[:5]
            worst = {"over": int(over.sum()), "pixels": pix[idx][k].tolist(),
                     "dir": ang[idx][k].tolist(), "pos": pos[idx][k].tolist(),
                     "spread_dir": s_dir[k].tolist(), "spread_pos": s_pos[k].tolist(),
                     "steps_changed": s_steps[k].tolist(), "turn": turn[k].tolist(),
                     "gpu_steps": g["steps"][idx][k].tolist(),
                     "oracle_steps": ref["steps"][idx][k].tolist(),
                     "gpu_exit": g["exit_pos"][idx][k].tolist(),
                     "oracle_exit": ref["exit_pos"][idx][k].tolist()}
        assert not over.any(), dict(st, **worst)
    st["max_ill"] = int(max_ill_frac * max(int(hit_r.sum()), 1)) + 2
    _log(st, label)
    assert st["n_ill"] <= st["max_ill"], st
    # image RMSE over every compared ray, excused ones included
    assert st["rmse"] <= RMSE_TOL, st
    assert np.array_equal(hit_g, hit_r)
    return st


def assert_parity_plain(gpu: dict, ref: dict, box, sel=None, label=None) -> dict:
    """Parity with no excusal at all: every ray within the exit position and
    direction tolerances with the oracle's flags, and the image RMSE bound.
    For schedules on which the march is well conditioned everywhere (fixed
    steps; Eq. 18 when it keeps every step at h_max)."""
    st = compare(gpu, ref, sel, box=box)
    g = {k: (v if sel is None else v[sel]) for k, v in gpu.items()}
    ang = angle(g["exit_dir"], ref["exit_dir"])
    pos = np.abs(g["exit_pos"] - ref["exit_pos"]).max(axis=1)
    bad = (ang > DIR_TOL) | (pos > POS_TOL) | (g["flags"] != ref["flags"])
    hit_r = (ref["flags"] & 1) != 0
    st.update({"n_bad": int(bad.sum()), "n_ill": 0, "n_turn": 0, "max_ill": 0,
               "worst_dir_over_tol": float(ang.max() / DIR_TOL) if len(ang) else 0.0,
               "worst_pos_over_tol": float(pos[hit_r].max() / POS_TOL) if hit_r.any() else 0.0,
               "rule": "plain"})
    _log(st, label)
    assert st["hit_mismatch"] == 0, st
    assert st["n_bad"] == 0, dict(st, pixels=np.flatnonzero(bad)[:5].tolist())
    assert st["rmse"] <= RMSE_TOL, st
    return st
