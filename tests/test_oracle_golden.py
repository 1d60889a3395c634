"""The oracle still reproduces its committed golden sample and the paper's
printed parameters are the ones the input presets use."""
import json
import os

import numpy as np

import hh_inputs as hi

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_golden_sample(oracle_lib):
    with open(os.path.join(GOLDEN, "oracle_plume64_sample.json")) as f:
        g = json.load(f)
    dims = (64, 64, 64)
    vol = oracle_lib.index_field(hi.plume_dn_grid(64).astype(np.float64), 1.0)
    cam = hi.orbit_camera(dims, 0.0, 0.0, 128, 128)
    out = oracle_lib.trace_grid(vol, cam, hi.params_rk4_fixed(dims, 0.5),
                                hi.checker_background(), pixels=np.array(g["pixels"]),
                                nthreads=2)
    np.testing.assert_allclose(out["rgb"], g["rgb"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["exit_pos"], g["exit_pos"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["exit_dir"], g["exit_dir"], rtol=0, atol=1e-12)
    assert out["steps"].tolist() == g["steps"] and out["flags"].tolist() == g["flags"]
    assert sum(1 for f in g["flags"] if f & 1) >= 6  # the sample does cross the plume


def test_paper_parameters_used_by_presets():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        p = json.load(f)
    assert hi.THETA_PAPER == p["theta_max"]["value"]
