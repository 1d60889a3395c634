"""Writes tests/golden/oracle_plume64_sample.json from the FP64 oracle alone.

The tiny plume scene (64^3 given dn grid, one 128x128 camera 1.5 grid widths
away, 60 degree vertical FOV, fixed-step RK4 h = 0.5, seeded checker
background) is traced by the oracle on a fixed set of pixels; the stored
values guard the oracle against accidental change. Run from the repo root:
    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hh_inputs as hi  # noqa: E402
import oracle  # noqa: E402

PIXELS = [0, 127, 4095, 5000, 6000, 7000, 8191, 8192, 8256, 8300, 9000, 10000, 11000,
          12345, 16383, 64 * 128 + 64, 40 * 128 + 90, 90 * 128 + 40]


def main():
    dims = (64, 64, 64)
    vol = oracle.index_field(hi.plume_dn_grid(64).astype(np.float64), 1.0)
    cam = hi.orbit_camera(dims, 0.0, 0.0, 128, 128)
    bg = hi.checker_background()
    P = hi.params_rk4_fixed(dims, 0.5)
    out = oracle.trace_grid(vol, cam, P, bg, pixels=np.array(PIXELS), nthreads=4)
    rec = {
        "what": "FP64 oracle on the 64^3 plume scene, RK4 h=0.5, 128x128 camera",
        "made_by": "tests/golden/make_oracle_golden.py (calls oracle/ only)",
        "pixels": PIXELS,
        "rgb": out["rgb"].tolist(),
        "exit_pos": out["exit_pos"].tolist(),
        "exit_dir": out["exit_dir"].tolist(),
        "steps": out["steps"].tolist(),
        "flags": out["flags"].tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_plume64_sample.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
