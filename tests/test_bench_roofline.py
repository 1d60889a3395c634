"""The bench line's roofline object (host logic of bench.py, no GPU): the
three legs follow their definitions, `bound` is the slowest of them, the
committed counters are used only for the march source they were taken on,
and without counters the line says so instead of reporting a partial bound."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FRAME = dict(ms_march=0.39, total_steps=62391878, n_rays=2073600,
             clocks={"sm_mhz": 2070.0}, sm_count=152, kernel="march_kernel")
COUNTERS = {"dram_bytes_per_launch": 185_000_000, "warp_instructions_per_launch": 360_000_000,
            "l1_hit_rate": 91.0}


def test_legs_follow_their_definitions(monkeypatch):
    monkeypatch.setattr(bench, "march_counters", lambda w: dict(COUNTERS))
    r = bench.roofline("frame", "fp32", **FRAME)
    sec = FRAME["ms_march"] * 1e-3
    hbm, _ = bench.measured_peaks()
    legs = r["legs"]
    assert set(legs) == {"hbm", "fp32", "issue"}
    assert legs["hbm"]["frac"] == pytest.approx(COUNTERS["dram_bytes_per_launch"] / sec / 1e9 / hbm,
                                                abs=1e-4)
    flops = FRAME["total_steps"] * bench.FLOPS_PER_STEP["fp32"]
    assert legs["fp32"]["frac"] == pytest.approx(flops / sec / (152 * 128 * 2 * 2070e6), abs=1e-4)
    assert legs["issue"]["frac"] == pytest.approx(
        COUNTERS["warp_instructions_per_launch"] / sec / (152 * 4 * 2070e6), abs=1e-4)
    # the bound is the slowest leg, and the line's figures are that leg's
    fr = {k: v["frac"] for k, v in legs.items()}
    assert r["bound"] == max(fr, key=fr.get) == "issue"
    assert (r["frac"], r["achieved"], r["peak"], r["unit"]) == (
        legs["issue"]["frac"], legs["issue"]["achieved"], legs["issue"]["peak"],
        legs["issue"]["unit"])
    assert r["traffic"] == COUNTERS["dram_bytes_per_launch"]
    # the counted corner fetches ride along, apart from the DRAM figure
    assert r["counted_fetch"]["bytes_per_launch"] == FRAME["total_steps"] * 128 + FRAME["n_rays"] * 24


def test_a_memory_bound_launch_is_reported_as_such(monkeypatch):
    monkeypatch.setattr(bench, "march_counters",
                        lambda w: {"dram_bytes_per_launch": 2_600_000_000,
                                   "warp_instructions_per_launch": 100_000_000})
    r = bench.roofline("frame", "fp32", **FRAME)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_without_counters_the_line_says_so(monkeypatch):
    monkeypatch.setattr(bench, "march_counters", lambda w: {})
    r = bench.roofline("frame", "fp32", **FRAME)
    assert set(r["legs"]) == {"fp32"} and r["traffic"] is None
    assert "absent" in r["note"]


def test_counters_are_tied_to_the_march_source(tmp_path, monkeypatch):
    """march_counters reads the record only when its hash is the current
    march.cu's (a record for another source is ignored, not misused)."""
    csrc = tmp_path / "paper_2603_02048_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "march.cu"
    src.write_bytes(b"// a march source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    rec = {"march_cu_sha256": sha, "workloads": {"frame": dict(COUNTERS)}}
    (tmp_path / "profiles" / "march_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.march_counters("frame") == COUNTERS
    assert bench.march_counters("batch") == {}
    src.write_bytes(b"// another march source\n")
    assert bench.march_counters("frame") == {}
