"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/hh.h declares, and the binding's ctypes
structures have the C layout (checked against sizeof/offsetof compiled from
the header by gcc)."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hh.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2603_02048_gb300 import build, hh

    build.build()
    return hh, hh.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    hh, so = lib
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(so, n), n
        assert n in hh.SIGNATURES, f"binding lacks {n}"
        assert hasattr(hh, n), f"binding has no Python function {n}"
    assert set(hh.SIGNATURES) == set(names)


def test_struct_layouts_match_header(lib):
    import ctypes

    hh, _ = lib
    structs = {"hh_particles": ["xyzm_dev", "n"],
               "hh_grid": ["nx", "ny", "nz", "h_kernel", "storage"],
               "hh_camera": ["eye", "look_at", "up", "vfov_deg", "width", "height"],
               "hh_step_params": ["stepper", "adaptive", "h_fixed", "h_min", "h_max", "theta_max",
                                  "eps", "max_steps"],
               "hh_background": ["rgb8_dev", "width", "height", "n_planes", "planes"],
               "hh_plane": ["origin", "u", "v", "rgb8_dev", "width", "height"],
               "hh_view_out": ["rgb", "exit_pos", "exit_dir", "steps", "flags", "rgb8"],
               "hh_batch_config": ["block_threads", "blocks_per_sm", "refill_min", "tile_w",
                                   "tile_order", "tile_group"],
               "hh_serve_stats": ["submitted", "admitted", "completed", "cancelled", "failed",
                                  "rejected", "pending", "running", "rays_completed",
                                  "pool_used", "pool_capacity", "worker_launches",
                                  "worker_idle_exits", "entry_timeouts"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             "int main(void) {"]
    for s, fields in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    c = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for s, fields in structs.items():
        cls = getattr(hh, s)
        assert ctypes.sizeof(cls) == int(c[s]), s
        for f in fields:
            assert getattr(cls, f).offset == int(c[f"{s}.{f}"]), f"{s}.{f}"


def test_library_refuses_to_run_without_build(tmp_path):
    """The binding raises when the CUDA library is absent: no CPU fallback."""
    from paper_2603_02048_gb300 import hh

    with pytest.raises(RuntimeError, match="missing"):
        saved, hh._lib = hh._lib, None
        try:
            hh.load(str(tmp_path / "libhh.so"))
        finally:
            hh._lib = saved
