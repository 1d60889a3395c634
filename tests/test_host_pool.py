"""CPU tests of the render server's host logic: its output-memory allocator
(tests/native/pool_test.cpp against csrc/pool.h) and its admission order
(tests/native/admission_test.cpp against csrc/admission.h), each compiled
with g++ and run."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_offset_pool(tmp_path):
    exe = tmp_path / "pool_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2603_02048_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "pool_test.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "pool ok" in r.stdout


def test_admission_order(tmp_path):
    exe = tmp_path / "admission_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2603_02048_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "admission_test.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "admission ok" in r.stdout
