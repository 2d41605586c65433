"""Host-only check of the kernel layouts (CPU): tests/layout_check.cpp is
compiled against the library's host sources and emulates, in FP64, one
explicit flux step over the replica layout (also with a shard halo) and the
SpMV warp kernel's chunks, runs and segmented scan, against the plain
edge-list computations."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1605_02043_gb300", "csrc")


def test_layouts_emulated_on_the_host(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "layout_check")
    srcs = [os.path.join(ROOT, "tests", "layout_check.cpp")] + [
        os.path.join(CSRC, f) for f in ("partition.cpp", "prescreen.cpp", "schedule.cpp")]
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, *srcs,
                    "-o", exe, "-lpthread"], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "total fails 0" in r.stdout, r.stdout[-3000:]
