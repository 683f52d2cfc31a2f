"""Launch shapes of the tiled polish and the batched FP64 re-decision (host
arithmetic only, no GPU): for every layer width, input dimension and
sign-word count the library accepts, in both builds (D <= 8 and D <= 10),
the busy blocks fit the CTA, tiles hold whole 4-vertex groups, workspace
regions are 16-byte aligned and shared memory stays within the launch
attribute (`tests/c/launch_shapes.cu` includes the kernel sources as they
are and launches nothing)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("max_d", [8, 10])
def test_launch_shapes(tmp_path, max_d):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / f"launch_shapes_{max_d}")
    cmd = [nvcc, "-std=c++17", f"-DPC_MAX_D={max_d}", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_2306_07212_gb300", "csrc"),
           os.path.join(ROOT, "tests", "c", "launch_shapes.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("0 failures"), r.stdout[-2000:]
