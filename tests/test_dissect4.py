"""The four-vertex dissection closed form used by the extension kernel equals Algorithm 1's
general smallest-vertex-first dissection on every four-vertex join (host build, no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not installed")
def test_dissect4_matches_dissect3(tmp_path):
    exe = tmp_path / "dissect4_check"
    subprocess.check_call(["nvcc", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2101_07690_gb300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "dissect4_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout
    assert "checked 1152" in out.stdout
