"""Host build of the kernel's index, key and hash helpers, checked against brute force and
against splitmix64 (Steele, Lea and Flood 2014) written here from its published definition."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not installed")
def test_device_helpers(tmp_path):
    exe = tmp_path / "device_helpers_check"
    subprocess.check_call(["nvcc", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2101_07690_gb300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "device_helpers_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr
    assert "fails 0" in out.stdout
    lines = [l.split() for l in out.stdout.splitlines() if l.startswith("hash ")]
    assert len(lines) == 48
    for _, sd, x, y, h in lines:
        ref = splitmix64(int(sd))
        ref = splitmix64(ref ^ (int(x) & 0xFFFFFFFF))
        ref = splitmix64(ref ^ (int(y) & 0xFFFFFFFF))
        assert int(h) == ref, (sd, x, y)


def test_splitmix64_published_first_output():
    # the first output of the reference generator seeded with 0 (state advanced once)
    assert splitmix64(0) == 0xE220A8397B1DCDAF
