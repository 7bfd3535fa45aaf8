"""The host-pool arena's quarantine of slow ranges, checked by a small C++
program compiled against the runtime's own header (no GPU needed)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_05549_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def test_quarantined_ranges_are_never_allocated(tmp_path):
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "arena_check")
    r = subprocess.run([NVCC, "-std=c++17", "-x", "c++", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "native", "arena_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "arena checks ok" in r.stdout
