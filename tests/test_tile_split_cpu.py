"""Host check of the contraction's weighted tile split (``tile_lo`` / ``tile_owner`` of the
tensor-core contraction header): compiled with nvcc for the host, no GPU needed.  The
ranges must partition the tiles, the O(1) owner formula must agree with the ranges for every
tile, and each CTA's share must follow its weight (1 for the 16 CTAs that also form the Gram
partials, 8 for the others)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_split_partitions_and_owner_formula(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "tile_split_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-diag-suppress", "177", "-I", os.path.join(ROOT, "paper_2410_15519_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "tile_split_check.cu"), "-o", exe],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "tile split ok" in out.stdout
