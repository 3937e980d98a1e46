"""Host checks of index arithmetic in the step kernel's headers, compiled with nvcc for the
host (no GPU needed):
  * the contraction's weighted tile split (``tile_lo`` / ``tile_owner``): the ranges must
    partition the tiles, the O(1) owner formula must agree with the ranges for every tile,
    and each CTA's share must follow its weight (1 for the 16 CTAs that also form the Gram
    partials, 8 for the others);
  * the tile-image layout (``tc_img_index``) against the canonical K-major core-matrix
    layout its descriptors declare, and the separated form's multiset table."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("source,ok", [("tile_split_check.cu", "tile split ok"), ("layout_check.cu", "layout ok")])
def test_host_index_checks(tmp_path, source, ok):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / source.replace(".cu", ""))
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-diag-suppress", "177", "-I", os.path.join(ROOT, "paper_2410_15519_gb300", "csrc"),
                    os.path.join(ROOT, "tests", source), "-o", exe],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    assert ok in out.stdout
