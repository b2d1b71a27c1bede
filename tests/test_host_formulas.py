"""Host checks of closed forms the kernels use, compiled from their own
headers with nvcc and run on the CPU (no GPU needed)."""
import os
import subprocess

import pytest

from paper_2403_06478_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))


def test_band_cells_closed_form(tmp_path):
    """band_cells_through (the cell count the 16-bit kernel reports) equals
    the anti-diagonal-by-anti-diagonal sum of band cells on every prefix."""
    exe = str(tmp_path / "band_cells_check")
    cmd = [B._nvcc()] + B.ARCH + ["-std=c++17", "-O2", "-I" + B.INCLUDE, "-I" + B.CSRC,
                                  os.path.join(HERE, "host", "band_cells_check.cu"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        pytest.fail(f"nvcc failed:\n{res.stdout}\n{res.stderr}")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert " 0 wrong" in run.stdout
