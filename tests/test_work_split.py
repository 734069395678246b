"""CPU check of the persistent work split of the tensor-core kernels: the split code
(tc_common.cuh) is compiled into a host program with nvcc and run here; it checks
coverage, the bands of whole row blocks and the contributor bookkeeping of the row-block
combine over fixed and random shapes (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_work_split_covers_every_unit_once(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "split_check")
    src = os.path.join(ROOT, "tests", "host", "split_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "work split ok" in out.stdout
