"""The bit-level FP64/FP32 helpers of the integrator (md_device.cuh: widen,
narrow_trunc, split_hilo, wrap_box_bits) against the hardware conversions
and their stated bounds, on the host (the helpers are __host__ __device__).
Host logic only: compiled with nvcc, no GPU needed."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


@pytest.mark.skipif(not Path(NVCC).exists(), reason="nvcc not available")
def test_bit_helpers_match_hardware_conversions(tmp_path):
    exe = tmp_path / "bits_check"
    cmd = [NVCC, "-O2", "-std=c++17", "-I", str(ROOT / "paper_1412_8502_b300" / "csrc"), "-I", str(ROOT / "include"),
           str(ROOT / "tests" / "bits_check.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe), "1000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "widen: 0 mismatches" in r.stdout and "wrap_box_bits: 0 mismatches" in r.stdout, r.stdout
