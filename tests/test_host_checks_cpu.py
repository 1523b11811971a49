"""Host-side checks of the library's __host__ __device__ building blocks
(no GPU): compiles tests/host/host_checks.cu as host code with nvcc and runs
it.  It pins the FP64 -> FP32 rounding, the FP32 -> FP64 widening and the
float-float split that the kernels do with integer operations against the
host's IEEE conversions, bit for bit, and the representation's folded
entry and row formulas against the plain sums over the basis elements."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _nvcc():
    for cand in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and Path(cand).exists():
            return cand
    return None


def test_host_checks(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "host_checks"
    cmd = [nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-x", "cu",
           f"-I{ROOT / 'include'}", f"-I{ROOT / 'paper_2503_06721_gb300' / 'csrc'}",
           str(ROOT / "tests" / "host" / "host_checks.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "conversion mismatches 0" in r.stdout
