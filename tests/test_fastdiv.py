"""Host check of the multiply-shift division constants (make_fast_div in
csrc/kernels.h) that the tensor-core kernel's tile and K-step decodes use:
compiled as host code with nvcc and compared with integer division over
small, near-multiple, random and extreme numerators below 2^31 for every
divisor up to 4096 and a few large ones (CPU only)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_03882_gb300", "csrc")


def test_fast_div_constants():
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if not nvcc:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fastdiv_check")
        r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "fastdiv_check.cu"), "-o", exe],
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
