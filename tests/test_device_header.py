"""The public device-callable header (include/tinylu_device.cuh) compiles for
sm_103a on its own: a user kernel that includes nothing else instantiates
tl::lupp_solve and tl::lupp_solve_subwarp (nvcc cross-compiles without a
GPU; the GPU parity of both entry points is tests/test_gpu_device_api.py)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_device_header_is_self_contained():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("no nvcc")
    with tempfile.TemporaryDirectory() as d:
        out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                              "-I" + os.path.join(ROOT, "include"), "-c",
                              os.path.join(ROOT, "tests", "cpu_helpers", "device_header_use.cu"),
                              "-o", os.path.join(d, "use.o")], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
