"""The public device-callable solvers (include/tinylu_device.cuh:
tl::lupp_solve, one thread per system, and tl::lupp_solve_subwarp, T lanes
per system) called from a user kernel that includes that header alone,
against the oracle system by system: pivots and info bit-identical, x within
backward error 10n and forward error 1e-12 kappa; special systems (exact
zero pivot, NaN, infinity, exact ties) in every batch; a batch that does not
fill the last warp."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

from test_gpu_lupp import check_solution  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [(1, 1), (3, 1), (7, 1), (9, 1), (10, 2), (13, 4), (20, 8), (32, 16), (32, 32)]


@pytest.fixture(scope="module")
def helper():
    out = os.path.join(tempfile.mkdtemp(), "device_api.so")
    src = os.path.join(ROOT, "tests", "gpu_helpers", "device_api.cu")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-I" + os.path.join(ROOT, "include"), "-Xcompiler", "-fPIC", "-shared", src, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.device_api_solve.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_int64]
    lib.device_api_solve.restype = ctypes.c_int
    return lib


def solve(helper, n, T, A, b):
    S = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1)).reshape(-1)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).cuda()
    dx = torch.full_like(db, -7.0)
    dp = torch.full((S * n,), -7, dtype=torch.int32, device="cuda")
    di = torch.full((S,), -7, dtype=torch.int32, device="cuda")
    assert helper.device_api_solve(n, T, dA.data_ptr(), db.data_ptr(), dx.data_ptr(), dp.data_ptr(),
                                   di.data_ptr(), S) == 0
    return (dx.cpu().numpy().reshape(S, n), dp.cpu().numpy().reshape(S, n), di.cpu().numpy())


@pytest.mark.parametrize("n,T", CASES)
def test_device_api_against_oracle(helper, n, T):
    S = 1000 + 13
    A, b, _, _ = inputs.sweep_systems(n, S, inputs.config_seed(7, n))
    A = A.copy()
    b = b.copy()
    # special systems: exact zero pivot (a zero column), NaN, Inf, exact ties
    A[0, :, n // 2] = 0.0
    A[1, n - 1, 0] = np.nan
    A[2, 0, n - 1] = np.inf
    A[3] = np.round(A[3] * 4.0)
    A[3, :, 0] = np.where(np.arange(n) % 2 == 0, 3.0, -3.0)
    x_o, piv_o, info_o, _ = oracle.gesv(A, b)
    x, piv, info = solve(helper, n, T, A, b)
    assert np.array_equal(info, info_o), np.nonzero(info != info_o)[0][:5]
    assert info[0] == n // 2 + 1 or n == 1
    assert info[1] == -1 and info[2] == -1
    assert np.array_equal(piv, piv_o), np.nonzero((piv != piv_o).any(axis=1))[0][:5]
    assert np.isnan(x[info != 0]).all()
    ok = info == 0
    check_solution(A[ok], b[ok], x[ok], x_o[ok])
