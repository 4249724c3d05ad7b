"""The integer-pipe reciprocal used by every elimination step must equal
CUDA's correctly rounded __drcp_rn bit for bit (both are RN(1/a) by IEEE
754; the LU factors' bit-exactness rests on it).  Inputs: random bit
patterns over the whole exponent range, significands whose 2^105 / X lies
within a hair of a rounding midpoint, power-of-two and all-ones
significands, and the fallback range (zero, subnormal, Inf, NaN, huge)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def helper():
    out = os.path.join(tempfile.mkdtemp(), "rcp_check.so")
    src = os.path.join(ROOT, "tests", "gpu_helpers", "rcp_check.cu")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_2609_15217_gb300", "csrc"),
           "-Xcompiler", "-fPIC", "-shared", src, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.rcp_check.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64]
    lib.rcp_check.restype = ctypes.c_int
    return lib


def run(helper, x):
    d = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    o = torch.empty_like(d)
    r = torch.empty_like(d)
    assert helper.rcp_check(d.data_ptr(), o.data_ptr(), r.data_ptr(), d.numel()) == 0
    return o.cpu().numpy(), r.cpu().numpy()


def assert_bitwise(o, r, x):
    ob, rb = o.view(np.uint64), r.view(np.uint64)
    nan = np.isnan(o) & np.isnan(r)
    bad = (ob != rb) & ~nan
    assert not bad.any(), f"{bad.sum()} mismatches, e.g. x={x[bad][:3]!r}"


def test_random_bit_patterns(helper):
    g = np.random.Generator(np.random.Philox(31))
    for _ in range(4):
        bits = g.integers(0, 2 ** 63, size=1 << 24, dtype=np.uint64) | (g.integers(0, 2, size=1 << 24, dtype=np.uint64) << np.uint64(63))
        x = bits.view(np.float64)
        o, r = run(helper, x)
        assert_bitwise(o, r, x)


def test_near_midpoint_significands(helper):
    g = np.random.Generator(np.random.Philox(32))
    Q = (1 << 52) + g.integers(0, 1 << 52, size=1 << 20, dtype=np.uint64).astype(object)
    X = [((1 << 106) + (2 * q + 1) // 2) // (2 * q + 1) for q in Q]
    X = np.array([v for v in X if (1 << 52) < v < (1 << 53)], dtype=np.uint64)
    exps = g.integers(1, 2045, size=X.size, dtype=np.uint64)
    bits = (exps << np.uint64(52)) | (X - np.uint64(1 << 52))
    x = bits.view(np.float64)
    o, r = run(helper, x)
    assert_bitwise(o, r, x)


def test_special_values(helper):
    vals = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 2.2250738585072014e-308, 2.2250738585072009e-308,
            1.0, -1.0, 2.0, 0.5, 3.0, 1.7976931348623157e308, 2.0 ** 1021, 2.0 ** 1022, 2.0 ** 1023,
            1.5 * 2.0 ** 1021, 1.9999999999999998 * 2.0 ** 1020, 2.0 ** -1022, 3 * 2.0 ** -1023]
    sig = [(1 << 53) - 1, (1 << 52) + 1, (1 << 52) + (1 << 29) - 1, (1 << 52) + (1 << 29), (1 << 52) + (1 << 28)]
    for e in (1, 2, 1023, 2043, 2044, 2045, 2046):
        for m in sig:
            vals.append(np.array([(e << 52) | (m - (1 << 52))], dtype=np.uint64).view(np.float64)[0])
    x = np.array(vals + [-v for v in vals])
    o, r = run(helper, x)
    assert_bitwise(o, r, x)
