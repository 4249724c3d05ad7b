"""GPU parity of the batched LUpp kernels against the CPU oracle, through
the C ABI (tl_gesv_batched / tl_getrf_batched / tl_getrs_batched).

Bar (paper Sec. 2.2 arithmetic, identical on both sides):
  * pivots, info and the LU factors: bit-identical to the oracle;
  * x: normwise backward error ||Ax - b|| / (||A|| ||x|| eps) <= 10 n and
    forward error against the oracle's x <= 1e-12 * kappa(A) (the GPU back
    substitution multiplies by RN(1/u_ii) where the oracle divides).
Sizes span several thread blocks and end on a ragged tail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402
from paper_2609_15217_gb300 import layout as L  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
DEV = "cuda"


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture(scope="module")
def h(tl):
    hh = tl.tl_create()
    yield hh
    tl.tl_destroy(hh)


def gpu_gesv(tl, h, A, b, layout, want_lu=True, ld=None):
    batch, n, _ = A.shape
    ld = ld or L.pad_ld(batch)
    dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
    db = L.vectors_to_layout(torch.from_numpy(b).to(DEV), layout, ld)
    dx = torch.full_like(db, -7.0)
    dLU = torch.full_like(dA, -7.0) if want_lu else None
    dpiv = torch.full((db.numel(),), -7, dtype=torch.int32, device=DEV)
    dinfo = torch.full((batch,), -7, dtype=torch.int32, device=DEV)
    st = tl.tl_gesv_batched(h, n, dA, dLU, db, dx, dpiv, dinfo, layout, ld, batch)
    tl.check("tl_gesv_batched", st, h)
    torch.cuda.synchronize()
    x = L.vectors_from_layout(dx, batch, n, layout, ld).cpu().numpy()
    piv = L.vectors_from_layout(dpiv, batch, n, layout, ld).cpu().numpy()
    info = dinfo.cpu().numpy()
    LU = L.matrices_from_layout(dLU, batch, n, layout, ld).cpu().numpy() if want_lu else None
    return x, piv, info, LU


def backward_error(A, x, b):
    r = np.einsum("sij,sj->si", A.astype(np.longdouble), x.astype(np.longdouble)) - b.astype(np.longdouble)
    r = np.abs(r).max(axis=1).astype(np.float64)
    return r / (np.abs(A).sum(axis=2).max(axis=1) * np.abs(x).max(axis=1) * EPS)


def check_solution(A, b, x_gpu, x_orc):
    n = A.shape[-1]
    be = backward_error(A, x_gpu, b)
    assert (be <= 10 * n).all(), f"backward error {be.max():.3g} > {10 * n}"
    kappa = np.linalg.cond(A)
    fe = np.abs(x_gpu - x_orc).max(axis=1) / np.maximum(np.abs(x_orc).max(axis=1), 1e-300)
    assert (fe <= 1e-12 * kappa).all(), f"forward error / kappa {np.max(fe / kappa):.3g}"


ALL_N = list(range(1, 33))


@pytest.mark.parametrize("layout", [0, 1], ids=["per_system", "interleaved"])
@pytest.mark.parametrize("n", ALL_N)
def test_gesv_parity(tl, h, n, layout):
    batch = 3 * 128 + 37
    A, b, _, _ = inputs.sweep_systems(n, batch, inputs.config_seed(2, n))
    x_o, piv_o, info_o, gap, LU_o = oracle.gesv(A, b, want_lu=True)
    x_g, piv_g, info_g, LU_g = gpu_gesv(tl, h, A, b, layout)
    assert np.array_equal(info_g, info_o)
    assert np.array_equal(piv_g, piv_o), f"pivot mismatches: {(piv_g != piv_o).any(axis=1).sum()}"
    assert np.array_equal(LU_g.view(np.int64), LU_o.view(np.int64)), "LU factors differ from the oracle (bitwise)"
    check_solution(A, b, x_g, x_o)
    # without the factors output (the fused kernel that keeps L unpermuted)
    x_g2, piv_g2, info_g2, _ = gpu_gesv(tl, h, A, b, layout, want_lu=False)
    assert np.array_equal(piv_g2, piv_o) and np.array_equal(info_g2, info_o)
    assert np.array_equal(x_g2, x_g)


@pytest.mark.parametrize("layout", [0, 1], ids=["per_system", "interleaved"])
@pytest.mark.parametrize("n", [1, 2, 5, 8, 9, 10, 12, 13, 16, 17, 24, 25, 31, 32])
def test_getrf_getrs_parity(tl, h, n, layout):
    batch = 2 * 128 + 5
    A, b = inputs.uniform_systems(n, batch, 4000 + n)
    LU_o, piv_o, info_o, _ = oracle.getrf(A)
    ld = L.pad_ld(batch)
    dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
    dpiv = torch.zeros(n * (ld if layout else batch), dtype=torch.int32, device=DEV)
    dinfo = torch.zeros(batch, dtype=torch.int32, device=DEV)
    tl.check("getrf", tl.tl_getrf_batched(h, n, dA, layout, ld, dpiv, dinfo, batch), h)
    torch.cuda.synchronize()
    LU_g = L.matrices_from_layout(dA, batch, n, layout, ld).cpu().numpy()
    piv_g = L.vectors_from_layout(dpiv, batch, n, layout, ld).cpu().numpy()
    assert np.array_equal(dinfo.cpu().numpy(), info_o)
    assert np.array_equal(piv_g, piv_o)
    assert np.array_equal(LU_g.view(np.int64), LU_o.view(np.int64))
    for nrhs in (1, 3):
        B = inputs.rng(4100 + n).uniform(-1, 1, size=(batch, nrhs, n))
        dB = L.multi_rhs_to_layout(torch.from_numpy(B).to(DEV), layout, ld)
        tl.check("getrs", tl.tl_getrs_batched(h, n, nrhs, dA, dpiv, layout, ld, dB, batch), h)
        torch.cuda.synchronize()
        X_g = L.multi_rhs_from_layout(dB, batch, nrhs, n, layout, ld).cpu().numpy()
        for r in range(nrhs):
            x_o = oracle.getrs(LU_o, piv_o, B[:, r, :])
            check_solution(A, B[:, r, :], X_g[:, r, :], x_o)


@pytest.mark.parametrize("n", [3, 8, 11, 16, 20, 32])
def test_edge_cases(tl, h, n):
    """Zero pivots, all-zero and non-finite systems, exact ties, a pivot
    below DBL_MIN, and the stress magnitude range of Sec. 4.2."""
    batch = 70
    A, b = inputs.uniform_systems(n, batch, 4200 + n)
    A[0, :, min(2, n - 1)] = 0.0                 # zero pivot at step 2 (or n-1)
    A[1] = 0.0                                   # every pivot zero
    A[2, n // 2, n // 3] = np.nan                # non-finite
    A[3, 0, 0] = np.inf
    A[4, :, 0] = 1.0                             # exact tie in column 0
    A[4, :, 0] *= np.where(np.arange(n) % 2, -1.0, 1.0)
    A[5] *= 2.0 ** -1060                         # subnormal pivots (quotient branch)
    A[6] = np.ldexp(A[6], -31)                   # stress range, U[-4.7e-10, 4.7e-10]
    A[7] = np.eye(n)[::-1] * 3.0                 # anti-diagonal permutation
    A[8, :, :] = A[8, :, :] * 0 + np.triu(np.ones((n, n)))  # upper triangular ones
    for layout in (0, 1):
        x_o, piv_o, info_o, _, LU_o = oracle.gesv(A, b, want_lu=True)
        x_g, piv_g, info_g, LU_g = gpu_gesv(tl, h, A, b, layout)
        assert np.array_equal(info_g, info_o)
        assert np.array_equal(piv_g, piv_o)
        ok = info_o == 0
        bad = info_o < 0
        assert np.array_equal(LU_g[~bad].view(np.int64), LU_o[~bad].view(np.int64))
        assert np.array_equal(LU_g[bad], A[bad], equal_nan=True)  # nothing factored
        assert np.isnan(x_g[~ok]).all()
        normal = ok & (np.arange(batch) != 5)
        check_solution(A[normal], b[normal], x_g[normal], x_o[normal])
        # pivots below DBL_MIN: both sides divide in the substitution, so the
        # solution is bit-identical too
        assert np.array_equal(x_g[5], x_o[5], equal_nan=True)


def test_x_aliases_b_and_tiny_batches(tl, h):
    n = 8
    for batch in (1, 2, 31, 33):
        A, b = inputs.uniform_systems(n, batch, 4300 + batch)
        x_o, piv_o, info_o, _ = oracle.gesv(A, b)
        for layout in (0, 1):
            ld = L.pad_ld(batch)
            dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
            db = L.vectors_to_layout(torch.from_numpy(b).to(DEV), layout, ld)
            dpiv = torch.zeros(db.numel(), dtype=torch.int32, device=DEV)
            dinfo = torch.zeros(batch, dtype=torch.int32, device=DEV)
            tl.check("gesv", tl.tl_gesv_batched(h, n, dA, None, db, db, dpiv, dinfo, layout, ld, batch), h)
            torch.cuda.synchronize()
            x_g = L.vectors_from_layout(db, batch, n, layout, ld).cpu().numpy()
            check_solution(A, b, x_g, x_o)


def test_argument_errors(tl, h):
    d = torch.zeros(64, dtype=torch.float64, device=DEV)
    i = torch.zeros(64, dtype=torch.int32, device=DEV)
    assert tl.tl_gesv_batched(h, 0, d, None, d, d, i, i, 0, 0, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 2
    assert tl.tl_gesv_batched(h, 33, d, None, d, d, i, i, 0, 0, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_gesv_batched(h, 4, d, None, d, d, i, i, 1, 3, 4) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 10          # ld_batch < batch
    assert tl.tl_gesv_batched(h, 4, None, None, d, d, i, i, 0, 0, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 3
    assert tl.tl_gesv_batched(h, 4, d, None, d, d, i, i, 7, 0, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 9
    assert tl.tl_gesv_batched(h, 4, d, None, d, d, i, i, 0, 0, -1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_gesv_batched(h, 4, d, None, d, d, i, i, 0, 0, 0) == tl.TL_OK  # empty batch
    assert tl.tl_getrs_batched(h, 4, 0, d, i, 0, 0, d, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 3
    assert tl.tl_getrf_batched(h, 4, d.data_ptr() + 4, 0, 0, i, i, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 3           # misaligned
