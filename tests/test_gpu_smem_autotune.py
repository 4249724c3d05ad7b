"""GPU parity of the shared-memory solver variants (run-time n, T lanes per
system, position -> row table for the interchanges) selected through the
dispatch table, and of the autotuned dispatch (Sec. 4.1 "best X" reporting
convention).  Same bar as the register kernels: pivots, info and LU
bit-identical to the oracle, x within BE 10 n and FE 1e-12 kappa."""
import json
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

from test_gpu_lupp import check_solution, gpu_gesv  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture()
def h(tl):
    hh = tl.tl_create()
    yield hh
    tl.tl_destroy(hh)


@pytest.mark.parametrize("lanes,walk", [(2, False), (4, False), (8, False), (16, False), (32, False),
                                        (2, True), (4, True), (8, True)])
@pytest.mark.parametrize("n", [2, 3, 7, 9, 10, 13, 16, 17, 24, 25, 31, 32])
def test_shared_memory_variants(tl, h, n, lanes, walk):
    batch = 3 * 64 + 11
    A, b, _, _ = inputs.sweep_systems(n, batch, inputs.config_seed(2, n) + 7)
    A[3, :, 1] = 0.0            # a zero pivot
    A[5, n - 1, n - 1] = np.nan  # a non-finite system
    x_o, piv_o, info_o, _, LU_o = oracle.gesv(A, b, want_lu=True)
    for layout in (0, 1):
        vid = tl.variant_id(lanes, shared=True, walk=walk)
        assert tl.tl_dispatch_set(h, n, layout, vid, 0) == tl.TL_OK
        assert tl.tl_dispatch_get(h, n, layout)[1] == vid
        x_g, piv_g, info_g, LU_g = gpu_gesv(tl, h, A, b, layout)
        assert np.array_equal(info_g, info_o)
        assert np.array_equal(piv_g, piv_o)
        bad = info_o < 0
        assert np.array_equal(LU_g[~bad].view(np.int64), LU_o[~bad].view(np.int64))
        assert np.array_equal(LU_g[bad], A[bad], equal_nan=True)
        ok = info_o == 0
        assert np.isnan(x_g[~ok]).all()
        check_solution(A[ok], b[ok], x_g[ok], x_o[ok])
        x_g2, piv_g2, info_g2, _ = gpu_gesv(tl, h, A, b, layout, want_lu=False)
        assert np.array_equal(piv_g2, piv_o) and np.array_equal(x_g2, x_g, equal_nan=True)


@pytest.mark.parametrize("lanes", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("n", [5, 13, 20, 27, 32])
def test_walk_pivot_ties(tl, h, n, lanes):
    """Integer entries in {-2..2}: nearly every column holds several entries
    of the largest magnitude, so the first-maximum rule (the smallest row
    among exact ties) decides most pivots; the 8-, 16- and 32-lane walks
    find it with warp reductions, the others with a shuffle butterfly.
    Pivots, info and LU bit-identical to the oracle, both layouts."""
    batch = 2 * 64 + 5
    g = inputs.rng(8100 + 33 * n + lanes)
    A = g.integers(-2, 3, size=(batch, n, n)).astype(np.float64)
    b = g.uniform(-1, 1, size=(batch, n))
    A[7, :, :] = 1.0               # every candidate of every column tied
    A[9] = np.eye(n)[::-1] * 2.0   # ties with zeros below
    x_o, piv_o, info_o, _, LU_o = oracle.gesv(A, b, want_lu=True)
    vid = tl.variant_id(lanes, shared=True, walk=lanes < 16)
    for layout in (0, 1):
        assert tl.tl_dispatch_set(h, n, layout, vid, 0) == tl.TL_OK
        x_g, piv_g, info_g, LU_g = gpu_gesv(tl, h, A, b, layout)
        assert np.array_equal(info_g, info_o)
        assert np.array_equal(piv_g, piv_o)
        assert np.array_equal(LU_g.view(np.int64), LU_o.view(np.int64))
        ok = info_o == 0
        check_solution(A[ok], b[ok], x_g[ok], x_o[ok])


@pytest.mark.parametrize("n", [9, 20, 32])
def test_shared_memory_getrf(tl, h, n):
    from paper_2609_15217_gb300 import layout as L
    batch = 150
    A, _ = inputs.uniform_systems(n, batch, 8000 + n)
    LU_o, piv_o, info_o, _ = oracle.getrf(A)
    for layout in (0, 1):
        tl.tl_dispatch_set(h, n, layout, tl.variant_id(8, shared=True), 64)
        ld = L.pad_ld(batch)
        dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
        dpiv = torch.zeros(n * (ld if layout else batch), dtype=torch.int32, device=DEV)
        dinfo = torch.zeros(batch, dtype=torch.int32, device=DEV)
        tl.check("getrf", tl.tl_getrf_batched(h, n, dA, layout, ld, dpiv, dinfo, batch), h)
        torch.cuda.synchronize()
        LU_g = L.matrices_from_layout(dA, batch, n, layout, ld).cpu().numpy()
        assert np.array_equal(L.vectors_from_layout(dpiv, batch, n, layout, ld).cpu().numpy(), piv_o)
        assert np.array_equal(LU_g.view(np.int64), LU_o.view(np.int64))
        assert np.array_equal(dinfo.cpu().numpy(), info_o)


def test_dispatch_errors(tl, h):
    assert tl.tl_dispatch_set(h, 0, 0, 1, 0) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_dispatch_set(h, 8, 0, 999, 0) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 4
    assert tl.tl_dispatch_set(h, 8, 0, 1, 48) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_dispatch_set(h, 8, 0, 101, 0) == tl.TL_ERR_INVALID_ARG  # one lane is not a shared variant
    assert tl.tl_dispatch_set(h, 8, 0, 0, 0) == tl.TL_OK
    assert tl.tl_dispatch_get(h, 8, 0)[1] == 1


def test_autotune_table_and_parity(tl, h):
    path = os.path.join(tempfile.mkdtemp(), "tune.json")
    st = tl.tl_autotune(h, 7, 10, 1, path)
    assert st == tl.TL_OK
    table = json.load(open(path))
    assert [e["n"] for e in table["entries"]] == [7, 8, 9, 10]
    for e in table["entries"]:
        assert tl.tl_dispatch_get(h, e["n"], 1)[1] == e["variant"]
        assert e["block"] in (32, 64, 128) and e["ms"] > 0
    for n in (7, 10):
        A, b, _, _ = inputs.sweep_systems(n, 300, 9100 + n)
        x_o, piv_o, info_o, _ = oracle.gesv(A, b)
        x_g, piv_g, info_g, _ = gpu_gesv(tl, h, A, b, 1, want_lu=False)
        assert np.array_equal(piv_g, piv_o) and np.array_equal(info_g, info_o)
        check_solution(A, b, x_g, x_o)
