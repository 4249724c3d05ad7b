"""GPU parity of tile-local pivoting (tl_gesv_batched_tilepiv; Sec. 3.2 Tiled
solvers with the 1e-10 acceptance threshold of Sec. 4.1) against the
oracle's getrf_tiled: pivots, info and LU factors bit-identical, x within
the forward-error bar of the oracle's solve with the same factors, on the
default and the stress distributions and both layouts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402
from paper_2609_15217_gb300 import layout as L  # noqa: E402

pytestmark = pytest.mark.gpu
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


def run(tl, h, A, b, tile, layout, thr=1e-10):
    batch, n = A.shape[0], A.shape[1]
    ld = L.pad_ld(batch)
    dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
    db = L.vectors_to_layout(torch.from_numpy(b).to(DEV), layout, ld)
    dLU = torch.empty_like(dA)
    dx = torch.empty_like(db)
    dpiv = torch.empty(db.numel(), dtype=torch.int32, device=DEV)
    dinfo = torch.empty(batch, dtype=torch.int32, device=DEV)
    tl.check("tilepiv", tl.tl_gesv_batched_tilepiv(h, n, tile, thr, dA, dLU, db, dx, dpiv, dinfo, layout, ld, batch), h)
    torch.cuda.synchronize()
    return (L.vectors_from_layout(dx, batch, n, layout, ld).cpu().numpy(),
            L.vectors_from_layout(dpiv, batch, n, layout, ld).cpu().numpy(), dinfo.cpu().numpy(),
            L.matrices_from_layout(dLU, batch, n, layout, ld).cpu().numpy())


@pytest.mark.parametrize("n", [2, 5, 9, 12, 17, 32])
@pytest.mark.parametrize("dist", ["default", "stress"])
def test_tile_local_pivoting(tl, h, n, dist):
    batch = 200 + 7
    A, b = inputs.uniform_systems(n, batch, 7000 + n, -0.5, 0.5)
    if dist == "stress":
        A, b = A * 1e-9, b * 1e-9        # U[+-5e-10]
    for tile in (2, 3, 6):
        LU_o, piv_o, info_o, oot = oracle.getrf_tiled(A, tile, 1e-10)
        if dist == "default":
            assert (oot == 0).all()
        for layout in (0, 1):
            x, piv, info, LU = run(tl, h, A, b, tile, layout)
            assert np.array_equal(piv, piv_o) and np.array_equal(info, info_o)
            assert np.array_equal(LU.view(np.int64), LU_o.view(np.int64))
            x_o = oracle.getrs(LU_o, piv_o, b)
            kappa = np.linalg.cond(A)
            fe = np.abs(x - x_o).max(axis=1) / np.abs(x_o).max(axis=1)
            assert (fe <= 1e-12 * kappa).all()
    if dist == "stress" and n >= 5:
        assert (oracle.getrf_tiled(A, 2, 1e-10)[3] > 0).any()


def test_tile_zero_is_textbook(tl, h):
    n, batch = 13, 150
    A, b = inputs.uniform_systems(n, batch, 7100)
    _, piv_o, info_o, _, LU_o = oracle.gesv(A, b, want_lu=True)
    for tile in (0, n, 40):
        x, piv, info, LU = run(tl, h, A, b, tile, 1)
        assert np.array_equal(piv, piv_o) and np.array_equal(LU.view(np.int64), LU_o.view(np.int64))


def test_tilepiv_argument_errors(tl, h):
    d = torch.zeros(64, dtype=torch.float64, device=DEV)
    i = torch.zeros(64, dtype=torch.int32, device=DEV)
    f = tl.tl_gesv_batched_tilepiv
    assert f(h, 4, -1, 1e-10, d, None, d, d, i, i, 0, 1, 1) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 3
    assert f(h, 4, 2, -1.0, d, None, d, d, i, i, 0, 1, 1) == tl.TL_ERR_INVALID_ARG
    assert f(h, 33, 2, 1e-10, d, None, d, d, i, i, 0, 1, 1) == tl.TL_ERR_INVALID_ARG
    assert f(h, 4, 2, 1e-10, d, None, d, d, i, i, 0, 1, 0) == tl.TL_OK
