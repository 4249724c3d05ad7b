"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times: the standalone sweep's batches (2^20 systems per n, capped
at 6 GiB), the Norton Newton batch (2^22 points) and the ragged mixed-size
batch (2^20 systems, binary64 and mixed precision).

The oracle cannot solve millions of systems in a test, so every launch is
checked two ways: (1) on a sample of systems (evenly spaced, plus the first
and the last ones of the batch, which sit in the ragged tail of the last
block) against the oracle, system by system, with the usual bar (pivots and
info bit-identical, x within backward error 10n and forward error
1e-12 kappa; Newton counts identical and states within 1e-10); (2) on every
system by properties that hold at any size (info 0 on these nonsingular
inputs, normwise backward error <= 10n computed on the device)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402
from paper_2609_15217_gb300 import layout as L  # noqa: E402

import bench  # noqa: E402  (sizes and seeds of the benchmark's workloads)

from test_gpu_lupp import check_solution  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture(scope="module")
def h(tl):
    hh = tl.tl_create()
    yield hh
    tl.tl_destroy(hh)


def sample_index(S, count=1500):
    idx = np.unique(np.concatenate([np.linspace(0, S - 1, count).astype(np.int64), np.arange(S - 40, S)]))
    return torch.from_numpy(idx).to(DEV)


@pytest.mark.parametrize("n,variant", [(8, 1), (20, 116), (27, 132), (32, 132), (32, 16)])
def test_sweep_full_size(tl, h, n, variant):
    S = bench.sweep_batch(n)
    A, b, _ = inputs.sweep_systems_torch(n, S, bench.rank_seed(1236, 0) * 1000 + n, DEV)
    ld = L.pad_ld(S)
    dA = L.matrices_to_layout(A, 1, ld)
    db = L.vectors_to_layout(b, 1, ld)
    dx = torch.empty_like(db)
    dp = torch.empty(db.numel(), dtype=torch.int32, device=DEV)
    di = torch.empty(S, dtype=torch.int32, device=DEV)
    assert tl.tl_dispatch_set(h, n, 1, variant, 0) == tl.TL_OK
    try:
        tl.check("gesv", tl.tl_gesv_batched(h, n, dA, None, db, dx, dp, di, 1, ld, S), h)
        torch.cuda.synchronize()
    finally:
        tl.tl_dispatch_set(h, n, 1, 0, 0)
    x = L.vectors_from_layout(dx, S, n, 1, ld)
    piv = L.vectors_from_layout(dp, S, n, 1, ld)
    # every system: info and backward error
    assert int((di != 0).sum()) == 0
    r = b - torch.matmul(A, x[:, :, None])[:, :, 0]
    be = r.abs().amax(dim=1) / (A.abs().sum(dim=2).amax(dim=1) * x.abs().amax(dim=1) * EPS)
    assert float(be.max()) <= 10 * n
    # sampled systems against the oracle
    idx = sample_index(S)
    As, bs = A[idx].cpu().numpy(), b[idx].cpu().numpy()
    x_o, piv_o, info_o, _ = oracle.gesv(As, bs)
    assert np.array_equal(piv[idx].cpu().numpy(), piv_o) and (info_o == 0).all()
    check_solution(As, bs, x[idx].cpu().numpy(), x_o)


def test_newton_full_size(tl, h):
    npts = bench.NEWTON_POINTS
    sig0, deps = inputs.norton_points_torch(npts, bench.rank_seed(1237, 0), DEV)
    fields = torch.cat([sig0.t(), deps.t()], dim=0).contiguous()
    x = torch.empty((7, npts), dtype=torch.float64, device=DEV)
    sig = torch.empty((6, npts), dtype=torch.float64, device=DEV)
    it = torch.empty(npts, dtype=torch.int32, device=DEV)
    st = torch.empty(npts, dtype=torch.int32, device=DEV)
    prm = (200000.0, 0.3, 1e-12, 4.0, 1.0)
    law = tl.make_law(tl.TL_LAW_NORTON, 7, prm)
    tl.check("newton", tl.tl_newton_integrate(h, law, npts, fields, x, sig, it, st, 1e-10, 20), h)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0 and int(it.max()) <= 20
    idx = sample_index(npts, 1000)
    r = oracle.newton_norton(np.array(prm), sig0[idx].cpu().numpy(), deps[idx].cpu().numpy(), rtol=1e-10,
                             max_iter=20)
    ok = r["rmin_ratio"] >= 1e-6
    assert np.array_equal(it[idx].cpu().numpy()[ok], r["iterations"][ok])
    xs = x[:, idx].cpu().numpy().T
    err = np.abs(xs - r["x"]).max(axis=1) / np.abs(r["x"]).max(axis=1)
    assert (err[ok] <= 1e-10).all()


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_full_size(tl, h, prec):
    d = bench.make_ragged_torch(bench.RAGGED_BATCH, bench.rank_seed(1238, 0), DEV, torch, inputs)
    batch = d["batch"]
    x = torch.empty_like(d["b"])
    ipiv = torch.empty(d["b"].numel(), dtype=torch.int32, device=DEV)
    info = torch.empty(batch, dtype=torch.int32, device=DEV)
    ref = torch.full((batch,), -9, dtype=torch.int32, device=DEV)
    tl.check("ragged", tl.tl_lupp_solve_batched(h, batch, d["sizes"], d["a_off"], d["A"], d["b_off"], d["b"], x,
                                                d["b_off"], ipiv, info, prec, ref if prec else None), h)
    torch.cuda.synchronize()
    assert int((info != 0).sum()) == 0
    be, _ = bench.ragged_errors(d, x, torch)
    assert be <= 1.0     # worst normwise backward error in units of n*eps
    for n, (sel, ia, ib) in d["buckets"].items():
        take = sel[:: max(1, sel.numel() // 300)]
        take = torch.cat([take, sel[-5:]])
        rows = torch.searchsorted(sel, take)
        A = d["A"][ia].reshape(-1, n, n).transpose(1, 2)[rows].cpu().numpy()
        bb = d["b"][ib].reshape(-1, n)[rows].cpu().numpy()
        xs = x[ib].reshape(-1, n)[rows].cpu().numpy()
        ps = ipiv[ib].reshape(-1, n)[rows].cpu().numpy()
        if prec == 0 or n <= 20:
            # binary64, or mixed precision on a size routed to binary64 by
            # default (refine count -1)
            x_o, piv_o, info_o, _ = oracle.gesv(A, bb)
            assert np.array_equal(ps, piv_o), n
            check_solution(A, bb, xs, x_o)
            if prec:
                assert (ref[take] == -1).all(), n
        else:
            x_o, piv_o, info_o, steps = oracle.ir_gesv(A, bb)
            assert np.array_equal(ref[take].cpu().numpy(), steps), n
            assert np.array_equal(ps, piv_o), n
            refined = steps >= 0
            assert np.array_equal(xs[refined].view(np.int64), x_o[refined].view(np.int64)), n
