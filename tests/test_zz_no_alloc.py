"""tl_lupp_solve_batched_noalloc: the ragged solve for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the allocating entry point,
tl_lupp_solve_batched, on two calls in a row: identical pivots and info,
solutions within the same bounds the other parity tests use (backward error
10 n, forward error 1e-12 kappa), no change of free device memory across a
call, and a clear rejection of batches above the scratch size.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_15217_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
EPS = np.finfo(np.float64).eps
SIZES = [6, 7, 12, 13, 19, 25, 32]
WEIGHTS = [0.2, 0.25, 0.15, 0.15, 0.1, 0.1, 0.05]


def _batch(seed, batch):
    """A ragged batch at packed per-system offsets, as device tensors."""
    g = inputs.rng(seed)
    sizes = g.choice(SIZES, size=batch, p=WEIGHTS).astype(np.int64)
    a_off = np.zeros(batch, np.int64)
    v_off = np.zeros(batch, np.int64)
    a_off[1:] = np.cumsum(sizes * sizes)[:-1]
    v_off[1:] = np.cumsum(sizes)[:-1]
    Abuf = np.empty(int((sizes * sizes).sum()))
    bbuf = np.empty(int(sizes.sum()))
    mats = {}
    for n in SIZES:
        idx = np.nonzero(sizes == n)[0]
        A, b, _, _ = inputs.sweep_systems(n, len(idx), seed * 100 + n)
        mats[n] = (idx, A, b)
        for q, s in enumerate(idx):
            Abuf[a_off[s]:a_off[s] + n * n] = A[q].T.reshape(-1)
            bbuf[v_off[s]:v_off[s] + n] = b[q]
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dt)  # noqa: E731
    dev = dict(n=t(sizes.astype(np.int32), torch.int32), a_off=t(a_off, torch.int64), A=t(Abuf, torch.float64),
               v_off=t(v_off, torch.int64), b=t(bbuf, torch.float64))
    return sizes, v_off, mats, dev


def _outputs(batch, nvec):
    return (torch.full((nvec,), -3.0, dtype=torch.float64, device=DEV),
            torch.full((nvec,), -3, dtype=torch.int32, device=DEV),
            torch.full((batch,), -3, dtype=torch.int32, device=DEV))


def _check_close(sizes, v_off, mats, x_ref, x_new):
    for n, (idx, A, b) in mats.items():
        xr = np.stack([x_ref[v_off[s]:v_off[s] + n] for s in idx])
        xn = np.stack([x_new[v_off[s]:v_off[s] + n] for s in idx])
        r = np.einsum("sij,sj->si", A.astype(np.longdouble), xn.astype(np.longdouble)) - b
        be = np.abs(r).max(axis=1).astype(float) / (np.abs(A).sum(axis=2).max(axis=1) * np.abs(xn).max(axis=1) * EPS)
        assert (be <= 10 * n).all()
        fe = np.abs(xn - xr).max(axis=1) / np.abs(xr).max(axis=1)
        assert (fe <= 1e-12 * np.linalg.cond(A)).all()


def test_noalloc_matches_allocating_entry_two_calls():
    from paper_2609_15217_gb300 import tinylu as tl
    h = tl.tl_create()
    try:
        first = True
        for seed, batch in ((501, 7000), (502, 1500)):
            sizes, v_off, mats, d = _batch(seed, batch)
            nvec = int(sizes.sum())
            x_ref, p_ref, i_ref = _outputs(batch, nvec)
            x_new, p_new, i_new = _outputs(batch, nvec)
            tl.check("tl_lupp_solve_batched", tl.tl_lupp_solve_batched(
                h, batch, d["n"], d["a_off"], d["A"], d["v_off"], d["b"], x_ref, d["v_off"], p_ref, i_ref), h)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            tl.check("tl_lupp_solve_batched_noalloc", tl.tl_lupp_solve_batched_noalloc(
                h, batch, d["n"], d["a_off"], d["A"], d["v_off"], d["b"], x_new, d["v_off"], p_new, i_new), h)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            if not first:  # the first call on the device looks up the scratch address
                assert free_after == free_before, "the no-allocation entry point changed free device memory"
            first = False
            assert np.array_equal(i_new.cpu().numpy(), i_ref.cpu().numpy())
            assert np.array_equal(p_new.cpu().numpy(), p_ref.cpu().numpy())
            assert (i_new.cpu().numpy() == 0).all()
            _check_close(sizes, v_off, mats, x_ref.cpu().numpy(), x_new.cpu().numpy())
    finally:
        tl.tl_destroy(h)


def test_noalloc_rejects_batches_above_the_scratch_size():
    from paper_2609_15217_gb300 import tinylu as tl
    h = tl.tl_create()
    try:
        d = torch.zeros(8, dtype=torch.float64, device=DEV)
        i32 = torch.zeros(8, dtype=torch.int32, device=DEV)
        i64 = torch.zeros(8, dtype=torch.int64, device=DEV)
        big = tl.TL_NOALLOC_MAX_BATCH + 1
        st = tl.tl_lupp_solve_batched_noalloc(h, big, i32, i64, d, i64, d, d, i64, i32, i32)
        assert st == tl.TL_ERR_INVALID_ARG and tl.tl_last_bad_arg(h) == 2
        assert tl.tl_lupp_solve_batched_noalloc(h, 0, None, None, None, None, None, None, None, None, None) == tl.TL_OK
    finally:
        tl.tl_destroy(h)
