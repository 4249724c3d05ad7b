"""GPU parity of the mixed-precision ragged solve (tl_lupp_solve_batched
with TL_PREC_FP32_IR: binary32 LUpp factor, binary64 iterative refinement,
binary64 LUpp fallback) against the oracle's ir_gesv, system by system.

Bar: the refinement count (or -1 for the binary64 fallback), pivots and info
identical for every system; x bit-identical for every refined system (each
operation of the scheme is one IEEE round-to-nearest operation in a fixed
order on both sides); fallback systems meet the binary64 bar (pivots and
info exact, backward error <= 10 n, forward error <= 1e-12 kappa).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

from test_gpu_ragged import RAGGED_N, RAGGED_W, make_ragged  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture(scope="module")
def h(tl):
    # every size refines (the default routes n <= 20 to binary64; see
    # test_default_route_to_binary64)
    hh = tl.tl_create()
    for n in range(1, 33):
        assert tl.tl_ragged_dispatch_set(hh, n, 0, 0) == tl.TL_OK
    yield hh
    tl.tl_destroy(hh)


def run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, prec=1):
    batch = len(sizes)
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dt)  # noqa: E731
    dn = d(sizes.astype(np.int32), torch.int32)
    da, db, dp = d(a_off, torch.int64), d(b_off, torch.int64), d(p_off, torch.int64)
    dA, dbv = d(Abuf, torch.float64), d(bbuf, torch.float64)
    dx = torch.full_like(dbv, -5.0)
    dpiv = torch.full((npiv,), -5, dtype=torch.int32, device=DEV)
    dinfo = torch.full((batch,), -5, dtype=torch.int32, device=DEV)
    dref = torch.full((batch,), -9, dtype=torch.int32, device=DEV)
    st = tl.tl_lupp_solve_batched(h, batch, dn, da, dA, db, dbv, dx, dp, dpiv, dinfo, prec=prec, refine_steps=dref)
    tl.check("tl_lupp_solve_batched", st, h)
    torch.cuda.synchronize()
    return dx.cpu().numpy(), dpiv.cpu().numpy(), dinfo.cpu().numpy(), dref.cpu().numpy()


def check_ir(systems, b_off, p_off, x, piv, info, ref):
    stats = {}
    for n, (idx, A, b) in systems.items():
        xo, pivo, infoo, steps = oracle.ir_gesv(A, b)
        xg = np.stack([x[b_off[s]:b_off[s] + n] for s in idx])
        pg = np.stack([piv[p_off[s]:p_off[s] + n] for s in idx])
        assert np.array_equal(ref[idx], steps), (n, np.nonzero(ref[idx] != steps)[0][:5])
        assert np.array_equal(info[idx], infoo), n
        assert np.array_equal(pg, pivo), n
        refined = steps >= 0
        assert np.array_equal(xg[refined].view(np.int64), xo[refined].view(np.int64)), n
        fb = ~refined & (infoo == 0)
        if fb.any():
            Af, xf = A[fb], xg[fb]
            r = np.einsum("sij,sj->si", Af.astype(np.longdouble), xf.astype(np.longdouble)) - b[fb]
            be = np.abs(r).max(axis=1).astype(float) / (np.abs(Af).sum(axis=2).max(axis=1) * np.abs(xf).max(axis=1) * EPS)
            assert (be <= 10 * n).all(), (n, be.max())
            fe = np.abs(xf - xo[fb]).max(axis=1) / np.abs(xo[fb]).max(axis=1)
            assert (fe <= 1e-12 * np.linalg.cond(Af)).all(), n
        bad = infoo != 0
        assert np.isnan(xg[bad]).all()
        stats[n] = np.bincount(steps + 1, minlength=5).tolist()
    return stats


def test_ir_mix_of_the_benchmark(tl, h):
    g = inputs.rng(177)
    sizes = g.choice(RAGGED_N, size=6000, p=RAGGED_W).astype(np.int64)
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 15)
    x, piv, info, ref = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    stats = check_ir(systems, b_off, p_off, x, piv, info, ref)
    # both paths are exercised at every size
    for n, hist in stats.items():
        assert hist[0] > 0 and sum(hist[1:]) > 0, (n, hist)


def test_ir_every_n_ragged_tails_and_invalid_sizes(tl, h):
    g = inputs.rng(178)
    sizes = g.integers(1, 33, size=3000).astype(np.int64)
    bad = g.choice(3000, size=20, replace=False)
    sizes[bad[:10]] = 0
    sizes[bad[10:]] = 33
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 16)
    x, piv, info, ref = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    assert (info[bad] == -2).all() and (ref[bad] == -1).all()
    for s in bad:
        assert x[b_off[s]] == -5.0 and piv[p_off[s]] == -5
    check_ir(systems, b_off, p_off, x, piv, info, ref)


def test_ir_special_systems(tl, h):
    """Out-of-range entries, NaN, a zero column, b = 0 and exactly
    representable systems, all in one call."""
    n = 12
    sizes = np.full(40, n, np.int64)
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 17)
    idx, A, b = systems[n]
    pos = {s: q for q, s in enumerate(idx)}
    edits = {0: (1, 1, 1e39), 1: (2, 3, 1e-39), 2: (0, 5, np.nan)}
    for s, (i, j, v) in edits.items():
        A[pos[s], i, j] = v
    A[pos[3], :, 4] = 0.0
    b[pos[4]] = 0.0
    A[pos[5]] = np.eye(n) * 2.0
    b[pos[5]] = np.arange(n, dtype=float)
    for s in range(6):
        q = pos[s]
        Abuf[a_off[s]:a_off[s] + n * n] = A[q].T.reshape(-1)
        bbuf[b_off[s]:b_off[s] + n] = b[q]
    x, piv, info, ref = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    check_ir(systems, b_off, p_off, x, piv, info, ref)
    assert (ref[:4] == -1).all() and info[2] == -1 and info[3] == 5
    assert ref[4] == 0 and ref[5] == 0
    assert np.array_equal(x[b_off[5]:b_off[5] + n], np.arange(n) / 2.0)


def test_ir_repeated_calls_and_binary64_mode(tl, h):
    for k, batch in enumerate((9, 4000, 31)):
        g = inputs.rng(280 + k)
        sizes = g.choice(RAGGED_N, size=batch, p=RAGGED_W).astype(np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 290 + k)
        x, piv, info, ref = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        check_ir(systems, b_off, p_off, x, piv, info, ref)
        # TL_PREC_FP64 leaves refine_steps alone
        _, _, _, ref64 = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, prec=0)
        assert (ref64 == -9).all()


def _special(systems, a_off, b_off, Abuf, bbuf, n):
    """Plant the special systems of test_ir_special_systems at size n."""
    idx, A, b = systems[n]
    pos = {s: q for q, s in enumerate(idx)}
    edits = {0: (1, 1, 1e39), 1: (n - 1, 0, 1e-39), 2: (0, n - 1, np.nan)}
    for s, (i, j, v) in edits.items():
        A[pos[s], i, j] = v
    A[pos[3], :, n // 2] = 0.0
    b[pos[4]] = 0.0
    A[pos[5]] = np.eye(n) * 2.0
    b[pos[5]] = np.arange(n, dtype=float)
    for s in range(6):
        q = pos[s]
        Abuf[a_off[s]:a_off[s] + n * n] = A[q].T.reshape(-1)
        bbuf[b_off[s]:b_off[s] + n] = b[q]


IR_VARIANT_CASES = ([(n, 132) for n in (2, 3, 5, 9, 10, 11, 16, 17, 20, 24, 25, 28, 31, 32)]
                    + [(n, 8) for n in (17, 20, 24)] + [(n, 16) for n in (25, 28, 32)])


@pytest.mark.parametrize("n,variant", IR_VARIANT_CASES)
def test_ir_each_kernel_with_special_systems(tl, h, n, variant):
    """Every mixed-precision kernel (the shared-memory warp kernel at every
    kind of n, the register group kernels at the sizes where they are not the
    default) on one size, with the special systems planted in the batch and
    a batch that is not a multiple of the warps per block."""
    sizes = np.full(333, n, np.int64)
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 400 + n)
    _special(systems, a_off, b_off, Abuf, bbuf, n)
    assert tl.tl_dispatch_set(h, n, tl.TL_LAYOUT_PER_SYSTEM, variant, 0) == tl.TL_OK
    try:
        x, piv, info, ref = run_ir(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    finally:
        tl.tl_dispatch_set(h, n, tl.TL_LAYOUT_PER_SYSTEM, 0, 0)
    stats = check_ir(systems, b_off, p_off, x, piv, info, ref)
    assert (ref[:4] == -1).all() and info[2] == -1 and info[3] == n // 2 + 1
    assert ref[4] == 0 and ref[5] == 0
    assert np.array_equal(x[b_off[5]:b_off[5] + n], np.arange(n) / 2.0)
    assert stats[n][0] >= 4 and sum(stats[n][1:]) > 200


def test_default_route_to_binary64(tl):
    # default routing: sizes up to 20 are solved in binary64 directly
    # (refine_steps -1, results bit-identical to TL_PREC_FP64), larger
    # sizes refine exactly as the oracle's scheme
    hd = tl.tl_create()
    try:
        for n in (6, 20, 21, 32):
            st, lanes, refines = tl.tl_ragged_dispatch_get(hd, n)
            assert st == tl.TL_OK and refines == (1 if n >= 21 else 0) and lanes in (1, 2, 4, 8, 16, 32)
        g = inputs.rng(190)
        sizes = g.choice([6, 13, 20, 21, 25, 32], size=2500).astype(np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 191)
        x, piv, info, ref = run_ir(tl, hd, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        x64, piv64, info64, _ = run_ir(tl, hd, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, prec=0)
        small = sizes <= 20
        assert (ref[small] == -1).all()
        for n, (idx, A, b) in systems.items():
            if n <= 20:
                for s in idx:
                    assert np.array_equal(x[b_off[s]:b_off[s] + n].view(np.int64), x64[b_off[s]:b_off[s] + n].view(np.int64))
                    assert np.array_equal(piv[p_off[s]:p_off[s] + n], piv64[p_off[s]:p_off[s] + n])
                assert np.array_equal(info[idx], info64[idx])
        big = {n: v for n, v in systems.items() if n >= 21}
        check_ir(big, b_off, p_off, x, piv, info, ref)
        # a size can be routed either way explicitly
        assert tl.tl_ragged_dispatch_set(hd, 6, 0, 0) == tl.TL_OK and tl.tl_ragged_dispatch_get(hd, 6)[2] == 1
        assert tl.tl_ragged_dispatch_set(hd, 25, 0, 1) == tl.TL_OK and tl.tl_ragged_dispatch_get(hd, 25)[2] == 0
        assert tl.tl_ragged_dispatch_set(hd, 25, 3, -1) == tl.TL_ERR_INVALID_ARG
        assert tl.tl_ragged_dispatch_set(hd, 8, 1, -1) == tl.TL_ERR_INVALID_ARG   # one thread only up to n = 7
    finally:
        tl.tl_destroy(hd)


def test_ragged_autotune_table(tl):
    import json
    import os
    import tempfile
    hd = tl.tl_create()
    try:
        path = os.path.join(tempfile.mkdtemp(), "ragged.json")
        assert tl.tl_autotune_ragged(hd, 11, 13, path) == tl.TL_OK
        entries = json.load(open(path))["entries"]
        assert [e["n"] for e in entries] == [11, 12, 13]
        for e in entries:
            st, lanes, refines = tl.tl_ragged_dispatch_get(hd, e["n"])
            assert lanes == e["lanes"] and refines == e["mixed_refines"]
            assert e["ms_fp64"] > 0 and e["ms_mixed"] > 0
            # the refinement kernel: the 4-lane register kernel or the warp kernel
            assert e["ir_variant"] in (4, 132)
        # tuned handle still matches the oracle
        g = inputs.rng(192)
        sizes = g.choice([11, 12, 13], size=900).astype(np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 193)
        x, piv, info, ref = run_ir(tl, hd, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, prec=0)
        for n, (idx, A, b) in systems.items():
            _, pivo, infoo, _ = oracle.gesv(A, b)
            assert np.array_equal(np.stack([piv[p_off[s]:p_off[s] + n] for s in idx]), pivo)
            assert np.array_equal(info[idx], infoo)
        # the tuned refinement kernels, every size refining, against the
        # oracle's scheme
        for n in (11, 12, 13):
            assert tl.tl_ragged_dispatch_set(hd, n, 0, 0) == tl.TL_OK
        x, piv, info, ref = run_ir(tl, hd, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        check_ir(systems, b_off, p_off, x, piv, info, ref)
    finally:
        tl.tl_destroy(hd)
