"""GPU parity of tl_lupp_solve_batched (ragged batches: every system has its
own n and its own place in memory) against the oracle, system by system.
Same bar as the fixed-size path: pivots and info bit-exact, x within
backward error 10 n and 1e-12 kappa of the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
EPS = np.finfo(np.float64).eps
RAGGED_N = [6, 7, 12, 13, 19, 25, 32]
RAGGED_W = [0.2, 0.25, 0.15, 0.15, 0.1, 0.1, 0.05]


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture(scope="module")
def h(tl):
    hh = tl.tl_create()
    yield hh
    tl.tl_destroy(hh)


def make_ragged(sizes, seed, gap=3):
    """Pack systems of the given sizes at shuffled, gapped offsets."""
    g = inputs.rng(seed)
    batch = len(sizes)
    systems = {}
    for n in sorted(set(int(v) for v in sizes if 1 <= v <= 32)):
        idx = np.nonzero(sizes == n)[0]
        A, b, _, _ = inputs.sweep_systems(n, len(idx), seed * 100 + n)
        systems[n] = (idx, A, b)
    order = g.permutation(batch)
    a_off = np.zeros(batch, np.int64)
    b_off = np.zeros(batch, np.int64)
    p_off = np.zeros(batch, np.int64)
    pa = pb = pp = 0
    for s in order:
        n = max(int(sizes[s]), 1)
        a_off[s], b_off[s], p_off[s] = pa, pb, pp
        pa += n * n + int(g.integers(0, gap))
        pb += n + int(g.integers(0, gap))
        pp += n + int(g.integers(0, gap))
    Abuf = np.full(pa + 1, 9.0)
    bbuf = np.full(pb + 1, 9.0)
    for n, (idx, A, b) in systems.items():
        for q, s in enumerate(idx):
            Abuf[a_off[s]:a_off[s] + n * n] = A[q].T.reshape(-1)   # column-major
            bbuf[b_off[s]:b_off[s] + n] = b[q]
    return systems, a_off, b_off, p_off, Abuf, bbuf, pp + 1


def run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, mode=None):
    batch = len(sizes)
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dt)  # noqa: E731
    dn = d(sizes.astype(np.int32), torch.int32)
    da, db, dp = d(a_off, torch.int64), d(b_off, torch.int64), d(p_off, torch.int64)
    dA, dbv = d(Abuf, torch.float64), d(bbuf, torch.float64)
    dx = torch.full_like(dbv, -5.0)
    dpiv = torch.full((npiv,), -5, dtype=torch.int32, device=DEV)
    dinfo = torch.full((batch,), -5, dtype=torch.int32, device=DEV)
    if mode is not None:
        assert tl.tl_ragged_set_mode(h, mode) == tl.TL_OK
    try:
        st = tl.tl_lupp_solve_batched(h, batch, dn, da, dA, db, dbv, dx, dp, dpiv, dinfo)
    finally:
        tl.tl_ragged_set_mode(h, tl.TL_RAGGED_PERSISTENT)
    tl.check("tl_lupp_solve_batched", st, h)
    torch.cuda.synchronize()
    return dx.cpu().numpy(), dpiv.cpu().numpy(), dinfo.cpu().numpy()


def check_ragged(sizes, systems, b_off, p_off, x, piv, info):
    for n, (idx, A, b) in systems.items():
        xo, pivo, infoo, _ = oracle.gesv(A, b)
        xg = np.stack([x[b_off[s]:b_off[s] + n] for s in idx])
        pg = np.stack([piv[p_off[s]:p_off[s] + n] for s in idx])
        assert np.array_equal(info[idx], infoo), n
        assert np.array_equal(pg, pivo), n
        r = np.einsum("sij,sj->si", A.astype(np.longdouble), xg.astype(np.longdouble)) - b
        be = np.abs(r).max(axis=1).astype(float) / (np.abs(A).sum(axis=2).max(axis=1) * np.abs(xg).max(axis=1) * EPS)
        assert (be <= 10 * n).all(), (n, be.max())
        kappa = np.linalg.cond(A)
        fe = np.abs(xg - xo).max(axis=1) / np.abs(xo).max(axis=1)
        assert (fe <= 1e-12 * kappa).all(), n


def test_ragged_mix_of_the_benchmark(tl, h):
    g = inputs.rng(77)
    sizes = g.choice(RAGGED_N, size=6000, p=RAGGED_W).astype(np.int64)
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 5)
    x, piv, info = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    check_ragged(sizes, systems, b_off, p_off, x, piv, info)


def test_ragged_every_n_and_invalid_sizes(tl, h):
    g = inputs.rng(78)
    sizes = g.integers(1, 33, size=3000).astype(np.int64)
    bad = g.choice(3000, size=20, replace=False)
    sizes[bad[:10]] = 0
    sizes[bad[10:]] = 33
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 6)
    x, piv, info = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
    assert (info[bad] == -2).all()
    for s in bad:  # skipped systems leave their outputs untouched
        assert x[b_off[s]] == -5.0 and piv[p_off[s]] == -5
    check_ragged(sizes, systems, b_off, p_off, x, piv, info)


def test_ragged_repeated_calls_and_growth(tl, h):
    for k, batch in enumerate((17, 5000, 40000, 3)):
        g = inputs.rng(80 + k)
        sizes = g.choice(RAGGED_N, size=batch, p=RAGGED_W).astype(np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 90 + k)
        x, piv, info = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        check_ragged(sizes, systems, b_off, p_off, x, piv, info)


def test_ragged_argument_errors(tl, h):
    d = torch.zeros(64, dtype=torch.float64, device=DEV)
    i32 = torch.zeros(64, dtype=torch.int32, device=DEV)
    i64 = torch.zeros(64, dtype=torch.int64, device=DEV)
    assert tl.tl_lupp_solve_batched(h, -1, i32, i64, d, i64, d, d, i64, i32, i32) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_lupp_solve_batched(h, 0, None, None, None, None, None, None, None, None, None) == tl.TL_OK
    assert tl.tl_lupp_solve_batched(h, 4, i32, i64, None, i64, d, d, i64, i32, i32) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 5
    assert tl.tl_lupp_solve_batched(h, 4, i32, i64, d, i64, d, d, i64, i32, i32, prec=7) == tl.TL_ERR_INVALID_ARG


def plant_special(systems, Abuf, bbuf, a_off):
    """A zero column and a NaN entry in a few systems of each size (the
    oracle copy is updated too)."""
    for n, (idx, A, b) in systems.items():
        for q, kind in ((0, "zero"), (1, "nan")):
            if q >= len(idx) or n < 2:
                continue
            s = idx[q]
            if kind == "zero":
                A[q, :, n // 2] = 0.0
            else:
                A[q, n - 1, 0] = np.nan
            Abuf[a_off[s]:a_off[s] + n * n] = A[q].T.reshape(-1)


def test_persistent_launch_equals_per_size_launches(tl, h):
    # one persistent launch over every size class against one launch per
    # size: identical x, pivots and info, bit for bit
    g = inputs.rng(84)
    sizes = g.integers(1, 33, size=4000).astype(np.int64)
    sizes[g.choice(4000, size=8, replace=False)] = 0
    systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 85)
    plant_special(systems, Abuf, bbuf, a_off)
    xp, pp, ip = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, tl.TL_RAGGED_PERSISTENT)
    xs, ps, is_ = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv, tl.TL_RAGGED_PER_SIZE)
    assert np.array_equal(ip, is_) and np.array_equal(pp, ps)
    assert np.array_equal(xp.view(np.int64), xs.view(np.int64))
    for n, (idx, A, b) in systems.items():
        _, pivo, infoo, _ = oracle.gesv(A, b)
        assert np.array_equal(ip[idx], infoo), n
        assert np.array_equal(np.stack([pp[p_off[s]:p_off[s] + n] for s in idx]), pivo), n


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_persistent_launch_every_lane_count(tl, h, lanes):
    # the ragged dispatch table sets the lanes per system of each size in
    # the single launch (one thread in registers only up to n = 7)
    top = 7 if lanes == 1 else 32
    for n in range(1, top + 1):
        assert tl.tl_ragged_dispatch_set(h, n, lanes, -1) == tl.TL_OK
        assert tl.tl_ragged_dispatch_get(h, n)[1] == lanes
    try:
        g = inputs.rng(86 + lanes)
        sizes = g.integers(1, 33, size=1500).astype(np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 87 + lanes)
        plant_special(systems, Abuf, bbuf, a_off)
        x, piv, info = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        for n, (idx, A, b) in systems.items():
            _, pivo, infoo, _ = oracle.gesv(A, b)
            assert np.array_equal(info[idx], infoo), n
            assert np.array_equal(np.stack([piv[p_off[s]:p_off[s] + n] for s in idx]), pivo), n
        ok = {n: (idx[info[idx] == 0], A[info[idx] == 0], b[info[idx] == 0]) for n, (idx, A, b) in systems.items()}
        check_ragged(sizes, ok, b_off, p_off, x, piv, info)
    finally:
        for n in range(1, 33):
            tl.tl_ragged_dispatch_set(h, n, 0, -1)


def test_ragged_one_size_only(tl, h):
    for n in (1, 5, 32):
        sizes = np.full(700, n, np.int64)
        systems, a_off, b_off, p_off, Abuf, bbuf, npiv = make_ragged(sizes, 200 + n)
        x, piv, info = run_ragged(tl, h, sizes, a_off, b_off, p_off, Abuf, bbuf, npiv)
        check_ragged(sizes, systems, b_off, p_off, x, piv, info)
