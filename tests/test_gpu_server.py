"""GPU tests of the request server (continuous batching of Newton and solve
requests): every request's results are bit-identical to the same request run
alone through tl_newton_integrate / tl_lupp_solve_batched, whether it shared
its ticks with other requests (batched mode) or ran on its own (plain mode);
admission against a small budget, refusals and timeouts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

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


class Newton:
    def __init__(self, tl, law_id, n, npts, seed):
        self.law = tl.make_law(law_id, n, tuple(oracle.norton_params()) if law_id == tl.TL_LAW_NORTON else ())
        self.n = 7 if law_id == tl.TL_LAW_NORTON else n
        self.norton = law_id == tl.TL_LAW_NORTON
        if self.norton:
            sig0, deps = inputs.norton_points(npts, seed)
            self.fields = np.ascontiguousarray(np.concatenate([sig0.T, deps.T], axis=0))
        else:
            A, c, b = inputs.tanh_points(n, npts, seed)
            Acm = A.transpose(0, 2, 1).reshape(npts, n * n)
            self.fields = np.ascontiguousarray(np.concatenate([Acm.T, c.T, b.T], axis=0))
        self.npts = npts
        self.x = np.full((self.n, npts), -7.0)
        self.aux = np.full((6, npts), -7.0) if self.norton else None
        self.it = np.full(npts, -7, np.int32)
        self.st = np.full(npts, -7, np.int32)

    def request(self, tl):
        return tl.make_request(tl.TL_REQ_NEWTON, self.npts, self.fields, self.x, self.it, self.st, law=self.law,
                               aux=self.aux)

    def alone(self, tl, h):
        d_in = torch.from_numpy(self.fields).to(DEV)
        d_x = torch.empty((self.n, self.npts), dtype=torch.float64, device=DEV)
        d_aux = torch.empty((6, self.npts), dtype=torch.float64, device=DEV) if self.norton else None
        d_it = torch.empty(self.npts, dtype=torch.int32, device=DEV)
        d_st = torch.empty(self.npts, dtype=torch.int32, device=DEV)
        tl.check("newton", tl.tl_newton_integrate(h, self.law, self.npts, d_in, d_x, d_aux, d_it, d_st, 1e-10, 20), h)
        torch.cuda.synchronize()
        return d_x.cpu().numpy(), (d_aux.cpu().numpy() if self.norton else None), d_it.cpu().numpy(), d_st.cpu().numpy()

    def check(self, tl, h):
        x, aux, it, st = self.alone(tl, h)
        assert np.array_equal(self.x.view(np.int64), x.view(np.int64))
        assert np.array_equal(self.it, it) and np.array_equal(self.st, st)
        if self.norton:
            assert np.array_equal(self.aux.view(np.int64), aux.view(np.int64))


class Solve:
    def __init__(self, n, count, seed):
        A, b, _, _ = inputs.sweep_systems(n, count, seed)
        self.n, self.count = n, count
        self.A = np.ascontiguousarray(A.transpose(0, 2, 1).reshape(-1))
        self.b = np.ascontiguousarray(b.reshape(-1))
        self.x = np.full(n * count, -7.0)
        self.piv = np.full(n * count, -7, np.int32)
        self.info = np.full(count, -7, np.int32)

    def request(self, tl):
        return tl.make_request(tl.TL_REQ_SOLVE, self.count, self.A, self.x, self.piv, self.info, n=self.n,
                               rhs=self.b)

    def check(self, tl, h):
        n, c = self.n, self.count
        d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dt)  # noqa: E731
        dn = torch.full((c,), n, dtype=torch.int32, device=DEV)
        da = torch.arange(c, dtype=torch.int64, device=DEV) * n * n
        db = torch.arange(c, dtype=torch.int64, device=DEV) * n
        dA, dbv = d(self.A, torch.float64), d(self.b, torch.float64)
        dx = torch.empty_like(dbv)
        dpiv = torch.empty(n * c, dtype=torch.int32, device=DEV)
        dinfo = torch.empty(c, dtype=torch.int32, device=DEV)
        tl.check("ragged", tl.tl_lupp_solve_batched(h, c, dn, da, dA, db, dbv, dx, db, dpiv, dinfo), h)
        torch.cuda.synchronize()
        assert np.array_equal(self.x.view(np.int64), dx.cpu().numpy().view(np.int64))
        assert np.array_equal(self.piv, dpiv.cpu().numpy()) and np.array_equal(self.info, dinfo.cpu().numpy())


def make_mix(tl, seed):
    g = inputs.rng(seed)
    work = []
    for k in range(18):
        kind = g.integers(0, 6)
        if kind == 0:
            work.append(Newton(tl, tl.TL_LAW_NORTON, 7, int(g.integers(300, 4000)), 1000 * seed + k))
        elif kind <= 4:
            n = [7, 13, 20, 32][kind - 1]
            work.append(Newton(tl, tl.TL_LAW_TANH, n, int(g.integers(100, 1500)), 1000 * seed + k))
        else:
            work.append(Solve(int(g.choice([3, 7, 12, 32])), int(g.integers(50, 1500)), 1000 * seed + k))
    return work


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_results_equal_alone(tl, h, mode):
    cap, slots = (6000, 3) if mode == "batched" else (0, 1)
    st, srv = tl.tl_server_create(h, 1 << 30, slots, cap)
    assert st == tl.TL_OK
    try:
        work = make_mix(tl, 3 if mode == "batched" else 4)
        reqs = [w.request(tl) for w in work]   # keep the descriptors alive
        ids = []
        for r in reqs:
            st, rid = tl.tl_server_submit(srv, r)
            assert st == tl.TL_OK
            ids.append(rid)
        for rid in ids:
            st, rs, lat = tl.tl_server_wait(srv, rid, 120.0)
            assert st == tl.TL_OK and rs == tl.TL_OK and lat > 0
        st, stats = tl.tl_server_stats_get(srv)
        assert stats["completed"] == len(work) and stats["failed"] == 0
        if mode == "batched":
            assert stats["ticks"] < len(work)      # requests shared ticks
        else:
            assert stats["ticks"] == len(work)
    finally:
        assert tl.tl_server_destroy(srv) == tl.TL_OK
    for w in work:
        w.check(tl, h)


def test_budget_refusals_and_timeouts(tl, h):
    # a 4 MiB arena: each ~1 MiB request waits for room, none is lost
    st, srv = tl.tl_server_create(h, 4 << 20, 2, 1 << 20)
    assert st == tl.TL_OK
    try:
        work = [Newton(tl, tl.TL_LAW_NORTON, 7, 4000, 50 + k) for k in range(6)]
        reqs = [w.request(tl) for w in work]
        ids = [tl.tl_server_submit(srv, r)[1] for r in reqs]
        big = Newton(tl, tl.TL_LAW_NORTON, 7, 40000, 60)
        assert tl.tl_server_submit(srv, big.request(tl))[0] == tl.TL_ERR_NO_MEMORY
        bad = tl.make_request(tl.TL_REQ_NEWTON, 10, None, None, None, None, law=tl.make_law(tl.TL_LAW_TANH, 40))
        assert tl.tl_server_submit(srv, bad)[0] == tl.TL_ERR_INVALID_ARG
        bad = tl.make_request(tl.TL_REQ_SOLVE, 10, work[0].fields, work[0].x, work[0].it, work[0].st, n=3)
        assert tl.tl_server_submit(srv, bad)[0] == tl.TL_ERR_INVALID_ARG   # no rhs
        for rid in ids:
            st, rs, _ = tl.tl_server_wait(srv, rid, 120.0)
            assert st == tl.TL_OK and rs == tl.TL_OK
            assert tl.tl_server_test(srv, rid)[0] == tl.TL_ERR_INVALID_ARG   # released
        st, stats = tl.tl_server_stats_get(srv)
        assert stats["arena_high_water"] <= 4 << 20 and stats["completed"] == 6
        # a request queued while admission is paused cannot be done: a zero
        # and a short wait both time out, it stays queued, and it completes
        # once admission resumes
        slow = Newton(tl, tl.TL_LAW_TANH, 13, 1500, 61)    # ~2.5 MiB: fits the arena
        sreq = slow.request(tl)
        assert tl.tl_server_pause(srv, True) == tl.TL_OK
        st, rid = tl.tl_server_submit(srv, sreq)
        assert st == tl.TL_OK
        assert tl.tl_server_wait(srv, rid, 0.0)[0] == tl.TL_ERR_TIMEOUT
        assert tl.tl_server_wait(srv, rid, 0.05)[0] == tl.TL_ERR_TIMEOUT
        assert tl.tl_server_test(srv, rid)[:2] == (tl.TL_OK, 0)
        assert tl.tl_server_pause(srv, False) == tl.TL_OK
        assert tl.tl_server_wait(srv, rid, 120.0)[:2] == (tl.TL_OK, tl.TL_OK)
        # an empty request completes
        empty = tl.make_request(tl.TL_REQ_NEWTON, 0, None, None, None, None, law=tl.make_law(tl.TL_LAW_NORTON, 7,
                                tuple(oracle.norton_params())))
        st, rid = tl.tl_server_submit(srv, empty)
        assert st == tl.TL_OK and tl.tl_server_wait(srv, rid, 60.0)[:2] == (tl.TL_OK, tl.TL_OK)
    finally:
        assert tl.tl_server_destroy(srv) == tl.TL_OK
    for w in work:
        w.check(tl, h)
    slow.check(tl, h)


def test_create_errors(tl, h):
    assert tl.tl_server_create(h, 1 << 10, 2, 100)[0] == tl.TL_ERR_INVALID_ARG
    assert tl.tl_server_create(h, 1 << 24, 0, 100)[0] == tl.TL_ERR_INVALID_ARG
    assert tl.tl_server_create(h, 1 << 24, 2, -1)[0] == tl.TL_ERR_INVALID_ARG


def test_solve_ticks_allocate_no_device_memory(tl, h):
    # every tick takes its ragged-solve workspace from the arena: a second,
    # larger solve tick leaves the device's free memory unchanged
    st, srv = tl.tl_server_create(h, 256 << 20, 2, 1 << 20)
    assert st == tl.TL_OK
    try:
        small, large = Solve(12, 200, 71), Solve(20, 60000, 72)
        st, rid = tl.tl_server_submit(srv, small.request(tl))
        assert st == tl.TL_OK and tl.tl_server_wait(srv, rid, 120.0)[:2] == (tl.TL_OK, tl.TL_OK)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        lreq = large.request(tl)
        st, rid = tl.tl_server_submit(srv, lreq)
        assert st == tl.TL_OK and tl.tl_server_wait(srv, rid, 120.0)[:2] == (tl.TL_OK, tl.TL_OK)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        st, stats = tl.tl_server_stats_get(srv)
        assert stats["kernel_busy_s"] > 0 and stats["host_enqueue_s"] > 0
    finally:
        assert tl.tl_server_destroy(srv) == tl.TL_OK
    small.check(tl, h)
    large.check(tl, h)


def test_pause_then_destroy_finishes_queued(tl, h):
    st, srv = tl.tl_server_create(h, 64 << 20, 1, 1 << 16)
    assert st == tl.TL_OK
    w = Solve(7, 500, 73)
    req = w.request(tl)
    assert tl.tl_server_pause(srv, True) == tl.TL_OK
    st, rid = tl.tl_server_submit(srv, req)
    assert st == tl.TL_OK
    assert tl.tl_server_destroy(srv) == tl.TL_OK     # resumes admission, drains the queue
    w.check(tl, h)
