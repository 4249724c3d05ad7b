"""The bounds-checked build of the library (libtinylu_checked.so, compiled with
-DTL_CHECK_BOUNDS): every shared-memory index of the element-walk
elimination and of the loads into shared memory is checked against its
system's block, and a violation is counted instead of performed.  This
stands in for a memory checker, which cannot run on the shared GPUs here.
On small cases of every shared-memory variant, both layouts, planted zero
columns and non-finite systems, and the single persistent ragged launch,
the checked library must count no violation and give results identical to
the normal library's."""
import ctypes as C
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_15217_gb300 import inputs  # noqa: E402
from paper_2609_15217_gb300 import layout as L  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def tl():
    from paper_2609_15217_gb300 import tinylu
    return tinylu


@pytest.fixture(scope="module")
def chk(tl):
    """ctypes binding of the checked library (same C ABI)."""
    lib = C.CDLL(os.path.join(os.path.dirname(tl.LIB_PATH), "libtinylu_checked.so"))
    for name, (args, res) in tl._SIGS.items():
        try:
            f = getattr(lib, name)
        except AttributeError:
            continue
        f.argtypes, f.restype = args, res
    lib.tl_check_bounds_violations.argtypes = [C.POINTER(C.c_ulonglong)]
    lib.tl_check_bounds_violations.restype = C.c_int
    return lib


@pytest.fixture(scope="module")
def handles(tl, chk):
    h = tl.tl_create()
    hc = C.c_void_p()
    assert chk.tl_create(C.byref(hc)) == 0
    yield h, hc.value
    tl.tl_destroy(h)
    chk.tl_destroy(hc.value)


def violations(chk):
    v = C.c_ulonglong(0)
    assert chk.tl_check_bounds_violations(C.byref(v)) == 0
    return v.value


def test_normal_library_has_no_checks(tl):
    v = C.c_ulonglong(7)
    assert tl.library().tl_check_bounds_violations(C.byref(v)) == tl.TL_ERR_UNSUPPORTED


def gesv_both(tl, chk, h, hc, n, variant, layout, A, b):
    batch = A.shape[0]
    ld = L.pad_ld(batch)
    dA = L.matrices_to_layout(torch.from_numpy(A).to(DEV), layout, ld)
    db = L.vectors_to_layout(torch.from_numpy(b).to(DEV), layout, ld)
    out = []
    for lib, hh in ((tl.library(), h), (chk, hc)):
        assert lib.tl_dispatch_set(hh, n, layout, variant, 0) == 0
        dx = torch.full_like(db, -3.0)
        dp = torch.full((db.numel(),), -3, dtype=torch.int32, device=DEV)
        di = torch.full((batch,), -3, dtype=torch.int32, device=DEV)
        st = lib.tl_gesv_batched(hh, n, dA.data_ptr(), None, db.data_ptr(), dx.data_ptr(), dp.data_ptr(),
                                 di.data_ptr(), layout, ld, batch, torch.cuda.current_stream().cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        lib.tl_dispatch_set(hh, n, layout, 0, 0)
        out.append((dx.cpu().numpy(), dp.cpu().numpy(), di.cpu().numpy()))
    return out


@pytest.mark.parametrize("variant", [102, 104, 108, 116, 132, 202, 204, 208])
def test_shared_memory_variants_within_bounds(tl, chk, handles, variant):
    h, hc = handles
    for n in (2, 5, 9, 13, 20, 27, 32):
        A, b, _, _ = inputs.sweep_systems(n, 97, 4100 + n)
        A[4, :, n // 2] = 0.0        # a zero pivot
        A[7, 0, n - 1] = np.inf      # a non-finite system
        for layout in (0, 1):
            (x0, p0, i0), (x1, p1, i1) = gesv_both(tl, chk, h, hc, n, variant, layout, A, b)
            assert np.array_equal(i0, i1) and np.array_equal(p0, p1), (n, layout)
            assert np.array_equal(x0.view(np.int64), x1.view(np.int64)), (n, layout)
    assert violations(chk) == 0


def test_persistent_ragged_launch_within_bounds(tl, chk, handles):
    h, hc = handles
    g = inputs.rng(4200)
    batch = 3000
    sizes = g.integers(1, 33, size=batch).astype(np.int32)
    nn = sizes.astype(np.int64) ** 2
    a_off = np.cumsum(nn) - nn
    b_off = np.cumsum(sizes.astype(np.int64)) - sizes
    Abuf = g.uniform(-1, 1, int(nn.sum()))
    bbuf = g.uniform(-1, 1, int(sizes.sum()))
    Abuf[a_off[5]:a_off[5] + nn[5]] = 0.0    # a singular system
    Abuf[a_off[9]] = np.nan                   # a non-finite one
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)  # noqa: E731
    dn, da, db_off, dA, dbv = d(sizes), d(a_off), d(b_off), d(Abuf), d(bbuf)
    out = []
    for lib, hh in ((tl.library(), h), (chk, hc)):
        dx = torch.full_like(dbv, -3.0)
        dp = torch.full((int(sizes.sum()),), -3, dtype=torch.int32, device=DEV)
        di = torch.full((batch,), -3, dtype=torch.int32, device=DEV)
        st = lib.tl_lupp_solve_batched(hh, batch, dn.data_ptr(), da.data_ptr(), dA.data_ptr(), db_off.data_ptr(),
                                       dbv.data_ptr(), dx.data_ptr(), db_off.data_ptr(), dp.data_ptr(),
                                       di.data_ptr(), 0, None, torch.cuda.current_stream().cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        out.append((dx.cpu().numpy(), dp.cpu().numpy(), di.cpu().numpy()))
    (x0, p0, i0), (x1, p1, i1) = out
    assert np.array_equal(i0, i1) and np.array_equal(p0, p1)
    assert np.array_equal(x0.view(np.int64), x1.view(np.int64))
    assert i0[5] > 0 and i0[9] == -1
    assert violations(chk) == 0
