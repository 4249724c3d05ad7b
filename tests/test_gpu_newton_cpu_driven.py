"""GPU parity of the batched, CPU-driven Newton loop
(tl_newton_integrate_cpu_driven, Algorithm 1): per iteration one assembly
kernel, one tl_gesv_batched over every point, one update kernel and a
device-to-host convergence count.

Bar: against the oracle, the same as the fused kernel (identical iteration
counts and status away from flagged threshold ties, states within 1e-10
relative); against the fused kernel (Algorithm 2) with the default dispatch,
bit-identical states, stresses, iteration counts and status, because both
run the same law code and the same one-thread LUpp arithmetic per point.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2609_15217_gb300 import inputs  # noqa: E402

from test_gpu_newton import compare_states, gpu_norton  # noqa: E402

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


def gpu_norton_cd(tl, h, prm, sig0, deps, rtol=1e-10, max_iter=20, want_sig=True):
    npts = sig0.shape[0]
    fields = np.ascontiguousarray(np.concatenate([sig0.T, deps.T], axis=0))
    d_in = torch.from_numpy(fields).to(DEV)
    d_x = torch.full((7, npts), -7.0, dtype=torch.float64, device=DEV)
    d_sig = torch.full((6, npts), -7.0, dtype=torch.float64, device=DEV) if want_sig else None
    d_it = torch.full((npts,), -7, dtype=torch.int32, device=DEV)
    d_st = torch.full((npts,), -7, dtype=torch.int32, device=DEV)
    law = tl.make_law(tl.TL_LAW_NORTON, 7, prm)
    st = tl.tl_newton_integrate_cpu_driven(h, law, npts, d_in, d_x, d_sig, d_it, d_st, rtol, max_iter)
    tl.check("tl_newton_integrate_cpu_driven", st, h)
    torch.cuda.synchronize()
    return (d_x.cpu().numpy().T, d_it.cpu().numpy(), d_st.cpu().numpy(),
            d_sig.cpu().numpy().T if want_sig else None)


@pytest.mark.parametrize("npts", [1, 33, 20000 + 37])
def test_cpu_driven_matches_oracle_and_fused(tl, h, npts):
    prm = oracle.norton_params()
    sig0, deps = inputs.norton_points(npts, inputs.config_seed(3) + 5 * npts)
    r = oracle.newton_norton(prm, sig0, deps, rtol=1e-10, max_iter=20)
    x_c, it_c, st_c, sig_c = gpu_norton_cd(tl, h, prm, sig0, deps)
    ok = r["rmin_ratio"] >= 1e-6
    assert np.array_equal(it_c[ok], r["iterations"][ok])
    assert np.array_equal(st_c[ok], r["status"][ok])
    compare_states(x_c[ok], r["x"][ok])
    compare_states(sig_c[ok], r["sig"][ok])
    x_f, it_f, st_f, sig_f = gpu_norton(tl, h, prm, sig0, deps)
    assert np.array_equal(it_c, it_f) and np.array_equal(st_c, st_f)
    assert np.array_equal(x_c.view(np.int64), x_f.view(np.int64))
    assert np.array_equal(sig_c.view(np.int64), sig_f.view(np.int64))


def test_cpu_driven_special_cases(tl, h):
    npts = 700
    sig0, deps = inputs.norton_points(npts, 77)
    prm = oracle.norton_params()
    # a mix of stop reasons in one batch: non-finite points, capped points
    sig_bad = sig0.copy()
    sig_bad[::9, 4] = np.inf
    for max_iter in (0, 1, 2, 20):
        x_c, it_c, st_c, sig_c = gpu_norton_cd(tl, h, prm, sig_bad, deps, max_iter=max_iter)
        x_f, it_f, st_f, sig_f = gpu_norton(tl, h, prm, sig_bad, deps, max_iter=max_iter)
        assert np.array_equal(it_c, it_f) and np.array_equal(st_c, st_f)
        assert (st_c[::9] == 3).all()
        assert np.array_equal(x_c, x_f, equal_nan=True)
        assert np.array_equal(sig_c, sig_f, equal_nan=True)
    # elastic: A = 0 -> zero residual at the predictor, no solve
    x_c, it_c, st_c, _ = gpu_norton_cd(tl, h, oracle.norton_params(A=0.0), sig0, deps, want_sig=False)
    assert (it_c == 0).all() and (st_c == 0).all()
    assert np.array_equal(x_c[:, :6], deps) and (x_c[:, 6] == 0).all()


def test_cpu_driven_argument_errors(tl, h):
    d = torch.zeros(64, dtype=torch.float64, device=DEV)
    i = torch.zeros(64, dtype=torch.int32, device=DEV)
    f = tl.tl_newton_integrate_cpu_driven
    law = tl.make_law(tl.TL_LAW_NORTON, 6, oracle.norton_params())
    assert f(h, law, 4, d, d, None, i, i, 1e-10, 20) == tl.TL_ERR_INVALID_ARG
    law = tl.make_law(tl.TL_LAW_NORTON, 7, oracle.norton_params())
    assert f(h, law, -1, d, d, None, i, i, 1e-10, 20) == tl.TL_ERR_INVALID_ARG
    assert f(h, law, 4, d, d, None, i, i, -1.0, 20) == tl.TL_ERR_INVALID_ARG
    assert f(h, law, 4, d, d, None, i, i, 1e-10, -1) == tl.TL_ERR_INVALID_ARG
    assert f(h, law, 4, None, d, None, i, i, 1e-10, 20) == tl.TL_ERR_INVALID_ARG
    assert tl.tl_last_bad_arg(h) == 4
    assert f(h, law, 0, d, d, None, i, i, 1e-10, 20) == tl.TL_OK
    law = tl.make_law(tl.TL_LAW_TANH, 4)
    assert f(h, law, 4, d, d, None, i, i, 1e-10, 20) == tl.TL_ERR_UNSUPPORTED
