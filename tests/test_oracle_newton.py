"""Pins of the CPU oracle's Newton driver (Sec. 2.1, Eqs. 1-3; Algorithm 2)
and its two laws: the implicit Norton viscoplastic law (Sec. 4.3 law class)
and the synthetic tanh law.

Independent references used here: the radial-return reduction of J2 +
Norton to one monotone scalar equation (solved by bisection, written from
the mechanics, not from the oracle), the elastic special cases, central
finite differences of the residual, quadratic convergence, the linear
special case of the tanh law and a scalar bisection for n = 1.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_15217_gb300 import inputs

PRM = oracle.norton_params()  # E=200000, nu=0.3, A=1e-12, m=4, dt=1


def _lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def radial_return(prm, sig0, deps):
    """Closed-form reduction of the implicit J2 + Norton step.

    With isotropic elasticity the flow direction is the trial one and the
    equivalent stress drops by 3 mu dp, so dp solves the scalar monotone
    equation h(dp) = dp - dt A (seq_tr - 3 mu dp)^m = 0 on [0, seq_tr/(3 mu)].
    Returns (de_el, dp)."""
    E, nu, A, m, dt = prm
    lam, mu = _lame(E, nu)
    one = np.array([1, 1, 1, 0, 0, 0], float)
    sig_tr = sig0 + lam * deps[:3].sum() * one + 2 * mu * deps
    s = sig_tr - sig_tr[:3].sum() / 3 * one
    seq = math.sqrt(1.5 * float(s @ s))
    if seq == 0.0 or A == 0.0:
        return deps.copy(), 0.0
    ntr = 1.5 * s / seq

    def h(dp):
        return dp - dt * A * (seq - 3 * mu * dp) ** int(m)

    lo, hi = 0.0, seq / (3 * mu)
    assert h(lo) < 0 < h(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if h(mid) < 0:
            lo = mid
        else:
            hi = mid
    dp = 0.5 * (lo + hi)
    return deps - dp * ntr, dp


def test_elastic_step_zero_viscosity():
    sig0, deps = inputs.norton_points(200, 11)
    prm = oracle.norton_params(A=0.0)
    r = oracle.newton_norton(prm, sig0, deps)
    assert (r["status"] == oracle.NEWTON_CONVERGED).all()
    assert (r["iterations"] == 0).all()
    assert np.array_equal(r["x"][:, :6], deps)
    assert (r["x"][:, 6] == 0.0).all()


def test_elastic_step_volumetric():
    """sig0 = 0 and a purely volumetric strain increment: the stress is
    hydrostatic and seq = 0 up to the rounding of the mean stress, so dp = 0
    and de_el = deps.  (The deviator is pure rounding noise here, so the
    relative stopping test may not be reachable: the run may end on the
    iteration cap, but the state must stay on the elastic solution.)"""
    g = inputs.rng(12)
    e = g.uniform(-1e-3, 1e-3, size=50)
    deps = np.zeros((50, 6))
    deps[:, :3] = e[:, None]
    r = oracle.newton_norton(PRM, np.zeros((50, 6)), deps)
    assert np.isin(r["status"], [0, 1]).all()
    assert np.allclose(r["x"][:, :6], deps, rtol=1e-14, atol=0)
    assert (np.abs(r["x"][:, 6]) <= 1e-40).all()


@pytest.mark.parametrize("rtol,tol", [(1e-10, 1e-8), (1e-13, 2e-11)])
def test_radial_return_closed_form(rtol, tol):
    """The 7x7 Newton state equals the scalar radial-return root.  The stop
    test bounds the residual, not the state error, so the state tolerance
    follows the residual tolerance (quadratic convergence makes it far
    smaller in practice)."""
    sig0, deps = inputs.norton_points(400, inputs.config_seed(3))
    r = oracle.newton_norton(PRM, sig0, deps, rtol=rtol, max_iter=30)
    assert (r["status"] == 0).all()
    for p in range(sig0.shape[0]):
        de_ref, dp_ref = radial_return(PRM, sig0[p], deps[p])
        x = r["x"][p]
        assert abs(x[6] - dp_ref) <= tol * abs(dp_ref) + 1e-22, (p, x[6], dp_ref)
        assert np.allclose(x[:6], de_ref, rtol=tol, atol=tol * np.abs(de_ref).max())
    # the workload really is visco-plastic: several solves per point
    it = r["iterations"]
    assert it.min() >= 2 and it.max() <= 20 and it.mean() > 3


def test_stress_output_matches_radial_return():
    sig0, deps = inputs.norton_points(50, 13)
    r = oracle.newton_norton(PRM, sig0, deps)
    E, nu = PRM[0], PRM[1]
    lam, mu = _lame(E, nu)
    one = np.array([1, 1, 1, 0, 0, 0], float)
    for p in range(50):
        de, dp = radial_return(PRM, sig0[p], deps[p])
        sig = sig0[p] + lam * de[:3].sum() * one + 2 * mu * de
        assert np.allclose(r["sig"][p], sig, rtol=1e-9, atol=1e-9 * np.abs(sig).max())


def test_norton_jacobian_finite_differences():
    sig0, deps = inputs.norton_points(30, 14)
    g = inputs.rng(15)
    for p in range(30):
        x = np.concatenate([deps[p] * g.uniform(0.5, 1.5, 6), [g.uniform(0, 1e-3)]])
        F, J, _ = oracle.norton_eval(PRM, sig0[p], deps[p], x)
        Jfd = np.empty((7, 7))
        for j in range(7):
            h = 1e-9
            xp, xm = x.copy(), x.copy()
            xp[j] += h
            xm[j] -= h
            Fp, _, _ = oracle.norton_eval(PRM, sig0[p], deps[p], xp)
            Fm, _, _ = oracle.norton_eval(PRM, sig0[p], deps[p], xm)
            Jfd[:, j] = (Fp - Fm) / (2 * h)
        assert np.allclose(J, Jfd, rtol=1e-5, atol=1e-6 * np.abs(J).max()), np.abs(J - Jfd).max()


def test_norton_quadratic_convergence():
    sig0, deps = inputs.norton_points(20, 16)
    for p in range(20):
        res = []
        for k in range(0, 12):
            r = oracle.newton_norton(PRM, sig0[p:p + 1], deps[p:p + 1], rtol=0.0, max_iter=k)
            F, _, _ = oracle.norton_eval(PRM, sig0[p], deps[p], r["x"][0])
            res.append(np.linalg.norm(F))
        res = np.array(res)
        r0 = res[0]
        # pick iterates in the quadratic basin, above the rounding floor
        for k in range(1, len(res) - 1):
            if 1e-13 * r0 < res[k + 1] and res[k] < 1e-3 * r0:
                assert res[k + 1] <= 1e3 * res[k] ** 2 / r0 + 1e-14 * r0, (p, k, res)


def test_newton_driver_status_codes():
    n = 4
    A, c, b = inputs.tanh_points(n, 3, 17)
    # max-iter: rtol = 0 never converges unless the residual is exactly zero
    r = oracle.newton_tanh(A, c, b, rtol=0.0, max_iter=5)
    assert (r["status"] == oracle.NEWTON_MAXITER).all() and (r["iterations"] == 5).all()
    # singular Jacobian: A = 0, c = 0
    r = oracle.newton_tanh(np.zeros_like(A), np.zeros_like(c), b)
    assert (r["status"] == oracle.NEWTON_SINGULAR).all() and (r["iterations"] == 0).all()
    # non-finite residual
    b2 = b.copy()
    b2[:, 1] = np.inf
    r = oracle.newton_tanh(A, c, b2)
    assert (r["status"] == oracle.NEWTON_NONFINITE).all()
    # zero initial residual: converged without a solve
    r = oracle.newton_tanh(A, c, np.zeros_like(b))
    assert (r["status"] == 0).all() and (r["iterations"] == 0).all() and (r["x"] == 0).all()


def test_tanh_linear_case_one_solve():
    for n in (1, 7, 13, 20, 32):
        A, c, b = inputs.tanh_points(n, 40, 18 + n)
        r = oracle.newton_tanh(A, np.zeros_like(c), b)
        assert (r["status"] == 0).all() and (r["iterations"] == 1).all()
        xs = np.linalg.solve(A, b[:, :, None])[:, :, 0]
        assert np.allclose(r["x"], xs, rtol=1e-12, atol=1e-12 * np.abs(xs).max())


def test_tanh_scalar_bisection():
    A, c, b = inputs.tanh_points(1, 200, 19)
    r = oracle.newton_tanh(A, c, b, rtol=1e-14, max_iter=40)
    assert (r["status"] == 0).all()
    for p in range(200):
        a, cc, bb = A[p, 0, 0], c[p, 0], b[p, 0]
        f = lambda x: a * x + cc * math.tanh(x) - bb  # noqa: E731
        lo, hi = -1e3, 1e3
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid in (lo, hi):
                break
            if f(mid) < 0:
                lo = mid
            else:
                hi = mid
        assert abs(r["x"][p, 0] - mid) <= 1e-12 * max(1.0, abs(mid))


def test_tanh_jacobian_finite_differences():
    for n in (3, 13):
        A, c, b = inputs.tanh_points(n, 5, 20 + n)
        g = inputs.rng(21)
        for p in range(5):
            x = g.uniform(-2, 2, n)
            F, J = oracle.tanh_eval(A[p], c[p], b[p], x)
            Jfd = np.empty((n, n))
            for j in range(n):
                h = 1e-6
                xp, xm = x.copy(), x.copy()
                xp[j] += h
                xm[j] -= h
                Jfd[:, j] = (oracle.tanh_eval(A[p], c[p], b[p], xp)[0] - oracle.tanh_eval(A[p], c[p], b[p], xm)[0]) / (2 * h)
            assert np.allclose(J, Jfd, rtol=1e-7, atol=1e-7 * np.abs(J).max())


def test_tanh_workload_iterations():
    """The served-stream law takes several Newton iterations per point."""
    for n in (7, 13, 20, 32):
        A, c, b = inputs.tanh_points(n, 100, 22 + n)
        r = oracle.newton_tanh(A, c, b)
        assert (r["status"] == 0).all()
        assert r["iterations"].min() >= 2 and r["iterations"].max() <= 20
        F = np.array([oracle.tanh_eval(A[p], c[p], b[p], r["x"][p])[0] for p in range(100)])
        assert (np.linalg.norm(F, axis=1) <= 1e-10 * np.linalg.norm(b, axis=1)).all()


def test_relative_stop_is_scale_invariant():
    """Scaling A, c, b by 2^e scales F and J exactly, so every Newton step
    and every (relative) stopping decision is bit-identical."""
    for n in (2, 13):
        A, c, b = inputs.tanh_points(n, 100, 40 + n)
        r1 = oracle.newton_tanh(A, c, b)
        for e in (-40, 40):
            r2 = oracle.newton_tanh(np.ldexp(A, e), np.ldexp(c, e), np.ldexp(b, e))
            assert np.array_equal(r1["iterations"], r2["iterations"])
            assert np.array_equal(r1["status"], r2["status"])
            assert np.array_equal(r1["x"], r2["x"])


# ---------------------------------------------------------------------------
# Consistent tangent operator (Sec. 4.3: the multi-RHS solve after
# convergence)
# ---------------------------------------------------------------------------

def _mandel_C(prm):
    E, nu = prm[0], prm[1]
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = 2 * mu * np.eye(6)
    C[:3, :3] += lam
    return C


def pin_tangent(lib=None):
    prm = oracle.norton_params()
    sig0, deps = inputs.norton_points(12, 4321)
    # elastic step: the tangent is the elasticity tensor exactly
    prm0 = oracle.norton_params(A=0.0)
    r = oracle.newton_norton(prm0, sig0, deps, lib=lib)
    for p in range(4):
        D, info = oracle.norton_tangent(prm0, sig0[p], deps[p], r["x"][p], lib=lib)
        assert info == 0 and np.array_equal(D, _mandel_C(prm0))
    r = oracle.newton_norton(prm, sig0, deps, rtol=1e-14, max_iter=40, lib=lib)
    assert (r["status"] == 0).all()
    h = 1e-7
    for p in range(6):
        D, info = oracle.norton_tangent(prm, sig0[p], deps[p], r["x"][p], lib=lib)
        assert info == 0
        # associative J2 flow: the consistent tangent is symmetric
        assert np.abs(D - D.T).max() <= 1e-9 * np.abs(D).max()
        # softer than elasticity along the flow, never stiffer
        assert np.linalg.eigvalsh(0.5 * (D + D.T)).max() <= np.linalg.eigvalsh(_mandel_C(prm)).max() * (1 + 1e-12)
        # central differences of the converged stress in deps
        Dfd = np.empty((6, 6))
        for j in range(6):
            dp_, dm_ = deps[p:p + 1].copy(), deps[p:p + 1].copy()
            dp_[0, j] += h
            dm_[0, j] -= h
            sp = oracle.newton_norton(prm, sig0[p:p + 1], dp_, rtol=1e-15, max_iter=60, lib=lib)["sig"][0]
            sm = oracle.newton_norton(prm, sig0[p:p + 1], dm_, rtol=1e-15, max_iter=60, lib=lib)["sig"][0]
            Dfd[:, j] = (sp - sm) / (2 * h)
        assert np.abs(D - Dfd).max() <= 1e-5 * np.abs(D).max(), np.abs(D - Dfd).max() / np.abs(D).max()


def test_tangent_pins():
    pin_tangent()
