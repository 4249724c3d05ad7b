"""Pins of the oracle's mixed-precision solve (binary32 LUpp factor, binary64
iterative refinement with at most 3 corrections, binary64 LUpp fallback; the
scheme of Langou et al. 2006 -- the paper itself factors in binary64 only)
against things other than itself: hand-worked binary32 eliminations,
exactly representable systems, the binary64 oracle (pinned separately), the
convergence guarantee of the stopping test, and exact invariances.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2609_15217_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ir_hand_examples.json")


def _val(v):
    """'p/q', 'M*2^e' or an integer string -> float (all exact dyadics)."""
    v = str(v)
    if "*2^" in v:
        m, e = v.split("*2^")
        return math.ldexp(float(int(m)), int(e))
    return float(Fraction(v))


def designed_dyadic(n, batch, seed):
    """A = P^T L U with |l_ij| in {0, 1/4, 1/2} below a unit diagonal and
    power-of-two diagonal u_kk, small dyadic u_kj: partial pivoting must
    recover P (every candidate below the pivot is at most half of it), and
    every binary32 operation of the elimination and of the solves is exact.
    Returns A, the designed ipiv, L, U and an exact dyadic x with b = A x."""
    g = inputs.rng(seed)
    As, piv, Ls, Us, xs, bs = [], [], [], [], [], []
    for _ in range(batch):
        L = np.eye(n) + np.tril(g.choice([0.0, 0.25, -0.25, 0.5, -0.5], size=(n, n)), -1)
        U = np.triu(g.integers(-16, 17, size=(n, n)) / 8.0, 1)
        U += np.diag(2.0 ** g.integers(0, 3, size=n) * g.choice([-1.0, 1.0], size=n))
        # sequential interchanges: step k swaps row k with a row p >= k
        ipiv = np.array([int(g.integers(k, n)) for k in range(n)])
        order = list(range(n))
        for k, p in enumerate(ipiv):
            order[k], order[p] = order[p], order[k]
        PA = L @ U                        # exact: few-bit dyadics
        A = np.empty_like(PA)
        A[order] = PA                     # A[order[k]] = (LU)[k]
        x = g.integers(-8, 9, size=n) / 4.0
        As.append(A)
        piv.append(ipiv + 1)
        Ls.append(L)
        Us.append(U)
        xs.append(x)
        bs.append(A @ x)
    return np.array(As), np.array(piv), np.array(Ls), np.array(Us), np.array(xs), np.array(bs)


# ---------------------------------------------------------------------------
# pin checks (take the library so that the planted-mistake test reuses them)
# ---------------------------------------------------------------------------

def pin_ir_golden(lib):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = np.array([[_val(v) for v in row] for row in c["A"]])[None]
        b = np.array([_val(v) for v in c["b"]])[None]
        LU, ipiv, ok = oracle.sgetrf(A.astype(np.float32), lib=lib)
        assert ok[0] and list(ipiv[0]) == c["ipiv"]
        U = np.array([[_val(v) for v in row] for row in c["U"]])
        assert LU[0, 1, 0] == np.float32(_val(c["L21"]))
        assert np.array_equal(np.triu(LU[0]).astype(np.float64), U)
        x, ipiv2, info, steps = oracle.ir_gesv(A, b, lib=lib)
        assert info[0] == 0 and steps[0] == c["steps"] and list(ipiv2[0]) == c["ipiv"]
        assert np.array_equal(x[0], [_val(v) for v in c["x"]])


def pin_ir_exact_designed(lib):
    for n in (2, 5, 9, 16):
        A, piv, L, U, x_true, b = designed_dyadic(n, 20, 40 + n)
        LU, ipiv, ok = oracle.sgetrf(A.astype(np.float32), lib=lib)
        assert ok.all() and np.array_equal(ipiv, piv)
        Lg = np.tril(LU, -1) + np.eye(n, dtype=np.float32)
        assert np.array_equal(Lg.astype(np.float64), L)
        assert np.array_equal(np.triu(LU).astype(np.float64), U)
        # the exact binary32 solve needs no correction
        x, ipiv2, info, steps = oracle.ir_gesv(A, b, lib=lib)
        assert (steps == 0).all() and (info == 0).all() and np.array_equal(ipiv2, piv)
        assert np.array_equal(x, x_true)


def pin_ir_accuracy(lib):
    for n in (3, 8, 13, 25):
        # well conditioned: refined, never the fallback
        A, x_true, b, kappa = inputs.kappa_systems(n, 60, 70 + n, 1e1, 1e3)
        x, ipiv, info, steps = oracle.ir_gesv(A, b, lib=lib)
        assert (steps >= 1).all() and (steps <= 3).all() and (info == 0).all()
        # the stopping test guarantees a binary64 backward error: recompute
        # the residual in extended precision
        Al = A.astype(np.longdouble)
        r = b.astype(np.longdouble) - np.einsum("sij,sj->si", Al, x.astype(np.longdouble))
        anrm = np.abs(A).sum(axis=2).max(axis=1)
        xnrm = np.abs(x).max(axis=1)
        be = np.abs(r).max(axis=1).astype(np.float64) / (anrm * xnrm)
        # bound of the test plus the rounding of the computed residual
        assert (be <= (math.sqrt(n) + 2 * n) * 2.0 ** -53 * 1.01).all()
        fe = np.abs(x - x_true).max(axis=1) / np.abs(x_true).max(axis=1)
        assert (fe <= 1e-12 * kappa).all()
        # binary32 pivots differ from binary64 ones only at near-ties
        _, piv64, _, _ = oracle.gesv(A, b, lib=lib)
        assert (ipiv == piv64).all(axis=1).mean() > 0.9
        # hopeless conditioning for binary32: every system falls back and
        # then is exactly the binary64 LUpp
        A, x_true, b, kappa = inputs.kappa_systems(n, 30, 80 + n, 1e9, 1e10)
        x, ipiv, info, steps = oracle.ir_gesv(A, b, lib=lib)
        x64, piv64, info64, _ = oracle.gesv(A, b, lib=lib)
        assert (steps == -1).all()
        assert np.array_equal(x, x64) and np.array_equal(ipiv, piv64) and np.array_equal(info, info64)


def pin_ir_special(lib):
    n = 6
    A, _, b, _ = inputs.kappa_systems(n, 8, 90, 1e1, 1e2)
    x64, piv64, info64, _ = oracle.gesv(A, b, lib=lib)
    base = oracle.ir_gesv(A, b, lib=lib)
    assert (base[3] >= 1).all()
    # b = 0: the zero solution with no correction
    x, _, info, steps = oracle.ir_gesv(A, np.zeros_like(b), lib=lib)
    assert (steps == 0).all() and (x == 0).all()
    # an entry that overflows binary32, one below FLT_MIN, a NaN, a zero
    # column: binary64 results
    for s, (i, j, v) in enumerate([(0, 0, 1e39), (1, 2, 1e-39), (2, 3, np.nan)]):
        A2 = A.copy()
        A2[s, i, j] = v
        x, ipiv, info, steps = oracle.ir_gesv(A2, b, lib=lib)
        xr, pr, ir, _ = oracle.gesv(A2, b, lib=lib)
        assert steps[s] == -1 and info[s] == ir[s] and np.array_equal(ipiv[s], pr[s])
        assert np.array_equal(x[s], xr[s], equal_nan=True)
        others = np.arange(len(A)) != s
        assert np.array_equal(x[others], base[0][others])
    A3 = A.copy()
    A3[4, :, 2] = 0.0
    x, ipiv, info, steps = oracle.ir_gesv(A3, b, lib=lib)
    assert steps[4] == -1 and info[4] == 3 and np.isnan(x[4]).all()
    # exact zeros are fine in binary32
    A4 = A.copy()
    A4[5, 0, 1] = 0.0
    x, ipiv, info, steps = oracle.ir_gesv(A4, b, lib=lib)
    assert steps[5] >= 0


def pin_ir_scaling(lib):
    """The mixed-precision solve commutes with power-of-two scaling: A and b
    by 2^e give the same x bit for bit; b alone by 2^e scales x by 2^e."""
    for n in (4, 12):
        A, b, _, _ = inputs.sweep_systems(n, 40, 95 + n)
        x, ipiv, info, steps = oracle.ir_gesv(A, b, lib=lib)
        for e in (-40, 37):
            x2, ipiv2, info2, steps2 = oracle.ir_gesv(np.ldexp(A, e), np.ldexp(b, e), lib=lib)
            assert np.array_equal(steps, steps2) and np.array_equal(ipiv, ipiv2)
            assert np.array_equal(x, x2)
            x3, _, _, steps3 = oracle.ir_gesv(A, np.ldexp(b, e), lib=lib)
            assert np.array_equal(steps, steps3) and np.array_equal(np.ldexp(x, e), x3)


IR_PINS = [pin_ir_golden, pin_ir_exact_designed, pin_ir_accuracy, pin_ir_special, pin_ir_scaling]


@pytest.mark.parametrize("pin", IR_PINS, ids=lambda p: p.__name__)
def test_ir_pin(pin):
    pin(oracle.load())


def test_sgetrf_reconstruction_is_binary32():
    """PA = LU holds to binary32 accuracy (and no better: the factor really
    is computed in binary32)."""
    n = 16
    A, _ = inputs.uniform_systems(n, 50, 123)
    A32 = A.astype(np.float32)
    LU, ipiv, ok = oracle.sgetrf(A32)
    assert ok.all()
    worst = 0.0
    for s in range(50):
        order = list(range(n))
        for k, p in enumerate(ipiv[s]):
            order[k], order[p - 1] = order[p - 1], order[k]
        L = (np.tril(LU[s], -1) + np.eye(n)).astype(np.float64)
        U = np.triu(LU[s]).astype(np.float64)
        E = np.abs(A32[s][order].astype(np.float64) - L @ U)
        bound = 2 * n * 2.0 ** -24 * (np.abs(L) @ np.abs(U))
        assert (E <= bound).all()
        worst = max(worst, (E / (np.abs(L) @ np.abs(U))).max())
    assert worst > 2.0 ** -30


def test_ir_steps_histogram_is_plausible():
    """On the sweep recipe most systems converge after 1-3 corrections and
    the binary64 fallback is taken for the badly conditioned part."""
    A, b, _, kappa = inputs.sweep_systems(8, 400, 77)
    _, _, _, steps = oracle.ir_gesv(A, b)
    assert set(np.unique(steps)) <= {-1, 1, 2, 3}
    assert (steps >= 1).mean() > 0.6
