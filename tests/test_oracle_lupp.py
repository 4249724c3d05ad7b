"""Pins of the CPU oracle's LUpp (getrf / getrs / gesv) against things other
than itself: hand-worked examples, exact rational elimination, Cramer's
rule, LAPACK, reconstruction and error bounds, and exact invariances.

Paper passage: Sec. 2.2 (LU with partial pivoting, PA = LU, Ly = Pb, Ux = y).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2609_15217_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lupp_hand_examples.json")


def _num(v):
    if isinstance(v, str):
        if v.startswith("2^"):
            return Fraction(2) ** int(v[2:])
        return Fraction(v)
    return Fraction(v)


def _split_lu(LU):
    n = LU.shape[-1]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return L, U


def _perm_from_ipiv(ipiv):
    """Row order produced by applying the 1-based sequential interchanges."""
    n = len(ipiv)
    order = list(range(n))
    for k, p in enumerate(ipiv):
        p -= 1
        order[k], order[p] = order[p], order[k]
    return order


# ---------------------------------------------------------------------------
# Hand-worked examples
# ---------------------------------------------------------------------------

def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_worked_examples(case):
    A = np.array([[float(_num(v)) for v in row] for row in case["A"]])[None]
    b = np.array([float(_num(v)) for v in case["b"]])[None]
    n = A.shape[-1]
    x, ipiv, info, _gap, LU = oracle.gesv(A, b, want_lu=True)
    assert list(ipiv[0]) == case["ipiv"]
    assert info[0] == case["info"]
    L, U = _split_lu(LU[0])
    Lg = np.array([[float(_num(v)) for v in row] for row in case["L"]])
    Ug = np.array([[float(_num(v)) for v in row] for row in case["U"]])
    scale = np.abs(Ug).max()
    assert np.allclose(L, Lg, rtol=4 * EPS, atol=0), (L, Lg)
    assert np.allclose(U, Ug, rtol=8 * EPS, atol=8 * EPS * scale), (U, Ug)
    if case["x"] is None:
        assert np.isnan(x).all()
    else:
        xg = np.array([float(_num(v)) for v in case["x"]])
        assert np.allclose(x[0], xg, rtol=1e-14, atol=1e-14)
    # getrf + getrs gives the same bits as the fused gesv
    LU2, ipiv2, info2, _ = oracle.getrf(A)
    assert np.array_equal(LU2, LU) and np.array_equal(ipiv2, ipiv)
    if case["info"] == 0:
        x2 = oracle.getrs(LU2, ipiv2, b)
        assert np.array_equal(x2, x)
    assert n == len(case["ipiv"])


# ---------------------------------------------------------------------------
# Exact rational elimination (brute force on small n)
# ---------------------------------------------------------------------------

def _exact_gepp(A):
    """Gaussian elimination with partial pivoting in exact rationals."""
    n = len(A)
    M = [[Fraction(float(v)) for v in row] for row in A]
    ipiv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        ipiv.append(p + 1)
        if M[p][k] == 0:
            continue
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
            for j in range(k + 1, n):
                M[i][j] -= M[i][k] * M[k][j]
    return M, ipiv


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_exact_rational_elimination(n):
    A, b = inputs.uniform_systems(n, 60, inputs.config_seed(90, n))
    LU, ipiv, info, gap = oracle.getrf(A)
    checked = 0
    for s in range(A.shape[0]):
        M, piv_exact = _exact_gepp(A[s])
        if gap[s] < 1e-8:
            continue  # near-tie: rounding may legitimately pick the other row
        checked += 1
        assert list(ipiv[s]) == piv_exact
        exact = np.array([[float(v) for v in row] for row in M])
        growth = max(1.0, np.abs(exact).max())
        assert np.allclose(LU[s], exact, rtol=0, atol=200 * n * EPS * growth)
    assert checked >= 50


# ---------------------------------------------------------------------------
# Cramer's rule (exact) for n <= 4
# ---------------------------------------------------------------------------

def _det(M):
    n = len(M)
    if n == 1:
        return M[0][0]
    return sum((-1) ** j * M[0][j] * _det([row[:j] + row[j + 1:] for row in M[1:]]) for j in range(n))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_cramer(n):
    A, b = inputs.uniform_systems(n, 100, inputs.config_seed(91, n))
    x, ipiv, info, _ = oracle.gesv(A, b)
    assert (info == 0).all()
    for s in range(A.shape[0]):
        M = [[Fraction(float(v)) for v in row] for row in A[s]]
        d = _det(M)
        xs = []
        for j in range(n):
            Mj = [row[:] for row in M]
            for i in range(n):
                Mj[i][j] = Fraction(float(b[s, i]))
            xs.append(_det(Mj) / d)
        xe = np.array([float(v) for v in xs])
        kappa = np.linalg.cond(A[s], np.inf)
        err = np.abs(x[s] - xe).max() / max(np.abs(xe).max(), 1e-300)
        assert err <= 10 * n * kappa * EPS, (s, err, kappa)


# ---------------------------------------------------------------------------
# PA = LU reconstruction, manufactured solutions, backward error
# ---------------------------------------------------------------------------

def _residual_exactish(A, x, b):
    Al = A.astype(np.longdouble)
    return np.einsum("sij,sj->si", Al, x.astype(np.longdouble)) - b.astype(np.longdouble)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13, 20, 32])
def test_pa_equals_lu(n):
    A, _ = inputs.uniform_systems(n, 200, inputs.config_seed(92, n))
    LU, ipiv, info, _ = oracle.getrf(A)
    assert (info == 0).all()
    for s in range(A.shape[0]):
        L, U = _split_lu(LU[s])
        PA = A[s][_perm_from_ipiv(ipiv[s])]
        E = np.abs(PA.astype(np.longdouble) - L.astype(np.longdouble) @ U.astype(np.longdouble))
        bound = n * EPS * (np.abs(L) @ np.abs(U))
        assert (E <= bound + 1e-300).all()
        assert np.abs(L).max() <= 1.0  # partial pivoting bounds the multipliers


@pytest.mark.parametrize("n", [2, 7, 8, 16, 25, 32])
def test_manufactured_and_backward_error(n):
    A, x_true, b, kappa = inputs.kappa_systems(n, 150, inputs.config_seed(93, n))
    x, ipiv, info, _ = oracle.gesv(A, b)
    assert (info == 0).all()
    fe = np.abs(x - x_true).max(axis=1) / np.abs(x_true).max(axis=1)
    assert (fe <= 1e-12 * kappa).all(), (fe / kappa).max()
    r = np.abs(_residual_exactish(A, x, b)).max(axis=1)
    be = r / (np.abs(A).sum(axis=2).max(axis=1) * np.abs(x).max(axis=1) * EPS)
    assert (be <= 10 * n).all(), be.max()


@pytest.mark.parametrize("n", [3, 8, 17, 32])
def test_backward_error_uniform(n):
    A, b = inputs.uniform_systems(n, 300, inputs.config_seed(94, n))
    x, ipiv, info, _ = oracle.gesv(A, b)
    r = np.abs(_residual_exactish(A, x, b)).max(axis=1)
    be = r / (np.abs(A).sum(axis=2).max(axis=1) * np.abs(x).max(axis=1) * EPS)
    assert (be <= 10 * n).all(), be.max()


# ---------------------------------------------------------------------------
# LAPACK cross-check (scipy dgetrf)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [4, 9, 16, 31])
def test_lapack_crosscheck(n):
    sl = pytest.importorskip("scipy.linalg")
    A, b = inputs.uniform_systems(n, 200, inputs.config_seed(95, n))
    LU, ipiv, info, gap = oracle.getrf(A)
    x, *_ = oracle.gesv(A, b)
    agree = 0
    for s in range(A.shape[0]):
        lu, piv = sl.lu_factor(A[s])
        if gap[s] > 1e-10:
            assert np.array_equal(piv + 1, ipiv[s])
            assert np.allclose(lu, LU[s], rtol=1e-11, atol=1e-11 * np.abs(lu).max())
            agree += 1
        xs = sl.lu_solve((lu, piv), b[s])
        assert np.allclose(x[s], xs, rtol=1e-9, atol=1e-9 * np.abs(xs).max())
    assert agree >= 150


# ---------------------------------------------------------------------------
# Exact invariances and special cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("e", [-31, -10, 3, 40])
def test_power_of_two_scaling(e):
    """Scaling A by 2^e is exact, so pivots and L are bit-identical and U is
    scaled exactly; e = -31 maps U[-1,1] onto the paper's 'stress' range
    U[-5e-10, 5e-10] (Sec. 4.2)."""
    n = 12
    A, _ = inputs.uniform_systems(n, 100, inputs.config_seed(96, n))
    LU, ipiv, info, _ = oracle.getrf(A)
    LU2, ipiv2, info2, _ = oracle.getrf(np.ldexp(A, e))
    assert np.array_equal(ipiv, ipiv2)
    L, U = np.tril(LU, -1), np.triu(LU)
    L2, U2 = np.tril(LU2, -1), np.triu(LU2)
    assert np.array_equal(L, L2)
    assert np.array_equal(np.ldexp(U, e), U2)


def test_permuted_triangular_pivots():
    """A = rows of a nonsingular upper-triangular matrix in a random order:
    every column has exactly one candidate, so the pivot sequence is the
    permutation itself and L = I, U is the triangular matrix."""
    g = inputs.rng(97)
    for n in (2, 5, 11, 32):
        for _ in range(20):
            U = np.triu(g.uniform(-1, 1, (n, n)))
            U[np.diag_indices(n)] = g.uniform(0.5, 1.0, n) * g.choice([-1, 1], n)
            perm = g.permutation(n)
            A = U[perm]
            # expected interchanges: bring the row holding U's row k to k
            order = list(perm)
            exp = []
            for k in range(n):
                p = order.index(k, k)
                exp.append(p + 1)
                order[k], order[p] = order[p], order[k]
            LU, ipiv, info, _ = oracle.getrf(A[None])
            assert list(ipiv[0]) == exp
            assert np.array_equal(np.triu(LU[0]), U)
            assert np.array_equal(np.tril(LU[0], -1), np.zeros((n, n)))


def test_singular_and_nonfinite():
    n = 5
    A, b = inputs.uniform_systems(n, 4, 98)
    A[0, :, 2] = 0.0          # zero column 2 -> pivot of step 2 is zero
    A[1] = 0.0                # all zero -> info = 1, identity pivots
    A[2, 3, 1] = np.nan       # non-finite entry
    A[3, 0, 4] = np.inf
    x, ipiv, info, _ = oracle.gesv(A, b)
    assert info[0] == 3
    assert info[1] == 1 and list(ipiv[1]) == [1, 2, 3, 4, 5]
    assert info[2] == -1 and list(ipiv[2]) == [1, 2, 3, 4, 5]
    assert info[3] == -1
    assert np.isnan(x).all()
    # rank-deficient by a repeated column: exact zero pivot at the last step
    B = np.array([[[1.0, 2.0, 2.0], [4.0, 8.0, 8.0], [2.0, 4.0, 4.0]]])
    _, _, info, _ = oracle.getrf(B)
    assert info[0] == 2


def test_near_tie_gap():
    A = np.array([[[1.0, 2.0, 0.0], [-1.0, 3.0, 1.0], [0.5, 1.0, 4.0]]])
    LU, ipiv, info, gap = oracle.getrf(A)
    assert ipiv[0, 0] == 1          # exact tie: first row
    assert gap[0] == 0.0
    A2 = A.copy()
    A2[0, 1, 0] = -1.0 + 2 ** -40  # |a_10| just below |a_00|: still row 0, tiny gap
    _, ipiv2, _, gap2 = oracle.getrf(A2)
    assert ipiv2[0, 0] == 1 and 0 < gap2[0] < 1e-11
    A3 = A.copy()
    A3[0, 1, 0] = -1.0 - 2 ** -40  # just above: row 1
    _, ipiv3, _, _ = oracle.getrf(A3)
    assert ipiv3[0, 0] == 2


def test_getrs_multiple_systems_match_gesv():
    n = 9
    A, b = inputs.uniform_systems(n, 64, 99)
    x, ipiv, info, gap, LU = oracle.gesv(A, b, want_lu=True)
    LU2, ipiv2, info2, gap2 = oracle.getrf(A)
    assert np.array_equal(LU, LU2) and np.array_equal(ipiv, ipiv2) and np.array_equal(gap, gap2)
    x2 = oracle.getrs(LU2, ipiv2, b)
    assert np.array_equal(x, x2)


def test_threads_do_not_change_results():
    n = 14
    A, b = inputs.uniform_systems(n, 500, 100)
    r1 = oracle.gesv(A, b, nthreads=1)
    r2 = oracle.gesv(A, b, nthreads=0)
    for u, v in zip(r1, r2):
        assert np.array_equal(u, v, equal_nan=True)


# ---------------------------------------------------------------------------
# Tile-local pivoting (Sec. 3.2, Tiled solvers; 1e-10 threshold of Sec. 4.1)
# ---------------------------------------------------------------------------

def pin_tiled(lib=None):
    for n in (5, 12, 32):
        A, b = inputs.uniform_systems(n, 40, 6000 + n, -0.5, 0.5)
        LU, piv, info, _ = oracle.getrf(A, lib=lib)
        # one tile covering the matrix, or an infinite threshold: textbook
        for tile, thr in ((n, 1e-10), (0, 1e-10), (2, np.inf)):
            LUt, pivt, infot, oot = oracle.getrf_tiled(A, tile, thr, lib=lib)
            assert np.array_equal(pivt, piv) and np.array_equal(LUt.view(np.int64), LU.view(np.int64))
        # the default distribution never looks below a tile (Sec. 4.1)
        for tile in (2, 3, 6):
            LUt, pivt, infot, oot = oracle.getrf_tiled(A, tile, 1e-10, lib=lib)
            assert (oot == 0).all() and (infot == 0).all()
            # every pivot stays inside its diagonal tile
            k = np.arange(n)
            hi = np.minimum((k // tile + 1) * tile, n)
            assert ((pivt - 1 >= k) & (pivt - 1 < hi)).all()
            # PA = LU with the permutation of the tile-local pivots
            for s in range(5):
                P = _perm_from_ipiv(pivt[s])
                L, U = _split_lu(LUt[s])
                assert np.abs(A[s][P] - L @ U).max() <= 4 * n * EPS * (np.abs(L) @ np.abs(U)).max()
        # the stress distribution U[+-5e-10] triggers lower-tile searches,
        # and a 2^31 scaling (entries above the threshold) suppresses them
        S = A * 1e-9
        _, pivs, _, oot = oracle.getrf_tiled(S, 2, 1e-10, lib=lib)
        assert (oot > 0).mean() > 0.3
        _, pivb, _, ootb = oracle.getrf_tiled(np.ldexp(S, 40), 2, 1e-10, lib=lib)
        assert (ootb == 0).all()


def test_tiled_pivoting_pins():
    pin_tiled()
