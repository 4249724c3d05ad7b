"""The oracle pins are sensitive: plant one plausible mistake at a time in a
copy of the oracle's C source (CPU only), rebuild it, and check that the pin
checks below reject every variant while accepting the real oracle.

Each mutation is a single textual edit of oracle/tinylu_oracle.c: a dropped
term, a wrong sign or index, a transposed operand, a wrong tie-break, a
missing guard.
"""
import json
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as obuild
from paper_2609_15217_gb300 import inputs

from test_oracle_ir import IR_PINS
from test_oracle_lupp import pin_tiled
from test_oracle_newton import pin_tangent, radial_return

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lupp_hand_examples.json")

MUTATIONS = {
    "tie_break_last": ("return fabs(a) > fabs(b);", "return fabs(a) >= fabs(b);"),
    "l_part_not_swapped": ("for (int j = 0; j < n; ++j) {\n                double t = AT(a, n, k, j);",
                           "for (int j = k; j < n; ++j) {\n                double t = AT(a, n, k, j);"),
    "update_sign": ("fma(-AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j))",
                    "fma(AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j))"),
    "update_transposed": ("fma(-AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j))",
                          "fma(-AT(a, n, i, k), AT(a, n, j, k), AT(a, n, i, j))"),
    "multiplier_perturbed": ("double r = 1.0 / akk;\n            for (int i = k + 1; i < n; ++i) AT(a, n, i, k) = AT(a, n, i, k) * r;",
                             "double r = 1.0 / akk;\n            for (int i = k + 1; i < n; ++i) AT(a, n, i, k) = AT(a, n, i, k) * r * 1.0000000001;"),
    "no_sfmin_guard": ("if (fabs(akk) >= DBL_MIN) {", "if (1) {"),
    "info_last_zero_pivot": ("if (info == 0) info = k + 1;", "info = k + 1;"),
    "forward_drops_term": ("for (int j = 0; j < i; ++j) s = fma(-AT(lu, n, i, j), b[j], s);",
                           "for (int j = 1; j < i; ++j) s = fma(-AT(lu, n, i, j), b[j], s);"),
    "backsolve_multiplies": ("b[i] = s / AT(lu, n, i, i);", "b[i] = s * AT(lu, n, i, i);"),
    "rhs_swaps_reversed": ("for (int k = 0; k < n; ++k) {\n        int p = ipiv[k] - 1;\n        if (p != k) {\n            double t",
                           "for (int k = n - 1; k >= 0; --k) {\n        int p = ipiv[k] - 1;\n        if (p != k) {\n            double t"),
    "ir_rhs_swaps_reversed": ("for (int k = 0; k < n; ++k) {\n        int p = ipiv[k] - 1;\n        if (p != k) {\n            float t",
                              "for (int k = n - 1; k >= 0; --k) {\n        int p = ipiv[k] - 1;\n        if (p != k) {\n            float t"),
    "norton_drops_flow": ("F[i] = de[i] - deps[i] + dp * nrm[i];", "F[i] = de[i] - deps[i];"),
    "norton_jacobian_sign": ("J[i + 7 * j] = (i == j ? 1.0 : 0.0) + c * v;",
                             "J[i + 7 * j] = (i == j ? 1.0 : 0.0) - c * v;"),
    "norton_power_off_by_one": ("for (int i = 0; i < m - 1; ++i) pw_m1 = pw_m1 * seq;",
                                "for (int i = 0; i < m - 2; ++i) pw_m1 = pw_m1 * seq;"),
    "norton_shear_modulus": ("const int m = (int)prm[3];\n    const double lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));\n    const double mu = E / (2.0 * (1.0 + nu));",
                             "const int m = (int)prm[3];\n    const double lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));\n    const double mu = E / (1.0 + nu);"),
    "newton_absolute_test": ("if (r <= rtol * r0 || r0 == 0.0)", "if (r <= rtol || r0 == 0.0)"),
    "newton_counts_evals": ("        ++k;\n        eval(ctx, x, F, J);", "        k += 2;\n        eval(ctx, x, F, J);"),
    "tanh_jacobian_sign": ("c[i] * (1.0 - t * t)", "c[i] * (1.0 + t * t)"),
    "tiled_never_looks_below": ("if (hi < n && fabs(AT(a, n, p, k)) < threshold) {", "if (0) {"),
    "tiled_tile_too_tall": ("hi = (k / tile + 1) * tile;", "hi = (k / tile + 2) * tile;"),
    "tangent_rhs_sign": ("for (int i = 0; i < 7; ++i) X[i] = (i == j) ? 1.0 : 0.0;",
                         "for (int i = 0; i < 7; ++i) X[i] = (i == j) ? -1.0 : 0.0;"),
    "tangent_drops_lambda": ("D[i + 6 * j] = 2.0 * mu * X[i] + (i < 3 ? lambda * tr : 0.0);",
                             "D[i + 6 * j] = 2.0 * mu * X[i];"),
    "ir_tie_break_last": ("return fabsf(a) > fabsf(b);", "return fabsf(a) >= fabsf(b);"),
    "ir_l_part_not_swapped": ("for (int j = 0; j < n; ++j) {\n                float t = AT(a, n, k, j);",
                              "for (int j = k; j < n; ++j) {\n                float t = AT(a, n, k, j);"),
    "ir_update_sign": ("fmaf(-AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j))",
                       "fmaf(AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j))"),
    "ir_residual_sign": ("for (int j = 0; j < n; ++j) r = fma(-AT(a, n, i, j), x[j], r);",
                         "for (int j = 0; j < n; ++j) r = fma(AT(a, n, i, j), x[j], r);"),
    "ir_correction_replaces": ("x[i] = x[i] + (double)y[i];", "x[i] = (double)y[i];"),
    "ir_one_correction_only": ("if (it == 3) return 1;", "if (it == 1) return 1;"),
    "ir_absolute_stop": ("if (rnrm <= xnrm * cte) {", "if (rnrm <= cte) {"),
}


# --------------------------- pin checks ----------------------------------

def _f(v):
    if isinstance(v, str) and v.startswith("2^"):
        return 2.0 ** int(v[2:])
    from fractions import Fraction
    return float(Fraction(v)) if isinstance(v, str) else float(v)


def pin_golden(lib):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = np.array([[_f(v) for v in row] for row in c["A"]])[None]
        b = np.array([_f(v) for v in c["b"]])[None]
        x, ipiv, info, _, LU = oracle.gesv(A, b, want_lu=True, lib=lib)
        assert list(ipiv[0]) == c["ipiv"] and info[0] == c["info"]
        n = A.shape[-1]
        L = np.tril(LU[0], -1) + np.eye(n)
        Lg = np.array([[_f(v) for v in row] for row in c["L"]])
        Ug = np.array([[_f(v) for v in row] for row in c["U"]])
        assert np.allclose(L, Lg, rtol=4 * EPS, atol=0)
        assert np.allclose(np.triu(LU[0]), Ug, rtol=8 * EPS, atol=8 * EPS * np.abs(Ug).max())
        if c["x"] is not None:
            assert np.allclose(x[0], [_f(v) for v in c["x"]], rtol=1e-14, atol=1e-14)


def pin_reconstruction_and_errors(lib):
    for n in (5, 12):
        A, x_true, b, kappa = inputs.kappa_systems(n, 40, 500 + n)
        x, ipiv, info, _, LU = oracle.gesv(A, b, want_lu=True, lib=lib)
        for s in range(40):
            order = list(range(n))
            for k, p in enumerate(ipiv[s]):
                order[k], order[p - 1] = order[p - 1], order[k]
            L = np.tril(LU[s], -1) + np.eye(n)
            U = np.triu(LU[s])
            E = np.abs(A[s][order] - L @ U)
            assert (E <= 2 * n * EPS * (np.abs(L) @ np.abs(U)) + 1e-300).all()
        fe = np.abs(x - x_true).max(axis=1) / np.abs(x_true).max(axis=1)
        assert (fe <= 1e-12 * kappa).all()


def pin_singular(lib):
    A = np.zeros((1, 4, 4))
    _, ipiv, info, _ = oracle.getrf(A, lib=lib)
    assert info[0] == 1 and list(ipiv[0]) == [1, 2, 3, 4]


def pin_norton(lib):
    prm = oracle.norton_params()
    sig0, deps = inputs.norton_points(40, 600)
    r = oracle.newton_norton(prm, sig0, deps, rtol=1e-13, max_iter=30, lib=lib)
    assert (r["status"] == 0).all()
    for p in range(40):
        de, dp = radial_return(prm, sig0[p], deps[p])
        assert abs(r["x"][p, 6] - dp) <= 1e-10 * abs(dp)
        assert np.allclose(r["x"][p, :6], de, rtol=1e-10, atol=1e-10 * np.abs(de).max())
    # iteration counts: a correct Newton from the elastic predictor needs a
    # handful of solves on this workload (quadratic convergence)
    r10 = oracle.newton_norton(prm, sig0, deps, rtol=1e-10, max_iter=20, lib=lib)
    assert r10["iterations"].max() <= 9 and r10["iterations"].min() >= 3
    x = np.concatenate([deps[0], [5e-4]])
    F, J, _ = oracle.norton_eval(prm, sig0[0], deps[0], x, lib=lib)
    for j in range(7):
        xp, xm = x.copy(), x.copy()
        xp[j] += 1e-9
        xm[j] -= 1e-9
        col = (oracle.norton_eval(prm, sig0[0], deps[0], xp, lib=lib)[0]
               - oracle.norton_eval(prm, sig0[0], deps[0], xm, lib=lib)[0]) / 2e-9
        assert np.allclose(J[:, j], col, rtol=1e-5, atol=1e-6 * np.abs(J).max())


def pin_tanh(lib):
    A, c, b = inputs.tanh_points(1, 50, 700)
    r = oracle.newton_tanh(A, c, b, rtol=1e-14, max_iter=40, lib=lib)
    for p in range(50):
        a, cc, bb = A[p, 0, 0], c[p, 0], b[p, 0]
        lo, hi = -1e3, 1e3
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if a * mid + cc * math.tanh(mid) - bb < 0:
                lo = mid
            else:
                hi = mid
        assert abs(r["x"][p, 0] - mid) <= 1e-12 * max(1.0, abs(mid))
    A, c, b = inputs.tanh_points(7, 20, 701)
    r = oracle.newton_tanh(A, np.zeros_like(c), b, lib=lib)
    assert (r["iterations"] == 1).all()
    r = oracle.newton_tanh(A, c, b, rtol=0.0, max_iter=4, lib=lib)
    assert (r["iterations"] == 4).all() and (r["status"] == 1).all()
    # the stop test is relative: scaling F and J by 2^e changes no decision
    r1 = oracle.newton_tanh(A, c, b, lib=lib)
    for e in (-30, 30):
        r2 = oracle.newton_tanh(np.ldexp(A, e), np.ldexp(c, e), np.ldexp(b, e), lib=lib)
        assert np.array_equal(r1["iterations"], r2["iterations"])
        assert np.array_equal(r1["x"], r2["x"])


PINS = [pin_golden, pin_reconstruction_and_errors, pin_singular, pin_norton, pin_tanh, pin_tangent, pin_tiled, *IR_PINS]


def failing_pins(lib):
    failed = []
    for pin in PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    return failed


def test_real_oracle_passes_every_pin():
    assert failing_pins(oracle.load()) == []


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, mutant_dir):
    old, new = MUTATIONS[name]
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/present"
    path_c = os.path.join(mutant_dir, f"{name}.c")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    path_so = os.path.join(mutant_dir, f"lib{name}.so")
    cmd = ["gcc", *obuild.BASE_FLAGS, path_c, "-o", path_so, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = oracle.load(path_so)
    assert failing_pins(lib), f"planted mistake '{name}' passed every pin"
