"""CPU oracle for tiny batched LUpp and the per-point Newton loop.

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The CUDA library
never imports, links or calls it, and this package imports nothing from the
CUDA library: the two share no code.

Everything here is a thin numpy <-> C marshalling layer over
`tinylu_oracle.c`, which holds all arithmetic (fp64, explicit fma, no
contraction).  Matrices on the numpy side are indexed mathematically,
``A[s, i, j] = a_ij`` for system ``s``; the wrapper passes column-major
copies to C.

Passages followed (paper: "Accelerating the Solving of Many Tiny General
Linear Systems on GPUs: Application to Constitutive Laws"):
  * getrf / getrs / gesv -- Sec. 2.2 (Gaussian elimination with partial
    pivoting, PA = LU, then Ly = Pb and Ux = y).
  * newton_* -- Sec. 2.1, Eqs. (1)-(3), per point as in Algorithm 2.
  * norton_eval -- the Norton law of Sec. 4.3 (equations not printed in the
    paper; standard implicit J2 + Norton form in Mandel notation).
  * tanh_eval -- synthetic law F(x) = A x + c*tanh(x) - b.
  * norton_tangent -- consistent tangent operator at a converged state
    (Sec. 4.3, the multi-right-hand-side solve after convergence).
  * getrf_tiled -- tile-local pivoting of the paper's Tiled solvers
    (Sec. 3.2), with the acceptance threshold of Sec. 4.1.
  * sgetrf / ir_gesv -- binary32 factorization and binary64 iterative
    refinement (not in the paper: the published scheme of Langou et al.
    2006, as LAPACK's dsgesv, with every operation's format and order
    fixed).

Parity pins live in tests/test_oracle_*.py; every function above is pinned
there by something other than itself (closed forms, exact rational
elimination, LAPACK, invariants).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

NEWTON_CONVERGED, NEWTON_MAXITER, NEWTON_SINGULAR, NEWTON_NONFINITE = 0, 1, 2, 3

_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)


def _ptr(a, t=_d):
    return a.ctypes.data_as(t) if a is not None else None


def _declare(lib):
    lib.orc_max_threads.restype = C.c_int
    lib.orc_getrf.restype = C.c_int
    lib.orc_getrf.argtypes = [C.c_int, _d, _i32, _d]
    lib.orc_getrs.restype = None
    lib.orc_getrs.argtypes = [C.c_int, _d, _i32, _d]
    lib.orc_gesv_batch.restype = None
    lib.orc_gesv_batch.argtypes = [C.c_int, C.c_int64, _d, _d, _d, _i32, _i32, _d, _d, C.c_int]
    lib.orc_getrf_batch.restype = None
    lib.orc_getrf_batch.argtypes = [C.c_int, C.c_int64, _d, _i32, _i32, _d, C.c_int]
    lib.orc_getrs_batch.restype = None
    lib.orc_getrs_batch.argtypes = [C.c_int, C.c_int64, _d, _i32, _d, C.c_int]
    lib.orc_getrf_tiled_batch.restype = None
    lib.orc_getrf_tiled_batch.argtypes = [C.c_int, C.c_int64, _d, _i32, _i32, _i32, C.c_int, C.c_double, C.c_int]
    lib.orc_sgetrf.restype = C.c_int
    lib.orc_sgetrf.argtypes = [C.c_int, C.POINTER(C.c_float), _i32]
    lib.orc_ir_gesv_batch.restype = None
    lib.orc_ir_gesv_batch.argtypes = [C.c_int, C.c_int64, _d, _d, _d, _i32, _i32, _i32, C.c_int]
    lib.orc_norton_tangent.restype = C.c_int
    lib.orc_norton_tangent.argtypes = [_d, _d, _d, _d, _d]
    lib.orc_norton_eval.restype = None
    lib.orc_norton_eval.argtypes = [_d, _d, _d, _d, _d, _d, _d]
    lib.orc_tanh_eval.restype = None
    lib.orc_tanh_eval.argtypes = [C.c_int, _d, _d, _d, _d, _d, _d]
    lib.orc_newton_norton_batch.restype = None
    lib.orc_newton_norton_batch.argtypes = [_d, C.c_int64, _d, _d, _d, C.c_int, _i32, _i32, _d,
                                            _d, C.c_double, C.c_int, C.c_int]
    lib.orc_newton_tanh_batch.restype = None
    lib.orc_newton_tanh_batch.argtypes = [C.c_int, C.c_int64, _d, _d, _d, _d, C.c_int, _i32,
                                          _i32, _d, C.c_double, C.c_int, C.c_int]
    return lib


def load(path=None):
    """Load the oracle library (building it first if needed).

    `path` selects another build of the same source (tests use this for
    variants with a planted mistake)."""
    global _LIB
    if path is not None:
        return _declare(C.CDLL(path))
    if _LIB is None:
        _LIB = _declare(C.CDLL(_build.build()))
    return _LIB


def max_threads(lib=None):
    return (lib or load()).orc_max_threads()


def _colmajor(A):
    A = np.asarray(A, dtype=np.float64)
    return np.ascontiguousarray(A.transpose(0, 2, 1))


def _mathidx(Acm):
    return np.ascontiguousarray(Acm.transpose(0, 2, 1))


def getrf(A, nthreads=0, lib=None):
    """LUpp of each A[s] (Sec. 2.2).  Returns (LU, ipiv, info, min_gap).

    LU[s] holds L (unit diagonal, strictly below) and U; ipiv is 1-based
    LAPACK sequential interchanges; info as LAPACK (k+1 for the first zero
    pivot), -1 for a non-finite input entry; min_gap is the smallest relative
    pivot separation (near-tie flag)."""
    lib = lib or load()
    Acm = _colmajor(A)
    batch, n = Acm.shape[0], Acm.shape[1]
    ipiv = np.zeros((batch, n), np.int32)
    info = np.zeros(batch, np.int32)
    gap = np.zeros(batch, np.float64)
    lib.orc_getrf_batch(n, batch, _ptr(Acm), _ptr(ipiv, _i32), _ptr(info, _i32), _ptr(gap), nthreads)
    return _mathidx(Acm), ipiv, info, gap


def getrf_tiled(A, tile, threshold=1e-10, nthreads=0, lib=None):
    """LU with tile-local pivoting (Sec. 3.2, Tiled solvers): the pivot is
    sought in the diagonal tile of `tile` rows and below it only when the
    in-tile best is under `threshold`.  Returns (LU, ipiv, info,
    out_of_tile) where out_of_tile counts the steps that looked below the
    tile."""
    lib = lib or load()
    Acm = _colmajor(A)
    batch, n = Acm.shape[0], Acm.shape[1]
    ipiv = np.zeros((batch, n), np.int32)
    info = np.zeros(batch, np.int32)
    oot = np.zeros(batch, np.int32)
    lib.orc_getrf_tiled_batch(n, batch, _ptr(Acm), _ptr(ipiv, _i32), _ptr(info, _i32), _ptr(oot, _i32), tile,
                              threshold, nthreads)
    return _mathidx(Acm), ipiv, info, oot


def getrs(LU, ipiv, B, nthreads=0, lib=None):
    """Solve with the factors of getrf (Sec. 2.2).  B is (batch, n)."""
    lib = lib or load()
    LUcm = _colmajor(LU)
    batch, n = LUcm.shape[0], LUcm.shape[1]
    X = np.ascontiguousarray(np.asarray(B, np.float64).reshape(batch, n)).copy()
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.orc_getrs_batch(n, batch, _ptr(LUcm), _ptr(piv, _i32), _ptr(X), nthreads)
    return X


def gesv(A, b, want_lu=False, nthreads=0, lib=None):
    """Factor and solve A[s] x[s] = b[s].  Returns (x, ipiv, info, min_gap[, LU])."""
    lib = lib or load()
    Acm = _colmajor(A)
    batch, n = Acm.shape[0], Acm.shape[1]
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(batch, n))
    x = np.empty((batch, n), np.float64)
    ipiv = np.zeros((batch, n), np.int32)
    info = np.zeros(batch, np.int32)
    gap = np.zeros(batch, np.float64)
    lu = np.empty_like(Acm) if want_lu else None
    lib.orc_gesv_batch(n, batch, _ptr(Acm), _ptr(b), _ptr(x), _ptr(ipiv, _i32), _ptr(info, _i32),
                       _ptr(lu), _ptr(gap), nthreads)
    if want_lu:
        return x, ipiv, info, gap, _mathidx(lu)
    return x, ipiv, info, gap


def sgetrf(A, lib=None):
    """Binary32 LUpp of each A[s] (float32 input, math-indexed) with the
    steps of getrf; stops at a pivot outside [FLT_MIN, Inf).  Returns
    (LU (float32), ipiv, ok) where ok[s] is False for a stopped system."""
    lib = lib or load()
    Acm = np.ascontiguousarray(np.asarray(A, np.float32).transpose(0, 2, 1))
    batch, n = Acm.shape[0], Acm.shape[1]
    ipiv = np.zeros((batch, n), np.int32)
    ok = np.zeros(batch, bool)
    for s in range(batch):
        ok[s] = lib.orc_sgetrf(n, Acm[s].ctypes.data_as(C.POINTER(C.c_float)),
                               ipiv[s].ctypes.data_as(_i32)) == 0
    return np.ascontiguousarray(Acm.transpose(0, 2, 1)), ipiv, ok


def ir_gesv(A, b, nthreads=0, lib=None):
    """Mixed-precision solve of every A[s] x[s] = b[s]: binary32 factor,
    binary64 iterative refinement (at most 3 corrections), binary64 LUpp
    fallback.  Returns (x, ipiv, info, steps); steps[s] = -1 marks a system
    solved by gesv instead."""
    lib = lib or load()
    Acm = _colmajor(A)
    batch, n = Acm.shape[0], Acm.shape[1]
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(batch, n))
    x = np.empty((batch, n), np.float64)
    ipiv = np.zeros((batch, n), np.int32)
    info = np.zeros(batch, np.int32)
    steps = np.zeros(batch, np.int32)
    lib.orc_ir_gesv_batch(n, batch, _ptr(Acm), _ptr(b), _ptr(x), _ptr(ipiv, _i32), _ptr(info, _i32),
                          _ptr(steps, _i32), nthreads)
    return x, ipiv, info, steps


def norton_params(E=200000.0, nu=0.3, A=1e-12, m=4, dt=1.0):
    """Parameter vector (E, nu, A, m, dt) of the Norton law."""
    return np.array([E, nu, A, float(m), dt], np.float64)


def norton_eval(prm, sig0, deps, x, lib=None):
    """Residual F (7) and Jacobian J (7x7, math-indexed) of the Norton law at
    one point; also the end-of-step stress."""
    lib = lib or load()
    prm = np.ascontiguousarray(prm, np.float64)
    sig0 = np.ascontiguousarray(sig0, np.float64)
    deps = np.ascontiguousarray(deps, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    F = np.empty(7)
    Jcm = np.empty(49)
    sig = np.empty(6)
    lib.orc_norton_eval(_ptr(prm), _ptr(sig0), _ptr(deps), _ptr(x), _ptr(F), _ptr(Jcm), _ptr(sig))
    return F, Jcm.reshape(7, 7).T.copy(), sig


def norton_tangent(prm, sig0, deps, x, lib=None):
    """Consistent tangent dsig/ddeps (6x6, math-indexed) of the Norton law
    at the converged state x of one point (Sec. 4.3), and the info of the
    Jacobian's factorization."""
    lib = lib or load()
    prm = np.ascontiguousarray(prm, np.float64)
    sig0 = np.ascontiguousarray(sig0, np.float64)
    deps = np.ascontiguousarray(deps, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    Dcm = np.empty(36)
    info = lib.orc_norton_tangent(_ptr(prm), _ptr(sig0), _ptr(deps), _ptr(x), _ptr(Dcm))
    return Dcm.reshape(6, 6).T.copy(), info


def tanh_eval(A, c, b, x, lib=None):
    """Residual and Jacobian of F(x) = A x + c*tanh(x) - b at one point."""
    lib = lib or load()
    n = len(x)
    Acm = np.ascontiguousarray(np.asarray(A, np.float64).T)
    c = np.ascontiguousarray(c, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    F = np.empty(n)
    Jcm = np.empty(n * n)
    lib.orc_tanh_eval(n, _ptr(Acm), _ptr(c), _ptr(b), _ptr(x), _ptr(F), _ptr(Jcm))
    return F, Jcm.reshape(n, n).T.copy()


def newton_norton(prm, sig0, deps, x0=None, rtol=1e-10, max_iter=20, nthreads=0, lib=None):
    """Per-point Newton on the Norton law (Algorithm 2, Eqs. 1-3).

    sig0, deps: (npoints, 6) Mandel components.  x0 None -> elastic
    predictor (deps, 0).  Returns dict(x, iterations, status, sig, rmin_ratio)."""
    lib = lib or load()
    prm = np.ascontiguousarray(prm, np.float64)
    sig0 = np.ascontiguousarray(sig0, np.float64)
    deps = np.ascontiguousarray(deps, np.float64)
    npts = sig0.shape[0]
    if x0 is None:
        x = np.zeros((npts, 7))
        init = 1
    else:
        x = np.ascontiguousarray(x0, np.float64).copy()
        init = 0
    it = np.zeros(npts, np.int32)
    st = np.zeros(npts, np.int32)
    sig = np.empty((npts, 6))
    rr = np.empty(npts)
    lib.orc_newton_norton_batch(_ptr(prm), npts, _ptr(sig0), _ptr(deps), _ptr(x), init,
                                _ptr(it, _i32), _ptr(st, _i32), _ptr(sig), _ptr(rr), rtol,
                                max_iter, nthreads)
    return dict(x=x, iterations=it, status=st, sig=sig, rmin_ratio=rr)


def newton_tanh(A, c, b, x0=None, rtol=1e-10, max_iter=20, nthreads=0, lib=None):
    """Per-point Newton on F(x) = A x + c*tanh(x) - b, all points of one n.

    A: (npoints, n, n) math-indexed; c, b: (npoints, n).  x0 None -> 0."""
    lib = lib or load()
    Acm = _colmajor(A)
    npts, n = Acm.shape[0], Acm.shape[1]
    c = np.ascontiguousarray(c, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    if x0 is None:
        x = np.zeros((npts, n))
        init = 1
    else:
        x = np.ascontiguousarray(x0, np.float64).copy()
        init = 0
    it = np.zeros(npts, np.int32)
    st = np.zeros(npts, np.int32)
    rr = np.empty(npts)
    lib.orc_newton_tanh_batch(n, npts, _ptr(Acm), _ptr(c), _ptr(b), _ptr(x), init, _ptr(it, _i32),
                              _ptr(st, _i32), _ptr(rr), rtol, max_iter, nthreads)
    return dict(x=x, iterations=it, status=st, rmin_ratio=rr)


def library_path():
    return _build.LIB if os.path.exists(_build.LIB) else _build.build()
