"""ctypes binding of the C ABI in include/tinylu.h (argument marshalling only).

Every function has the C name and argument order; tensor arguments may be
torch tensors (their data_ptr() is passed), raw integer addresses, or None
for a NULL pointer.  `stream` defaults to torch's current CUDA stream.  Every
step of the computation runs in libtinylu.so: importing this module raises
if the library has not been built -- there is no fallback.
"""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtinylu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the CUDA library is the only compute path)")

_lib = C.CDLL(LIB_PATH)

TL_OK, TL_ERR_INVALID_ARG, TL_ERR_CUDA, TL_ERR_NO_MEMORY, TL_ERR_UNSUPPORTED, TL_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
TL_LAYOUT_PER_SYSTEM, TL_LAYOUT_INTERLEAVED = 0, 1
TL_PREC_FP64, TL_PREC_FP32_IR = 0, 1
TL_RAGGED_PERSISTENT, TL_RAGGED_PER_SIZE = 0, 1
TL_LAW_NORTON, TL_LAW_TANH = 0, 1
TL_NEWTON_CONVERGED, TL_NEWTON_MAX_ITER, TL_NEWTON_SINGULAR, TL_NEWTON_NONFINITE = 0, 1, 2, 3
TL_MAX_N = 32


class tl_law(C.Structure):
    _fields_ = [("id", C.c_int32), ("n", C.c_int32), ("params", C.c_double * 6)]


_vp = C.c_void_p
_i64 = C.c_int64
_int = C.c_int

TL_REQ_NEWTON, TL_REQ_SOLVE = 0, 1


class tl_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("law", tl_law), ("count", C.c_int64),
                ("ld_in", C.c_int64), ("in_", _vp), ("rhs", _vp), ("x", _vp), ("aux", _vp), ("i1", _vp), ("i2", _vp)]


class tl_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("slots", C.c_int32), ("max_points_per_tick", C.c_int64),
                ("rtol", C.c_double), ("max_iter", C.c_int32)]


class tl_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("ticks", C.c_int64),
                ("points", C.c_int64), ("arena_high_water", C.c_size_t), ("host_enqueue_s", C.c_double),
                ("kernel_busy_s", C.c_double)]

_SIGS = {
    "tl_create": ([C.POINTER(_vp)], _int),
    "tl_destroy": ([_vp], _int),
    "tl_status_string": ([_int], C.c_char_p),
    "tl_last_cuda_error": ([_vp, C.POINTER(_int)], _int),
    "tl_last_bad_arg": ([_vp], _int),
    "tl_getrf_batched": ([_vp, _int, _vp, _int, _i64, _vp, _vp, _i64, _vp], _int),
    "tl_getrs_batched": ([_vp, _int, _int, _vp, _vp, _int, _i64, _vp, _i64, _vp], _int),
    "tl_gesv_batched": ([_vp, _int, _vp, _vp, _vp, _vp, _vp, _vp, _int, _i64, _i64, _vp], _int),
    "tl_lupp_solve_batched": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _int, _vp, _vp], _int),
    "tl_lupp_solve_batched_noalloc": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _int),
    "tl_newton_integrate": ([_vp, C.POINTER(tl_law), _i64, _vp, _vp, _vp, _vp, _vp, C.c_double, _int, _vp], _int),
    "tl_newton_integrate_tangent": ([_vp, C.POINTER(tl_law), _i64, _vp, _vp, _vp, _vp, _vp, _vp, C.c_double,
                                     _int, _vp], _int),
    "tl_newton_integrate_cpu_driven": ([_vp, C.POINTER(tl_law), _i64, _vp, _vp, _vp, _vp, _vp, C.c_double, _int,
                                        _vp], _int),
    "tl_gesv_batched_tilepiv": ([_vp, _int, _int, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _int, _i64, _i64, _vp],
                                _int),
    "tl_autotune": ([_vp, _int, _int, _int, C.c_char_p], _int),
    "tl_server_create": ([_vp, C.POINTER(tl_server_config), C.POINTER(_vp)], _int),
    "tl_server_submit": ([_vp, C.POINTER(tl_request), C.POINTER(_i64)], _int),
    "tl_server_test": ([_vp, _i64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)], _int),
    "tl_server_wait": ([_vp, _i64, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double)], _int),
    "tl_server_stats_get": ([_vp, C.POINTER(tl_server_stats)], _int),
    "tl_server_pause": ([_vp, _int], _int),
    "tl_server_destroy": ([_vp], _int),
    "tl_dispatch_set": ([_vp, _int, _int, _int, _int], _int),
    "tl_ragged_set_mode": ([_vp, _int], _int),
    "tl_autotune_ragged": ([_vp, _int, _int, C.c_char_p], _int),
    "tl_ragged_dispatch_set": ([_vp, _int, _int, _int], _int),
    "tl_ragged_dispatch_get": ([_vp, _int, C.POINTER(_int), C.POINTER(_int)], _int),
    "tl_check_bounds_violations": ([C.POINTER(C.c_ulonglong)], _int),
    "tl_measure_fma_peak": ([_vp, _int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), _vp],
                            _int),
    "tl_dispatch_get": ([_vp, _int, _int, C.POINTER(_int), C.POINTER(_int)], _int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _p(x):
    """Pointer of a tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


class TinyLUError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        msg = _lib.tl_status_string(status).decode()
        super().__init__(f"{fn}: {msg}{detail}")
        self.status = status


def check(fn, status, h=None):
    if status == TL_OK:
        return status
    detail = ""
    if h is not None:
        if status == TL_ERR_INVALID_ARG:
            detail = f" (argument {tl_last_bad_arg(h)})"
        elif status == TL_ERR_CUDA:
            e = C.c_int(0)
            _lib.tl_last_cuda_error(h, C.byref(e))
            detail = f" (cudaError {e.value})"
    raise TinyLUError(fn, status, detail)


# ---------------------------------------------------------------------------
# C ABI entry points (same names)
# ---------------------------------------------------------------------------

def tl_create():
    h = _vp()
    check("tl_create", _lib.tl_create(C.byref(h)))
    return h


def tl_destroy(h):
    return _lib.tl_destroy(h)


def tl_status_string(status):
    return _lib.tl_status_string(status).decode()


def tl_last_cuda_error(h):
    e = C.c_int(0)
    _lib.tl_last_cuda_error(h, C.byref(e))
    return e.value


def tl_last_bad_arg(h):
    return _lib.tl_last_bad_arg(h)


def tl_getrf_batched(h, n, A, layout, ld_batch, ipiv, info, batch, stream=None):
    return _lib.tl_getrf_batched(h, n, _p(A), layout, ld_batch, _p(ipiv), _p(info), batch, _stream(stream))


def tl_getrs_batched(h, n, nrhs, LU, ipiv, layout, ld_batch, B, batch, stream=None):
    return _lib.tl_getrs_batched(h, n, nrhs, _p(LU), _p(ipiv), layout, ld_batch, _p(B), batch, _stream(stream))


def tl_gesv_batched(h, n, A, LU_out, b, x, ipiv, info, layout, ld_batch, batch, stream=None):
    return _lib.tl_gesv_batched(h, n, _p(A), _p(LU_out), _p(b), _p(x), _p(ipiv), _p(info), layout, ld_batch,
                                batch, _stream(stream))


def tl_lupp_solve_batched(h, batch, n, a_off, A, b_off, b, x, piv_off, ipiv, info, prec=TL_PREC_FP64,
                          refine_steps=None, stream=None):
    return _lib.tl_lupp_solve_batched(h, batch, _p(n), _p(a_off), _p(A), _p(b_off), _p(b), _p(x), _p(piv_off),
                                      _p(ipiv), _p(info), prec, _p(refine_steps), _stream(stream))


def tl_lupp_solve_batched_noalloc(h, batch, n, a_off, A, b_off, b, x, piv_off, ipiv, info, stream=None):
    return _lib.tl_lupp_solve_batched_noalloc(h, batch, _p(n), _p(a_off), _p(A), _p(b_off), _p(b), _p(x),
                                              _p(piv_off), _p(ipiv), _p(info), _stream(stream))


TL_NOALLOC_MAX_BATCH = 1 << 20


def make_law(law_id, n, params=()):
    law = tl_law()
    law.id = law_id
    law.n = n
    for i, v in enumerate(params):
        law.params[i] = float(v)
    return law


def tl_newton_integrate(h, law, npoints, inputs, x, outputs, iterations, status, rtol, max_iter, stream=None):
    return _lib.tl_newton_integrate(h, C.byref(law), npoints, _p(inputs), _p(x), _p(outputs), _p(iterations),
                                    _p(status), rtol, max_iter, _stream(stream))


def tl_newton_integrate_tangent(h, law, npoints, inputs, x, outputs, tangent, iterations, status, rtol, max_iter,
                                stream=None):
    return _lib.tl_newton_integrate_tangent(h, C.byref(law), npoints, _p(inputs), _p(x), _p(outputs), _p(tangent),
                                            _p(iterations), _p(status), rtol, max_iter, _stream(stream))


def tl_newton_integrate_cpu_driven(h, law, npoints, inputs, x, outputs, iterations, status, rtol, max_iter,
                                   stream=None):
    return _lib.tl_newton_integrate_cpu_driven(h, C.byref(law), npoints, _p(inputs), _p(x), _p(outputs),
                                               _p(iterations), _p(status), rtol, max_iter, _stream(stream))


def tl_gesv_batched_tilepiv(h, n, tile, threshold, A, LU_out, b, x, ipiv, info, layout, ld_batch, batch,
                            stream=None):
    return _lib.tl_gesv_batched_tilepiv(h, n, tile, threshold, _p(A), _p(LU_out), _p(b), _p(x), _p(ipiv), _p(info),
                                        layout, ld_batch, batch, _stream(stream))


def tl_autotune(h, n_min, n_max, layout, table_path=None):
    return _lib.tl_autotune(h, n_min, n_max, layout, table_path.encode() if table_path else None)


def tl_check_bounds_violations():
    """Returns (status, violations); TL_ERR_UNSUPPORTED in this (unchecked)
    library -- libtinylu_checked.so carries the checks."""
    v = C.c_ulonglong(0)
    st = _lib.tl_check_bounds_violations(C.byref(v))
    return st, v.value


def tl_autotune_ragged(h, n_min, n_max, table_path=None):
    return _lib.tl_autotune_ragged(h, n_min, n_max, table_path.encode() if table_path else None)


def tl_ragged_dispatch_set(h, n, lanes=0, mixed_route=-1):
    return _lib.tl_ragged_dispatch_set(h, n, lanes, mixed_route)


def tl_ragged_dispatch_get(h, n):
    """Returns (status, lanes, refines)."""
    lanes, refines = C.c_int(0), C.c_int(0)
    st = _lib.tl_ragged_dispatch_get(h, n, C.byref(lanes), C.byref(refines))
    return st, lanes.value, refines.value


def tl_ragged_set_mode(h, mode):
    return _lib.tl_ragged_set_mode(h, mode)


def tl_dispatch_set(h, n, layout, variant, block=0):
    return _lib.tl_dispatch_set(h, n, layout, variant, block)


def tl_dispatch_get(h, n, layout):
    """Returns (status, variant, block)."""
    v, b = C.c_int(0), C.c_int(0)
    st = _lib.tl_dispatch_get(h, n, layout, C.byref(v), C.byref(b))
    return st, v.value, b.value


def tl_measure_fma_peak(h, bits=64, stream=None):
    """Returns (status, TFLOP/s, FMA lanes per SM per clock, SM MHz)."""
    tf, per_clk, mhz = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    st = _lib.tl_measure_fma_peak(h, bits, C.byref(tf), C.byref(per_clk), C.byref(mhz), _stream(stream))
    return st, tf.value, per_clk.value, mhz.value


def make_request(kind, count, in_, x, i1, i2, law=None, n=0, rhs=None, aux=None, ld_in=0):
    """A tl_request over host arrays (numpy arrays or raw addresses)."""
    r = tl_request()
    r.kind = kind
    r.n = n
    if law is not None:
        r.law = law
    r.count = count
    r.ld_in = ld_in
    r.in_, r.rhs, r.x, r.aux, r.i1, r.i2 = (_p(v) for v in (in_, rhs, x, aux, i1, i2))
    return r


def tl_server_create(h, budget_bytes, slots=4, max_points_per_tick=1 << 20, rtol=1e-10, max_iter=20):
    """Returns (status, server handle)."""
    cfg = tl_server_config(budget_bytes, slots, max_points_per_tick, rtol, max_iter)
    out = _vp()
    st = _lib.tl_server_create(h, C.byref(cfg), C.byref(out))
    return st, out.value


def tl_server_submit(s, req):
    """Returns (status, request id)."""
    rid = _i64(0)
    st = _lib.tl_server_submit(s, C.byref(req), C.byref(rid))
    return st, rid.value


def tl_server_test(s, rid):
    """Returns (status, done, request status, latency in s)."""
    done, rs, lat = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    st = _lib.tl_server_test(s, rid, C.byref(done), C.byref(rs), C.byref(lat))
    return st, done.value, rs.value, lat.value


def tl_server_wait(s, rid, timeout_s=60.0):
    """Returns (status, request status, latency in s)."""
    rs, lat = C.c_int32(0), C.c_double(0.0)
    st = _lib.tl_server_wait(s, rid, timeout_s, C.byref(rs), C.byref(lat))
    return st, rs.value, lat.value


def tl_server_stats_get(s):
    out = tl_server_stats()
    st = _lib.tl_server_stats_get(s, C.byref(out))
    return st, {k: getattr(out, k) for k, _ in tl_server_stats._fields_}


def tl_server_pause(s, paused=True):
    return _lib.tl_server_pause(s, 1 if paused else 0)


def tl_server_destroy(s):
    return _lib.tl_server_destroy(s)


def variant_id(lanes, shared=False, walk=False):
    """Dispatch id of a kernel variant: lanes per system + 100 for the
    shared-memory storage (+ 200 instead for the shared-memory solver whose
    2..8 lanes walk the trailing update element by element)."""
    return lanes + (200 if walk else 100 if shared else 0)


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib
