"""CPU oracle for the k-register Gumbel-Max sketch -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` /
``--impl reference`` leg may import this package.  The product path (the CUDA
library and its binding) never touches it, and the two share no code.

The arithmetic lives in ``gm_oracle.c`` (plain C, FP64, unpruned full stream);
this module only marshals numpy arrays through ctypes.  What each routine
computes, and which passage of the paper (Zhang et al., arXiv 2302.05176) it
follows, is documented in the C file:

* ``sketch``          -- Eq. sjv / Eq. yjpi over all k arrivals of Eq. biz_dis.
* ``fastgm_alg1``     -- Algorithm 1 (FastSearch + FastPrune), host cross-check.
* ``stream_fastgm``   -- Algorithm 2 (Stream-FastGM).
* ``jaccard`` / ``cardinality`` / ``merge`` -- Sec. 1 estimators, Sec. 2.3 union.
* ``fastsearch_budgets`` -- R_i = ceil(R v_i / sum v) (Sec. 2.1 example, Eq. exiri).
"""
import contextlib
import ctypes
import os
import concurrent.futures as _cf

import numpy as np

from . import build as _build

_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.gmo_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.gmo_philox4x32_10.restype = None
        L.gmo_uniform_from_words.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.gmo_uniform_from_words.restype = ctypes.c_double
        L.gmo_randint_from_words.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32]
        L.gmo_randint_from_words.restype = ctypes.c_int32
        L.gmo_exact_sum.argtypes = [_f64p, ctypes.c_int64, _f64p]
        L.gmo_arrivals.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_int32, _f64p, _i32p]
        L.gmo_sketch_rows.argtypes = [_i64p, _i32p, _f64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                      _i32p, _f64p, _f64p, _i32p]
        L.gmo_fastsearch_budgets.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, _i64p]
        L.gmo_fastgm_alg1.argtypes = [_i32p, _f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_int32, _i32p, _f64p, _i64p, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]
        L.gmo_stream_fastgm.argtypes = [_i32p, _f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        _i32p, _f64p, _i64p]
        L.gmo_jaccard.argtypes = [_i32p, _i32p, ctypes.c_int64, ctypes.c_int32, _f64p]
        L.gmo_cardinality.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int32, _f64p]
        L.gmo_merge.argtypes = [_i32p, _f64p, _i32p, _f64p, ctypes.c_int64, _i32p, _f64p]
        L.gmo_set_mutation.argtypes = [ctypes.c_int]
        L.gmo_set_mutation.restype = None
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


@contextlib.contextmanager
def mutation(m):
    """Plant a known mistake in the oracle (tests use this to show the pins bite)."""
    lib().gmo_set_mutation(int(m))
    try:
        yield
    finally:
        lib().gmo_set_mutation(0)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().gmo_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def uniform_from_words(w0, w1):
    return lib().gmo_uniform_from_words(int(w0), int(w1))


def randint_from_words(w2, w3, z, k):
    return lib().gmo_randint_from_words(int(w2), int(w3), int(z), int(k))


def exact_sum(t):
    a = np.ascontiguousarray(t, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().gmo_exact_sum(_p(a, _f64p), a.size, ctypes.byref(out)), "exact_sum")
    return out.value


def arrivals(elem_id, v, k, seed, n_steps=None):
    """First n_steps (default k) arrival times and servers of one element."""
    n = k if n_steps is None else n_steps
    b = np.zeros(n, dtype=np.float64)
    c = np.zeros(n, dtype=np.int32)
    _check(lib().gmo_arrivals(int(elem_id), float(v), int(k), int(seed), int(n), _p(b, _f64p), _p(c, _i32p)),
           "arrivals")
    return b, c


def sketch(row_ptr, ids, w, k, seed, runner_up=False):
    """Unpruned sketch of CSR rows -> (s [n_rows, k] int32, y [n_rows, k] f64); with
    runner_up=True also (y2, s2): per register the second candidate in (time, id)
    order over distinct elements (+inf / -1 if there is none)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ii = np.ascontiguousarray(ids, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    n_rows = rp.size - 1
    s = np.zeros((n_rows, k), dtype=np.int32)
    y = np.zeros((n_rows, k), dtype=np.float64)
    y2 = np.zeros((n_rows, k), dtype=np.float64) if runner_up else None
    s2 = np.zeros((n_rows, k), dtype=np.int32) if runner_up else None
    rc = lib().gmo_sketch_rows(_p(rp, _i64p), _p(ii, _i32p), _p(ww, _f64p), n_rows, int(k), int(seed),
                               _p(s, _i32p), _p(y, _f64p), _p(y2, _f64p) if runner_up else None,
                               _p(s2, _i32p) if runner_up else None)
    _check(rc, "sketch")
    return (s, y, y2, s2) if runner_up else (s, y)


def sketch_rows_parallel(row_ptr, ids, w, k, seed, rows, threads=None, runner_up=False):
    """Sketch the listed rows, one ctypes call per row spread over host threads.

    ctypes drops the GIL during each call, so this uses several cores while the
    C oracle itself stays single-threaded.  Returns arrays indexed like ``rows``
    (the longest rows are started first, so that they do not finish last).
    """
    rp = np.asarray(row_ptr, dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    threads = threads or os.cpu_count() or 1
    s = np.zeros((rows.size, k), dtype=np.int32)
    y = np.zeros((rows.size, k), dtype=np.float64)
    y2 = np.zeros((rows.size, k), dtype=np.float64) if runner_up else None
    s2 = np.zeros((rows.size, k), dtype=np.int32) if runner_up else None

    def one(q):
        r = rows[q]
        lo, hi = int(rp[r]), int(rp[r + 1])
        out = sketch(np.array([0, hi - lo]), ids[lo:hi], w[lo:hi], k, seed, runner_up=runner_up)
        s[q], y[q] = out[0][0], out[1][0]
        if runner_up:
            y2[q], s2[q] = out[2][0], out[3][0]

    order = np.argsort(-(rp[rows + 1] - rp[rows]), kind="stable")
    with _cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, order))
    return (s, y, y2, s2) if runner_up else (s, y)


def fastsearch_budgets(v, R):
    a = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(a.size, dtype=np.int64)
    _check(lib().gmo_fastsearch_budgets(_p(a, _f64p), a.size, int(R), _p(out, _i64p)), "budgets")
    return out


def fastgm_alg1(ids, w, k, seed, delta=None, search=False):
    """Algorithm 1 on one vector -> (s, y, arrivals generated); with search=True also
    (R at which FastSearch found every server filled, arrivals released by then)."""
    ii = np.ascontiguousarray(ids, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    s = np.zeros(k, dtype=np.int32)
    y = np.zeros(k, dtype=np.float64)
    n_arr, sR, s_arr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib().gmo_fastgm_alg1(_p(ii, _i32p), _p(ww, _f64p), ii.size, int(k), int(seed),
                               int(delta or k), _p(s, _i32p), _p(y, _f64p), ctypes.byref(n_arr), ctypes.byref(sR),
                               ctypes.byref(s_arr))
    _check(rc, "fastgm_alg1")
    if search:
        return s, y, n_arr.value, sR.value, s_arr.value
    return s, y, n_arr.value


def stream_fastgm(ids, w, k, seed):
    """Algorithm 2 over a stream (ids may repeat) -> (s, y, arrivals generated)."""
    ii = np.ascontiguousarray(ids, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    s = np.zeros(k, dtype=np.int32)
    y = np.zeros(k, dtype=np.float64)
    n_arr = ctypes.c_int64()
    rc = lib().gmo_stream_fastgm(_p(ii, _i32p), _p(ww, _f64p), ii.size, int(k), int(seed),
                                 _p(s, _i32p), _p(y, _f64p), ctypes.byref(n_arr))
    _check(rc, "stream_fastgm")
    return s, y, n_arr.value


def jaccard(sa, sb):
    a = np.ascontiguousarray(sa, dtype=np.int32)
    b = np.ascontiguousarray(sb, dtype=np.int32)
    a2 = a.reshape(-1, a.shape[-1])
    b2 = b.reshape(-1, b.shape[-1])
    out = np.zeros(a2.shape[0], dtype=np.float64)
    _check(lib().gmo_jaccard(_p(a2, _i32p), _p(b2, _i32p), a2.shape[0], a2.shape[1], _p(out, _f64p)), "jaccard")
    return out


def cardinality(y):
    a = np.ascontiguousarray(y, dtype=np.float64)
    a2 = a.reshape(-1, a.shape[-1])
    out = np.zeros(a2.shape[0], dtype=np.float64)
    _check(lib().gmo_cardinality(_p(a2, _f64p), a2.shape[0], a2.shape[1], _p(out, _f64p)), "cardinality")
    return out


def merge(sa, ya, sb, yb):
    sa = np.ascontiguousarray(sa, dtype=np.int32)
    ya = np.ascontiguousarray(ya, dtype=np.float64)
    sb = np.ascontiguousarray(sb, dtype=np.int32)
    yb = np.ascontiguousarray(yb, dtype=np.float64)
    s = np.zeros_like(sa)
    y = np.zeros_like(ya)
    lib().gmo_merge(_p(sa, _i32p), _p(ya, _f64p), _p(sb, _i32p), _p(yb, _f64p), sa.size, _p(s, _i32p),
                    _p(y, _f64p))
    return s, y
