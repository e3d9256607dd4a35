"""Binding of libgm's serving engine (include/gm_server.h): marshalling only.

The engine (scheduler thread, device arena, batching, admission) is native code
in libgm; this module passes numpy arrays and tickets through the C-ABI and
keeps every submitted array alive until its request has finished.
"""
import ctypes

import numpy as np

from . import gm

GM_EAGAIN, GM_ECANCELED = 6, 7
GM_REQ_SKETCH, GM_REQ_JACCARD, GM_REQ_CARDINALITY = 0, 1, 2
_vp = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("staging_bytes", ctypes.c_size_t),
                ("max_batch_nnz", ctypes.c_int64), ("max_batch_rows", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("params", _vp), ("margin", ctypes.c_float), ("stage_pinned", ctypes.c_int32),
                ("fake_device", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("value", ctypes.c_double), ("t_submit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "finished", "cancelled", "refused", "failed", "sketch_batches", "query_batches",
        "sketch_rows", "sketch_elements", "queries", "arena_bytes", "arena_peak_bytes", "arena_resident_bytes",
        "queued", "in_flight_batches", "staged_requests", "direct_requests", "pack_ns", "launch_ns")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_bound = False


def _lib():
    global _bound
    L = gm.lib()
    if not _bound:
        L.gm_server_config_default.argtypes = [ctypes.POINTER(Config)]
        L.gm_server_config_default.restype = None
        L.gm_server_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_vp)]
        L.gm_server_destroy.argtypes = [_vp]
        L.gm_server_now_ns.restype = ctypes.c_int64
        L.gm_server_submit_sketch.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_uint64)]
        L.gm_server_submit_jaccard.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.gm_server_submit_cardinality.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.gm_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Result)]
        L.gm_server_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]
        L.gm_server_read_sketch.argtypes = [_vp, ctypes.c_uint64, _vp, _vp]
        L.gm_server_release.argtypes = [_vp, ctypes.c_uint64]
        L.gm_server_cancel.argtypes = [_vp, ctypes.c_uint64]
        L.gm_server_stats_get.argtypes = [_vp, ctypes.POINTER(Stats)]
        L.gm_server_pause.argtypes = [_vp, ctypes.c_int32]
        _bound = True
    return L


def now_ns():
    return int(_lib().gm_server_now_ns())


class Server:
    """A serving engine on the current CUDA device (or a fake device)."""

    def __init__(self, device_bytes=8 << 30, staging_bytes=64 << 20, max_batch_nnz=1 << 23, max_batch_rows=4096,
                 n_streams=4, seed=1, flags=0, params=None, margin=0.0, stage_pinned=False, fake_device=False):
        L = _lib()
        cfg = Config()
        L.gm_server_config_default(ctypes.byref(cfg))
        cfg.device_bytes, cfg.staging_bytes = int(device_bytes), int(staging_bytes)
        cfg.max_batch_nnz, cfg.max_batch_rows, cfg.n_streams = int(max_batch_nnz), int(max_batch_rows), int(n_streams)
        cfg.seed, cfg.flags = int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags)
        self._params = params  # keep the model alive
        cfg.params = _vp(params.data_ptr()) if params is not None else _vp(0)
        cfg.margin = float(margin)
        cfg.stage_pinned = 1 if stage_pinned else 0
        cfg.fake_device = 1 if fake_device else 0
        h = _vp()
        gm._check(L.gm_server_create(ctypes.byref(cfg), ctypes.byref(h)), "gm_server_create")
        self._h = h
        self._keep = {}  # ticket -> arrays the engine reads

    def close(self):
        if self._h:
            gm._check(_lib().gm_server_destroy(self._h), "gm_server_destroy")
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_sketch(self, ids, w, k):
        """Queue the sketch of one vector (host arrays; pinned torch tensors are copied asynchronously)."""
        ids_p, w_p, keep, n = _host_vec(ids, w)
        t = ctypes.c_uint64()
        gm._check(_lib().gm_server_submit_sketch(self._h, ids_p, w_p, n, int(k), ctypes.byref(t)),
                  "gm_server_submit_sketch")
        self._keep[t.value] = keep
        return t.value

    def submit_jaccard(self, a, b):
        t = ctypes.c_uint64()
        gm._check(_lib().gm_server_submit_jaccard(self._h, int(a), int(b), ctypes.byref(t)), "gm_server_submit_jaccard")
        return t.value

    def submit_cardinality(self, a):
        t = ctypes.c_uint64()
        gm._check(_lib().gm_server_submit_cardinality(self._h, int(a), ctypes.byref(t)),
                  "gm_server_submit_cardinality")
        return t.value

    def _final(self, ticket, rc, res):
        if rc != GM_EAGAIN:
            self._keep.pop(ticket, None)
        return rc, res.as_dict()

    def poll(self, ticket):
        """(status code, result dict); GM_EAGAIN while pending."""
        res = Result()
        rc = _lib().gm_server_poll(self._h, int(ticket), ctypes.byref(res))
        if rc == gm.GM_EINVAL and res.kind == 0 and res.t_submit_ns == 0:
            raise gm.GmError(rc, "gm_server_poll")
        return self._final(ticket, rc, res)

    def wait(self, ticket, timeout=60.0):
        res = Result()
        rc = _lib().gm_server_wait(self._h, int(ticket), float(timeout), ctypes.byref(res))
        return self._final(ticket, rc, res)

    def read_sketch(self, ticket, k):
        s = np.empty(k, dtype=np.int32)
        y = np.empty(k, dtype=np.float64)
        gm._check(_lib().gm_server_read_sketch(self._h, int(ticket), s.ctypes.data_as(_vp), y.ctypes.data_as(_vp)),
                  "gm_server_read_sketch")
        return s, y

    def release(self, ticket):
        gm._check(_lib().gm_server_release(self._h, int(ticket)), "gm_server_release")

    def cancel(self, ticket):
        return _lib().gm_server_cancel(self._h, int(ticket))

    def pause(self, paused=True):
        gm._check(_lib().gm_server_pause(self._h, 1 if paused else 0), "gm_server_pause")

    def stats(self):
        st = Stats()
        gm._check(_lib().gm_server_stats_get(self._h, ctypes.byref(st)), "gm_server_stats_get")
        return st.as_dict()


def _host_vec(ids, w):
    """Pointers to host int32 ids and float64 weights (numpy arrays or CPU torch tensors)."""
    if hasattr(ids, "data_ptr"):
        if ids.is_cuda or w.is_cuda or ids.dtype.itemsize != 4 or w.dtype.itemsize != 8:
            raise ValueError("ids / w must be CPU int32 / float64 tensors")
        ids_c, w_c = ids.contiguous(), w.contiguous()
        return _vp(ids_c.data_ptr()), _vp(w_c.data_ptr()), (ids_c, w_c), int(ids_c.numel())
    ids_c = np.ascontiguousarray(ids, dtype=np.int32)
    w_c = np.ascontiguousarray(w, dtype=np.float64)
    if ids_c.size != w_c.size:
        raise ValueError("ids and w differ in length")
    return ids_c.ctypes.data_as(_vp), w_c.ctypes.data_as(_vp), (ids_c, w_c), int(ids_c.size)
