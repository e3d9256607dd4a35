"""Thin Python binding of libgm (include/gm.h): argument marshalling only.

Every step of the sketch runs inside libgm's CUDA kernels; this module only
passes device pointers (torch tensors) and sizes through the C-ABI, allocates
outputs and workspaces with torch, and turns status codes into exceptions.
There is no fallback: if the library is missing, every call raises.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgm.so")

GM_OK, GM_EINVAL, GM_ENOMEM, GM_ECUDA, GM_ETIMEOUT, GM_EDATA = 0, 1, 2, 3, 4, 5
GM_FLAG_VALIDATE = 1 << 0
GM_FLAG_FP64_UNIT = 1 << 2
GM_FLAG_INT_PRODUCTS = 1 << 1
GM_FLAG_TIGHT_BOUND = 1 << 3
GM_FLAG_COMPACT_LONG = 1 << 6
GM_BOUND_CLOSED = 0 << 4
GM_BOUND_NONE = 1 << 4
GM_BOUND_LEARNED = 2 << 4
GM_MAX_K = 4096
GM_MODEL_FEATURES = 8
GM_MODEL_HIDDEN = 64
GM_MODEL_PARAMS = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


class GmError(RuntimeError):
    """A non-zero status of a libgm call: .code (GM_E*) and the call's name."""

    def __init__(self, code, what):
        super().__init__("%s: %s (code %d)" % (what, strerror(code) if _lib else "libgm", code))
        self.code = code


class gm_stats(ctypes.Structure):
    """gm_stats of include/gm.h: the status and work counters of one call."""
    _fields_ = [("arrivals", ctypes.c_uint64), ("elements", ctypes.c_uint64), ("screened_out", ctypes.c_uint64),
                ("heavy_elements", ctypes.c_uint64), ("rows_escalated", ctypes.c_uint64),
                ("cas_retries", ctypes.c_uint64), ("cycles_light", ctypes.c_uint64),
                ("cycles_medium", ctypes.c_uint64), ("cycles_heavy", ctypes.c_uint64),
                ("cycles_dense", ctypes.c_uint64), ("cycles_wait", ctypes.c_uint64),
                ("cycles_setup", ctypes.c_uint64), ("cycles_finish", ctypes.c_uint64),
                ("cycles_total", ctypes.c_uint64), ("kept", ctypes.c_uint64), ("rows_fallback", ctypes.c_uint64),
                ("status", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "reserved"}


class gm_tuning(ctypes.Structure):
    """gm_tuning of include/gm.h: first-pass quantile and routing thresholds."""
    _fields_ = [("p_first", ctypes.c_float), ("light_max", ctypes.c_float), ("medium_max", ctypes.c_float),
                ("heavy_max", ctypes.c_float)]

    def as_dict(self):
        return {f: float(getattr(self, f)) for f, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load libgm.so (built in-tree by paper_2302_05176_gb300.build / __graft_entry__.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgm.so is missing at %s: run __graft_entry__.build() first" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.gm_sketch_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32]
        L.gm_sketch_workspace_bytes.restype = ctypes.c_size_t
        sk = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
              _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.gm_sketch.argtypes = sk
        L.gm_sketch_plain.argtypes = sk
        L.gm_status.argtypes = [_vp, ctypes.POINTER(gm_stats), _vp]
        L.gm_jaccard.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp]
        L.gm_cardinality.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
        L.gm_merge.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]
        L.gm_features.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp, _vp]
        L.gm_row_ln_ystar.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
        L.gm_model_init.argtypes = [_vp, ctypes.c_uint64, _vp]
        L.gm_model_forward.argtypes = [_vp, _vp, ctypes.c_int32, _vp, _vp]
        L.gm_model_grad_workspace_bytes.restype = ctypes.c_size_t
        L.gm_model_grad.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp, _vp, _vp, ctypes.c_size_t,
                                    _vp]
        L.gm_model_adam.argtypes = [_vp, _vp, _vp, ctypes.c_float, ctypes.c_int32, _vp]
        L.gm_model_save.argtypes = [_vp, ctypes.c_char_p, _vp]
        L.gm_model_load.argtypes = [_vp, ctypes.c_char_p, _vp]
        L.gm_learned_bound_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64]
        L.gm_learned_bound_workspace_bytes.restype = ctypes.c_size_t
        L.gm_learned_bound.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp, ctypes.c_float,
                                       _vp, _vp, ctypes.c_size_t, _vp]
        L.gm_sketch_learned_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
        L.gm_sketch_learned_workspace_bytes.restype = ctypes.c_size_t
        L.gm_sketch_learned.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_uint32, _vp, ctypes.c_float, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.gm_graph_create.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_uint32, _vp, _vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
        L.gm_graph_launch.argtypes = [_vp, _vp]
        L.gm_graph_destroy.argtypes = [_vp]
        tp = ctypes.POINTER(gm_tuning)
        L.gm_tuning_default.argtypes = [tp]
        L.gm_tuning_default.restype = None
        L.gm_tune.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                              ctypes.c_uint32, _vp, _vp, _vp, ctypes.c_size_t, tp, ctypes.POINTER(ctypes.c_double), _vp]
        L.gm_tuning_set.argtypes = [ctypes.c_int32, ctypes.c_int64, tp]
        L.gm_tuning_get.argtypes = [ctypes.c_int32, ctypes.c_int64, tp]
        L.gm_tuning_save.argtypes = [ctypes.c_char_p]
        L.gm_tuning_load.argtypes = [ctypes.c_char_p]
        L.gm_stream_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
        L.gm_stream_workspace_bytes.restype = ctypes.c_size_t
        L.gm_stream_reset.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
        L.gm_stream_ingest.argtypes = [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, _vp, ctypes.c_size_t, _vp]
        L.gm_sketch_budget.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_uint32, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.gm_sketch_bounded_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
        L.gm_sketch_bounded_workspace_bytes.restype = ctypes.c_size_t
        L.gm_sketch_bounded.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_uint32, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.gm_row_ystar.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
        L.gm_sketch_fastsearch.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                           ctypes.c_size_t, _vp]
        L.gm_sketch_noalloc_status.argtypes = [ctypes.POINTER(gm_stats), _vp]
        L.gm_sketch_host_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
        L.gm_sketch_host_workspace_bytes.restype = ctypes.c_size_t
        L.gm_sketch_host_workspace_bytes_csr.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
        L.gm_sketch_host_workspace_bytes_csr.restype = ctypes.c_size_t
        L.gm_sketch_host.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                     ctypes.c_uint32, _vp, _vp, _vp, ctypes.c_size_t]
        L.gm_strerror.argtypes = [ctypes.c_int]
        L.gm_strerror.restype = ctypes.c_char_p
        L.gm_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code):
    """The message of a libgm status code."""
    return lib().gm_strerror(int(code)).decode()


def version():
    """libgm's version string."""
    return lib().gm_version().decode()


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _need_cuda(t, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dtype))


def _check(rc, what):
    if rc != GM_OK:
        raise GmError(rc, what)


def sketch_workspace_bytes(n_rows, nnz, k, flags=0):
    """Device workspace bytes gm_sketch / gm_sketch_plain need for this batch shape."""
    n = lib().gm_sketch_workspace_bytes(int(n_rows), int(nnz), int(k), int(flags))
    if n == 0:
        raise GmError(GM_EINVAL, "gm_sketch_workspace_bytes")
    return n


def workspace(n_rows, nnz, k, flags=0, device=None):
    """A device workspace (uint8 tensor) for gm_sketch on this batch shape."""
    return torch.empty(sketch_workspace_bytes(n_rows, nnz, k, flags), dtype=torch.uint8,
                       device=device or torch.device("cuda"))


def _sketch(fn, name, row_ptr, ids, w, k, seed, flags, s_out, y_out, ws, stream):
    _need_cuda(row_ptr, torch.int64, "row_ptr")
    _need_cuda(ids, torch.int32, "ids")
    _need_cuda(w, torch.float64, "w")
    n_rows = row_ptr.numel() - 1
    nnz = ids.numel()
    if w.numel() != nnz:
        raise ValueError("ids and w differ in length")
    dev = row_ptr.device
    if s_out is None:
        s_out = torch.empty((n_rows, k), dtype=torch.int32, device=dev)
    if y_out is None:
        y_out = torch.empty((n_rows, k), dtype=torch.float64, device=dev)
    _need_cuda(s_out, torch.int32, "s_out")
    _need_cuda(y_out, torch.float64, "y_out")
    if ws is None:
        ws = workspace(n_rows, nnz, k, flags, dev)
    rc = fn(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, nnz, int(k), int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags),
            _ptr(s_out), _ptr(y_out), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, name)
    return s_out, y_out, ws


def gm_sketch(row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None, stream=None):
    """FastGM over CSR rows (device tensors) -> (s [n_rows,k] int32, y [n_rows,k] f64, workspace)."""
    return _sketch(lib().gm_sketch, "gm_sketch", row_ptr, ids, w, k, seed, flags, s_out, y_out, ws, stream)


def gm_sketch_plain(row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None, stream=None):
    """The O(k n+) sketch; same output as gm_sketch."""
    return _sketch(lib().gm_sketch_plain, "gm_sketch_plain", row_ptr, ids, w, k, seed, flags, s_out, y_out, ws,
                   stream)


def gm_status(ws, stream=None):
    """Synchronise the stream and return (device status code, counters dict)."""
    st = gm_stats()
    rc = lib().gm_status(_ptr(ws), ctypes.byref(st), _stream_handle(stream))
    if rc == GM_ECUDA:
        raise GmError(rc, "gm_status")
    return rc, st.as_dict()


def gm_jaccard(s_a, s_b, out=None, stream=None):
    """Per pair, the fraction of registers holding the same element (Sec. 1): float64 [n_pairs]."""
    _need_cuda(s_a, torch.int32, "s_a")
    _need_cuda(s_b, torch.int32, "s_b")
    if s_a.shape != s_b.shape or s_a.dim() != 2:
        raise ValueError("s_a and s_b must both be [n_pairs, k]")
    n, k = s_a.shape
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=s_a.device)
    _check(lib().gm_jaccard(_ptr(s_a), _ptr(s_b), n, k, _ptr(out), _stream_handle(stream)), "gm_jaccard")
    return out


def gm_cardinality(y, out=None, stream=None):
    """Per row, (k - 1) / sum_j y_j (Sec. 2.4): float64 [n_rows]; 0 when a register is unfilled."""
    _need_cuda(y, torch.float64, "y")
    n, k = y.shape
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=y.device)
    _check(lib().gm_cardinality(_ptr(y), n, k, _ptr(out), _stream_handle(stream)), "gm_cardinality")
    return out


def gm_merge(s_a, y_a, s_b, y_b, s_out=None, y_out=None, stream=None):
    """The sketch of the union (Sec. 2.3): per register the smaller (y, id)."""
    for t, d, nm in ((s_a, torch.int32, "s_a"), (s_b, torch.int32, "s_b"), (y_a, torch.float64, "y_a"),
                     (y_b, torch.float64, "y_b")):
        _need_cuda(t, d, nm)
    s_out = torch.empty_like(s_a) if s_out is None else s_out
    y_out = torch.empty_like(y_a) if y_out is None else y_out
    _check(lib().gm_merge(_ptr(s_a), _ptr(y_a), _ptr(s_b), _ptr(y_b), s_a.numel(), _ptr(s_out), _ptr(y_out),
                          _stream_handle(stream)), "gm_merge")
    return s_out, y_out


def to_device(csr, device="cuda"):
    """Copy a workloads.CSR to device tensors (row_ptr, ids, w)."""
    return (torch.from_numpy(csr.row_ptr).to(device), torch.from_numpy(csr.ids).to(device),
            torch.from_numpy(csr.w).to(device))


# --- learned first-pass bound (gm_features / gm_model_* / gm_sketch_learned) ----------------------

def gm_features(row_ptr, ids, w, k, out=None, stream=None):
    """Per-row features [n_rows, 8] float32 (ln n+, ln sum v, ln max v, 4 quantiles, ln k)."""
    _need_cuda(row_ptr, torch.int64, "row_ptr")
    _need_cuda(w, torch.float64, "w")
    n_rows = row_ptr.numel() - 1
    if out is None:
        out = torch.empty((n_rows, GM_MODEL_FEATURES), dtype=torch.float32, device=row_ptr.device)
    _need_cuda(out, torch.float32, "out")
    _check(lib().gm_features(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, w.numel(), int(k), _ptr(out),
                             _stream_handle(stream)), "gm_features")
    return out


def gm_row_ln_ystar(y, out=None, stream=None):
    """ln max_j y[r, j] per row (float32; +inf where a register is unfilled)."""
    _need_cuda(y, torch.float64, "y")
    n, k = y.shape
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=y.device)
    _check(lib().gm_row_ln_ystar(_ptr(y), n, k, _ptr(out), _stream_handle(stream)), "gm_row_ln_ystar")
    return out


def gm_model_init(seed, params=None, device=None, stream=None):
    """Seeded initial network parameters (float32 [GM_MODEL_PARAMS])."""
    if params is None:
        params = torch.empty(GM_MODEL_PARAMS, dtype=torch.float32, device=device or torch.device("cuda"))
    _need_cuda(params, torch.float32, "params")
    _check(lib().gm_model_init(_ptr(params), int(seed) & 0xFFFFFFFFFFFFFFFF, _stream_handle(stream)),
           "gm_model_init")
    return params


def gm_model_forward(params, feats, out=None, stream=None):
    """The predicted ln bound of each sample (float32 [n]) from its 8 features."""
    _need_cuda(params, torch.float32, "params")
    _need_cuda(feats, torch.float32, "feats")
    n = feats.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feats.device)
    _check(lib().gm_model_forward(_ptr(params), _ptr(feats), n, _ptr(out), _stream_handle(stream)),
           "gm_model_forward")
    return out


def gm_model_grad_workspace_bytes():
    """Device workspace bytes of gm_model_grad."""
    return int(lib().gm_model_grad_workspace_bytes())


def gm_model_grad(params, feats, target, tau, grad=None, loss=None, ws=None, stream=None):
    """Gradient of the mean pinball loss (level tau) -> (grad [P] f32, loss [1] f32, workspace)."""
    _need_cuda(params, torch.float32, "params")
    _need_cuda(feats, torch.float32, "feats")
    _need_cuda(target, torch.float32, "target")
    dev = params.device
    grad = torch.empty(GM_MODEL_PARAMS, dtype=torch.float32, device=dev) if grad is None else grad
    loss = torch.empty(1, dtype=torch.float32, device=dev) if loss is None else loss
    if ws is None:
        ws = torch.empty(gm_model_grad_workspace_bytes(), dtype=torch.uint8, device=dev)
    _check(lib().gm_model_grad(_ptr(params), _ptr(feats), _ptr(target), target.numel(), float(tau), _ptr(grad),
                               _ptr(loss), _ptr(ws), ws.numel(), _stream_handle(stream)), "gm_model_grad")
    return grad, loss, ws


def gm_model_adam(params, adam, grad, lr, step, stream=None):
    """One Adam step on the parameters in place; `adam` holds the moments (updated too)."""
    _check(lib().gm_model_adam(_ptr(params), _ptr(adam), _ptr(grad), float(lr), int(step), _stream_handle(stream)),
           "gm_model_adam")


def gm_model_save(params, path, stream=None):
    """Write the parameters to a file (header with magic and shape)."""
    _check(lib().gm_model_save(_ptr(params), os.fsencode(path), _stream_handle(stream)), "gm_model_save")


def gm_model_load(path, params=None, device=None, stream=None):
    """Read parameters written by gm_model_save into params."""
    if params is None:
        params = torch.empty(GM_MODEL_PARAMS, dtype=torch.float32, device=device or torch.device("cuda"))
    _check(lib().gm_model_load(_ptr(params), os.fsencode(path), _stream_handle(stream)), "gm_model_load")
    return params


def gm_learned_bound(row_ptr, w, k, params, margin=0.0, out=None, ws=None, stream=None):
    """Per-row learned first-pass bound exp(prediction + margin), float32 [n_rows]."""
    _need_cuda(row_ptr, torch.int64, "row_ptr")
    _need_cuda(w, torch.float64, "w")
    _need_cuda(params, torch.float32, "params")
    n_rows, nnz = row_ptr.numel() - 1, w.numel()
    dev = row_ptr.device
    out = torch.empty(n_rows, dtype=torch.float32, device=dev) if out is None else out
    if ws is None:
        n = lib().gm_learned_bound_workspace_bytes(n_rows, nnz)
        ws = torch.empty(max(1, n), dtype=torch.uint8, device=dev)
    _check(lib().gm_learned_bound(_ptr(row_ptr), _ptr(w), n_rows, nnz, int(k), _ptr(params), float(margin), _ptr(out),
                                  _ptr(ws), ws.numel(), _stream_handle(stream)), "gm_learned_bound")
    return out


def sketch_learned_workspace_bytes(n_rows, nnz, k):
    """Device workspace bytes of gm_sketch_learned for this batch shape."""
    n = lib().gm_sketch_learned_workspace_bytes(int(n_rows), int(nnz), int(k))
    if n == 0:
        raise GmError(GM_EINVAL, "gm_sketch_learned_workspace_bytes")
    return n


def gm_sketch_learned(row_ptr, ids, w, k, seed, params, margin=0.0, flags=0, s_out=None, y_out=None, ws=None,
                      stream=None):
    """FastGM with a learned first-pass bound per row; the same registers as gm_sketch."""
    _need_cuda(row_ptr, torch.int64, "row_ptr")
    _need_cuda(ids, torch.int32, "ids")
    _need_cuda(w, torch.float64, "w")
    _need_cuda(params, torch.float32, "params")
    n_rows, nnz = row_ptr.numel() - 1, ids.numel()
    if w.numel() != nnz:
        raise ValueError("ids and w differ in length")
    dev = row_ptr.device
    s_out = torch.empty((n_rows, k), dtype=torch.int32, device=dev) if s_out is None else s_out
    y_out = torch.empty((n_rows, k), dtype=torch.float64, device=dev) if y_out is None else y_out
    if ws is None:
        ws = torch.empty(sketch_learned_workspace_bytes(n_rows, nnz, k), dtype=torch.uint8, device=dev)
    rc = lib().gm_sketch_learned(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, nnz, int(k),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), _ptr(params), float(margin),
                                 _ptr(s_out), _ptr(y_out), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "gm_sketch_learned")
    return s_out, y_out, ws


class SketchGraph:
    """One gm_sketch call over fixed buffers, captured as a CUDA graph (gm_graph_*).
    replay() re-runs it on whatever the buffers hold; s / y are the outputs."""

    def __init__(self, row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None):
        _need_cuda(row_ptr, torch.int64, "row_ptr")
        _need_cuda(ids, torch.int32, "ids")
        _need_cuda(w, torch.float64, "w")
        n_rows, nnz = row_ptr.numel() - 1, ids.numel()
        dev = row_ptr.device
        self.s = torch.empty((n_rows, k), dtype=torch.int32, device=dev) if s_out is None else s_out
        self.y = torch.empty((n_rows, k), dtype=torch.float64, device=dev) if y_out is None else y_out
        self.ws = workspace(n_rows, nnz, k, flags, dev) if ws is None else ws
        self._keep = (row_ptr, ids, w)
        h = _vp()
        _check(lib().gm_graph_create(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, nnz, int(k),
                                     int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), _ptr(self.s), _ptr(self.y),
                                     _ptr(self.ws), self.ws.numel(), ctypes.byref(h)), "gm_graph_create")
        self._h = h

    def replay(self, stream=None):
        _check(lib().gm_graph_launch(self._h, _stream_handle(stream)), "gm_graph_launch")
        return self.s, self.y

    def close(self):
        if getattr(self, "_h", None):
            lib().gm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- autotuning (gm_tune / gm_tuning_*) -------------------------------------------------------

def tuning_default():
    """The compiled default tuning as a dict."""
    t = gm_tuning()
    lib().gm_tuning_default(ctypes.byref(t))
    return t.as_dict()


def _tuning(d):
    t = gm_tuning()
    lib().gm_tuning_default(ctypes.byref(t))
    for f, v in d.items():
        setattr(t, f, float(v))
    return t


def gm_tune(row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None, stream=None):
    """Time candidate tunings on this batch; installs and returns (best dict, best ms)."""
    n_rows, nnz = row_ptr.numel() - 1, ids.numel()
    dev = row_ptr.device
    s_out = torch.empty((n_rows, k), dtype=torch.int32, device=dev) if s_out is None else s_out
    y_out = torch.empty((n_rows, k), dtype=torch.float64, device=dev) if y_out is None else y_out
    ws = workspace(n_rows, nnz, k, flags, dev) if ws is None else ws
    best = gm_tuning()
    ms = ctypes.c_double()
    _check(lib().gm_tune(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, nnz, int(k), int(seed) & 0xFFFFFFFFFFFFFFFF,
                         int(flags), _ptr(s_out), _ptr(y_out), _ptr(ws), ws.numel(), ctypes.byref(best),
                         ctypes.byref(ms), _stream_handle(stream)), "gm_tune")
    return best.as_dict(), ms.value


def tuning_set(k, mean_row_len, **values):
    """Install a tuning for (k, mean row length) in the process-wide table."""
    _check(lib().gm_tuning_set(int(k), int(mean_row_len), ctypes.byref(_tuning(values))), "gm_tuning_set")


def tuning_get(k, mean_row_len):
    """The table entry for (k, mean row length), or None."""
    t = gm_tuning()
    return t.as_dict() if lib().gm_tuning_get(int(k), int(mean_row_len), ctypes.byref(t)) == GM_OK else None


def tuning_clear():
    """Empty the process-wide tuning table."""
    lib().gm_tuning_clear()


def tuning_save(path):
    """Write the tuning table as text."""
    _check(lib().gm_tuning_save(os.fsencode(path)), "gm_tuning_save")


def tuning_load(path):
    """Read a tuning table written by tuning_save (entries are added)."""
    _check(lib().gm_tuning_load(os.fsencode(path)), "gm_tuning_load")


# --- Stream-FastGM (gm_stream_*) ------------------------------------------------------------------

class StreamSketch:
    """A running sketch fed chunk by chunk (Algorithm 2): s, y are device tensors [k]."""

    def __init__(self, k, seed, flags=0, device=None, stream=None):
        dev = device or torch.device("cuda")
        self.k, self.seed, self.flags = int(k), int(seed), int(flags)
        self.s = torch.empty(self.k, dtype=torch.int32, device=dev)
        self.y = torch.empty(self.k, dtype=torch.float64, device=dev)
        self.ws = torch.empty(0, dtype=torch.uint8, device=dev)
        _check(lib().gm_stream_reset(_ptr(self.s), _ptr(self.y), self.k, _stream_handle(stream)), "gm_stream_reset")

    def ingest(self, ids, w, stream=None):
        _need_cuda(ids, torch.int32, "ids")
        _need_cuda(w, torch.float64, "w")
        n = ids.numel()
        need = lib().gm_stream_workspace_bytes(n, self.k)
        if need == 0:
            raise GmError(GM_EINVAL, "gm_stream_workspace_bytes")
        if self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.s.device)
        _check(lib().gm_stream_ingest(_ptr(self.s), _ptr(self.y), self.k, _ptr(ids), _ptr(w), n,
                                      self.seed & 0xFFFFFFFFFFFFFFFF, self.flags, _ptr(self.ws), self.ws.numel(),
                                      _stream_handle(stream)), "gm_stream_ingest")
        return self


# --- FastSearch's budgets and caller-given bounds --------------------------------------------------

def gm_sketch_budget(row_ptr, ids, w, k, seed, R_row, flags=0, s_out=None, y_out=None, ws=None, stream=None):
    """Release min(k, ceil(R_row[r] v_i / sum v)) arrivals of each element (FastSearch's step)."""
    _need_cuda(R_row, torch.float64, "R_row")
    fn = lambda *a: lib().gm_sketch_budget(*a[:8], _ptr(R_row), *a[8:])
    return _sketch(fn, "gm_sketch_budget", row_ptr, ids, w, k, seed, flags, s_out, y_out, ws, stream)


def gm_sketch_bounded(row_ptr, ids, w, k, seed, bound_row, flags=0, s_out=None, y_out=None, ws=None, stream=None):
    """FastGM with the caller's first-pass bound per row (device doubles)."""
    _need_cuda(bound_row, torch.float64, "bound_row")
    n_rows, nnz = row_ptr.numel() - 1, ids.numel()
    if ws is None:
        ws = torch.empty(lib().gm_sketch_bounded_workspace_bytes(n_rows, nnz, int(k)), dtype=torch.uint8,
                         device=row_ptr.device)
    fn = lambda *a: lib().gm_sketch_bounded(*a[:8], _ptr(bound_row), *a[8:])
    return _sketch(fn, "gm_sketch_bounded", row_ptr, ids, w, k, seed, flags, s_out, y_out, ws, stream)


def gm_sketch_fastsearch(row_ptr, ids, w, k, seed, delta=None, flags=0, rounds_out=None, s_out=None, y_out=None,
                         ws=None, stream=None):
    """FastGM under the paper's FastSearch schedule, all rounds on the device
    (Algorithm 1; delta defaults to k) -> (s, y, workspace, rounds int32 [n_rows])."""
    n_rows = row_ptr.numel() - 1
    delta = int(delta or k)
    if rounds_out is None:
        rounds_out = torch.zeros(n_rows, dtype=torch.int32, device=row_ptr.device)
    _need_cuda(rounds_out, torch.int32, "rounds_out")
    fn = lambda *a: lib().gm_sketch_fastsearch(*a[:8], delta, _ptr(rounds_out), *a[8:])
    s, y, ws = _sketch(fn, "gm_sketch_fastsearch", row_ptr, ids, w, k, seed, flags, s_out, y_out, ws, stream)
    return s, y, ws, rounds_out


def gm_row_ystar(y, out=None, stream=None):
    """Per row, the largest register y* (float64 [n_rows]; +inf if one is unfilled)."""
    _need_cuda(y, torch.float64, "y")
    n, k = y.shape
    out = torch.empty(n, dtype=torch.float64, device=y.device) if out is None else out
    _check(lib().gm_row_ystar(_ptr(y), n, k, _ptr(out), _stream_handle(stream)), "gm_row_ystar")
    return out


# --- host-memory batches (gm_sketch_host) --------------------------------------------------------

def sketch_host_workspace(n_rows, nnz, k, device=None, row_ptr=None):
    """Device workspace for gm_sketch_host: sized by the batch's largest chunk when
    the host row offsets are given, else for any row offsets."""
    if row_ptr is not None:
        rp = row_ptr
        if not isinstance(rp, torch.Tensor) or rp.is_cuda or rp.dtype != torch.int64 or not rp.is_contiguous() or rp.numel() != int(n_rows) + 1:
            raise ValueError("row_ptr must be a contiguous CPU int64 tensor of n_rows + 1 offsets")
        n = lib().gm_sketch_host_workspace_bytes_csr(_ptr(rp), int(n_rows), int(k))
        name = "gm_sketch_host_workspace_bytes_csr"
    else:
        n = lib().gm_sketch_host_workspace_bytes(int(n_rows), int(nnz), int(k))
        name = "gm_sketch_host_workspace_bytes"
    if n == 0:
        raise GmError(GM_EINVAL, name)
    return torch.empty(n, dtype=torch.uint8, device=device or torch.device("cuda"))


def gm_sketch_host(row_ptr, ids, w, k, seed, flags=0, s_out=None, y_out=None, ws=None):
    """gm_sketch over CPU tensors (pinned for asynchronous copies); returns CPU (s, y, ws)."""
    for t, d, nm in ((row_ptr, torch.int64, "row_ptr"), (ids, torch.int32, "ids"), (w, torch.float64, "w")):
        if t.is_cuda or t.dtype != d or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CPU %s tensor" % (nm, d))
    n_rows, nnz = row_ptr.numel() - 1, ids.numel()
    s_out = torch.empty((n_rows, k), dtype=torch.int32) if s_out is None else s_out
    y_out = torch.empty((n_rows, k), dtype=torch.float64) if y_out is None else y_out
    ws = sketch_host_workspace(n_rows, nnz, k, row_ptr=row_ptr) if ws is None else ws
    _check(lib().gm_sketch_host(_ptr(row_ptr), _ptr(ids), _ptr(w), n_rows, nnz, int(k),
                                int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), _ptr(s_out), _ptr(y_out), _ptr(ws),
                                ws.numel()), "gm_sketch_host")
    return s_out, y_out, ws
