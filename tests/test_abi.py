"""The C-ABI library loads and exports every symbol include/*.h declares (CPU only: no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libgm():
    from paper_2302_05176_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gm_sketch", "gm_sketch_plain", "gm_jaccard", "gm_cardinality", "gm_merge", "gm_status",
                 "gm_strerror", "gm_sketch_workspace_bytes"):
        assert must in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(libgm, name):
    assert hasattr(libgm, name), name


def test_host_side_queries(libgm):
    libgm.gm_strerror.restype = ctypes.c_char_p
    assert libgm.gm_strerror(0) == b"ok"
    assert libgm.gm_strerror(5) == b"invalid input data"
    f = libgm.gm_sketch_workspace_bytes
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32]
    f.restype = ctypes.c_size_t
    assert f(10, 1000, 128, 0) >= 1000 * 4 + 128 * 8
    assert f(10, 1000, 0, 0) == 0           # k < 1
    assert f(10, 1000, 1 << 20, 0) == 0     # k > GM_MAX_K
    assert f(-1, 1000, 128, 0) == 0


def test_argument_errors_before_launch(libgm):
    """Bad sizes are rejected on the host, before any CUDA call."""
    sk = libgm.gm_sketch
    vp = ctypes.c_void_p
    sk.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                   vp, vp, vp, ctypes.c_size_t, vp]
    fake = vp(0x1000)
    assert sk(fake, fake, fake, 1, 10, 0, 1, 0, fake, fake, fake, 1 << 20, None) == 1      # k = 0
    assert sk(fake, fake, fake, -1, 10, 8, 1, 0, fake, fake, fake, 1 << 20, None) == 1     # n_rows < 0
    assert sk(fake, fake, fake, 1, 10, 8, 1, 0, fake, fake, None, 1 << 20, None) == 1      # no workspace
    assert sk(fake, fake, fake, 1, 10, 8, 1, 0, fake, fake, fake, 16, None) == 2           # too small
    assert sk(fake, fake, fake, 1, 10, 8, 1, 0, fake, fake, vp(0x1010), 1 << 20, None) == 1  # workspace off 256 B


def test_host_side_workspace_sizes(libgm):
    """The host pipeline's workspace follows its largest chunk of rows; the learned
    pre-pass's grows with the batch; invalid shapes give 0 (host-only queries)."""
    import numpy as np
    vp = ctypes.c_void_p
    loose = libgm.gm_sketch_host_workspace_bytes
    loose.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
    loose.restype = ctypes.c_size_t
    tight = libgm.gm_sketch_host_workspace_bytes_csr
    tight.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    tight.restype = ctypes.c_size_t
    lens = np.where(np.arange(4000) < 100, 1000, 1)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    p = rp.ctypes.data_as(vp)
    t, l = tight(p, 4000, 256), loose(4000, int(rp[-1]), 256)
    assert 0 < t < l
    even = np.arange(4001, dtype=np.int64) * 26  # the same elements spread evenly: smaller chunks
    assert tight(even.ctypes.data_as(vp), 4000, 256) < t
    bad = rp.copy()
    bad[10], bad[11] = bad[11], bad[10]  # decreasing
    assert tight(bad.ctypes.data_as(vp), 4000, 256) == 0
    assert tight(p, 4000, 0) == 0 and loose(4000, int(rp[-1]), 1 << 20) == 0
    lb = libgm.gm_learned_bound_workspace_bytes
    lb.argtypes = [ctypes.c_int32, ctypes.c_int64]
    lb.restype = ctypes.c_size_t
    assert 0 < lb(10, 1000) < lb(10, 1_000_000) and lb(10, 1000) < lb(100_000, 1000)
    assert lb(-1, 10) == 0 and lb(10, -1) == 0


def header_constants():
    """The integer #defines of include/gm.h (plain numbers and shifts), by name."""
    text = open(os.path.join(ROOT, "include", "gm.h")).read()
    out = {}
    for m in re.finditer(r"^#define (GM_[A-Z0-9_]+)\s+(\(?\s*\d+u?\s*(?:<<\s*\d+)?\s*\)?)", text, flags=re.M):
        expr = m.group(2).replace("u", "")
        out[m.group(1)] = eval(expr, {"__builtins__": {}})
    return out


def test_binding_constants_match_the_header():
    """Every status code, flag and size the Python binding names has the header's value."""
    from paper_2302_05176_gb300 import gm
    consts = header_constants()
    assert "GM_FLAG_COMPACT_LONG" in consts and "GM_BOUND_LEARNED" in consts
    checked = 0
    for name, value in consts.items():
        if hasattr(gm, name):
            assert getattr(gm, name) == value, name
            checked += 1
    assert checked >= 14
