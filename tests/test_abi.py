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
