"""The device arithmetic of one arrival against independent references (GPU).

* -ln(u): the integer-pipe logarithm against 120-bit mpmath values (error bound
  0.501 ulp: the method's analysis gives 0.5 + 2^-8) and against CUDA's own log
  (documented 1 ulp) and glibc's (numpy);
* RN(a b), RN(1/v): bit-identical to IEEE-754 products / quotients (numpy);
* whole arrival streams: the warp path against the CPU oracle;
* the first-arrival screen: it never skips an element whose first arrival is
  within the bound, and it skips nearly all of those that are not.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2302_05176_gb300 import build as libbuild
from parity import ulp_distance

pytestmark = pytest.mark.gpu
vp = ctypes.c_void_p


@pytest.fixture(scope="module")
def L():
    lib = ctypes.CDLL(libbuild.build())
    lib.gm_diag_neglog.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    lib.gm_diag_dmul.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    lib.gm_diag_drcp.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    lib.gm_diag_arrivals.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                     ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp]
    lib.gm_diag_first_arrival.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_float,
                                          vp, vp, vp]
    return lib


def P(t):
    return vp(t.data_ptr())


def S():
    return vp(torch.cuda.current_stream().cuda_stream)


def neglog_dev(L, words, fp64):
    x = torch.from_numpy(words.view(np.int64)).cuda()
    out = torch.empty(words.size, dtype=torch.float64, device="cuda")
    assert L.gm_diag_neglog(P(x), words.size, fp64, P(out), S()) == 0
    return out.cpu().numpy()


def test_neglog_against_mpmath(L):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rng = np.random.default_rng(1)
    words = [rng.integers(0, 2**63, size=4000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=4000, dtype=np.uint64)]
    # u near 1 (top bits all ones), u tiny (top bits zero), and the ends
    near1 = np.uint64(0xFFFFFFFFFFFFF000) - (rng.integers(0, 2**45, size=1500, dtype=np.uint64) << np.uint64(12))
    tiny = rng.integers(0, 2**20, size=800, dtype=np.uint64) << np.uint64(12)
    ends = np.array([0, 0xFFFFFFFFFFFFFFFF, 1 << 63, (1 << 63) - 1, 0xFFFFF00000000000], dtype=np.uint64)
    w = np.concatenate(words + [near1, tiny, ends])
    got = neglog_dev(L, w, 0)
    ref = np.empty(w.size)
    ulps = np.empty(w.size)
    for i, x in enumerate(w.tolist()):
        m = x >> 12
        e = -mpmath.log(mpmath.mpf(2 * m + 1) / mpmath.mpf(2) ** 53)
        ref[i] = float(e)
        ulp = mpmath.ldexp(1, int(mpmath.floor(mpmath.log(e, 2))) - 52)
        ulps[i] = float(abs(mpmath.mpf(got[i]) - e) / ulp)
    assert ulps.max() <= 0.501, ulps.max()
    assert np.mean(got != ref) < 1e-3  # correctly rounded almost always
    # CUDA's log (1 ulp) and glibc's agree with it to within one ulp
    cuda = neglog_dev(L, w, 1)
    u = (2.0 * (w >> np.uint64(12)).astype(np.float64) + 1.0) * 2.0 ** -53
    assert ulp_distance(got, cuda).max() <= 1
    assert ulp_distance(got, -np.log(u)).max() <= 1


@pytest.mark.parametrize("fp64", [0, 1])
def test_dmul_and_drcp_bit_exact(L, fp64):
    rng = np.random.default_rng(2 + fp64)
    n = 200000
    a = np.ldexp(1.0 + rng.random(n), rng.integers(-600, 600, size=n))
    b = np.ldexp(1.0 + rng.random(n), rng.integers(-600, 600, size=n))
    a[:1000] = np.ldexp(1.0 + rng.random(1000), rng.integers(-1022, -1000, size=1000))  # near-subnormal products
    b[:1000] = np.ldexp(1.0 + rng.random(1000), rng.integers(-60, 0, size=1000))
    a[1000:2000] = (a[1000:2000].view(np.int64) | 0xFFFFFFF).view(np.float64)          # rounding ties and carries
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    assert L.gm_diag_dmul(P(ta), P(tb), n, fp64, P(out), S()) == 0
    assert np.array_equal(out.cpu().numpy().view(np.int64), (a * b).view(np.int64))
    v = np.concatenate([a, [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, 2.0 ** 1023, 1.7976931348623157e308, 5e-324]])
    tv = torch.from_numpy(v).cuda()
    out = torch.empty(v.size, dtype=torch.float64, device="cuda")
    assert L.gm_diag_drcp(P(tv), v.size, fp64, P(out), S()) == 0
    with np.errstate(over="ignore"):
        want = 1.0 / v
    assert np.array_equal(out.cpu().numpy().view(np.int64), want.view(np.int64))


@pytest.mark.parametrize("k,v", [(1, 0.7), (5, 2.0), (64, 0.01), (1000, 1e-5), (4096, 3.5)])
def test_warp_path_arrivals_match_oracle(L, k, v):
    """Dense and hashed permutations, both arithmetics: servers exact, times <= 4 ulp."""
    ctab = torch.empty(k, dtype=torch.float64, device="cuda")
    for elem in (0, 17, 2**31 - 1):
        b_ref, c_ref = oracle.arrivals(elem, v, k, 123456789)
        outs = []
        for variant in (0, 1, 2, 3):
            n = k if variant < 2 else min(k, 352)
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            c = torch.empty(n, dtype=torch.int32, device="cuda")
            assert L.gm_diag_arrivals(elem, v, k, 123456789, n, variant, P(b), P(c), P(ctab), S()) == 0
            outs.append((b.cpu().numpy(), c.cpu().numpy()))
            assert np.array_equal(outs[-1][1], c_ref[:n])
            assert ulp_distance(outs[-1][0], b_ref[:n]).max() <= 4
        assert ulp_distance(outs[0][0], outs[1][0]).max() <= 4
        assert np.array_equal(outs[0][0][:outs[2][0].size], outs[2][0])  # hash == dense, bit for bit


def test_first_arrival_screen_is_conservative(L):
    rng = np.random.default_rng(5)
    n = 400000
    ids = rng.integers(0, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
    v = np.exp(rng.uniform(np.log(1e-6), np.log(1e3), size=n))
    v[:2000] = np.exp(rng.uniform(np.log(1e-300), np.log(1e-36), size=2000))  # below FP32's normal range
    v[2000:4000] = np.exp(rng.uniform(np.log(1e37), np.log(1e300), size=2000))  # above it
    ti, tv = torch.from_numpy(ids).cuda(), torch.from_numpy(v).cuda()
    scr = torch.empty(n, dtype=torch.uint8, device="cuda")
    b0 = torch.empty(n, dtype=torch.float64, device="cuda")
    for k, T in ((1024, 1e-3), (4096, 2e-5), (128, 0.05), (1, 3.0), (64, 1e30), (256, 1e-33)):
        assert L.gm_diag_first_arrival(P(ti), P(tv), n, k, 77, T, P(scr), P(b0), S()) == 0
        s, b = scr.cpu().numpy().astype(bool), b0.cpu().numpy()
        Tf = float(np.float32(T))
        assert not np.any(s & (b <= Tf)), "screen skipped an arrival within the bound"
        above = (b > Tf) & (v > 1e-30) & (v < 1e30) & (v * Tf > 1e-28)
        if above.any():
            assert s[above].mean() > 0.999  # and it is tight where it decides
