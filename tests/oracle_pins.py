"""Pins for the CPU oracle: checks against facts the paper and the mathematics fix.

Each pin returns a list of failure messages (empty = pass), so the pin tests can
assert on it and the planted-mistake tests can show that a mistake makes it fail.
None of these pins calls the CUDA path, and none re-types the oracle's formula:
each compares the oracle with a published vector, a closed form, a library
routine that computes the same quantity independently, or brute force.
"""
import math
import os

import numpy as np
from scipy import stats

import oracle
from paper_2302_05176_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
P_MIN = 1e-4  # family-wise floor for the fixed-seed statistical pins


def _harmonic(n):
    return sum(1.0 / m for m in range(1, n + 1))


def _blocks(v, n_blocks, stride=None):
    """n_blocks copies of the weight vector v, copy r on ids r*stride + l (independent streams)."""
    v = np.asarray(v, dtype=np.float64)
    stride = stride or v.size
    rows = [(np.arange(v.size, dtype=np.int32) + r * stride, v) for r in range(n_blocks)]
    return W.from_rows(rows)


# --------------------------------------------------------------------------- PRNG
def pin_philox_kat():
    fails = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            x = [int(t, 16) for t in line.split()]
            got = oracle.philox(x[0:4], x[4:6])
            if list(got) != x[6:10]:
                fails.append("philox KAT %s -> %s" % (x[:6], [hex(g) for g in got]))
    return fails


def pin_uniform_and_randint():
    fails = []
    lo = oracle.uniform_from_words(0, 0)
    hi = oracle.uniform_from_words(0xFFFFFFFF, 0xFFFFFFFF)
    if lo != 2.0 ** -53 or not (0.0 < lo):
        fails.append("u(0,0) != 2^-53")
    if hi != 1.0 - 2.0 ** -53 or not (hi < 1.0):
        fails.append("u(max) != 1 - 2^-53 (must stay below 1)")
    # the top 52 bits of (w1:w0) define m; u = (2m+1) 2^-53, exactly
    from fractions import Fraction
    for x in (0x123456789ABCDEF0, 0xFFFFFFFFFFFFF000, 0x8000000000000000, 0x0000000000001FFF):
        m = x >> 12
        got = oracle.uniform_from_words(x & 0xFFFFFFFF, x >> 32)
        if Fraction(got) != Fraction(2 * m + 1, 2 ** 53):
            fails.append("u(%x) is not exactly (2m+1)2^-53" % x)
    # RandInt(z, k) = z + floor(r (k - z) / 2^64)
    for (r, z, k) in [(0, 3, 10), (2 ** 64 - 1, 3, 10), (2 ** 63, 0, 7), (0x5555555555555555, 2, 5)]:
        want = z + (r * (k - z)) // 2 ** 64
        got = oracle.randint_from_words(r & 0xFFFFFFFF, r >> 32, z, k)
        if got != want:
            fails.append("randint(%x,%d,%d)=%d want %d" % (r, z, k, got, want))
    return fails


# --------------------------------------------------------------------------- exact sum
def pin_exact_sum(seed=11):
    """The oracle's exact accumulator against math.fsum (a correctly rounded sum)."""
    fails = []
    rng = np.random.default_rng(seed)
    for trial in range(300):
        n = int(rng.integers(1, 400))
        expo = rng.integers(-70, 6, size=n)
        t = np.ldexp(1.0 + rng.random(n), expo)
        got = oracle.exact_sum(t)
        want = math.fsum(t.tolist())
        if got != want:
            fails.append("exact_sum trial %d: %r vs fsum %r" % (trial, got, want))
            break
    # ties to even and sticky bits
    cases = [([1.0, 2.0 ** -53], 1.0),
             ([1.0, 2.0 ** -53, 2.0 ** -100], 1.0 + 2.0 ** -52),
             ([1.0 + 2.0 ** -52, 2.0 ** -53], 1.0 + 2.0 ** -51),
             ([2.0 ** -60] * 1024, 2.0 ** -50)]
    for terms, want in cases:
        got = oracle.exact_sum(terms)
        if got != want:
            fails.append("exact_sum %r -> %r want %r" % (terms[:3], got, want))
    return fails


# --------------------------------------------------------------------------- arrivals
def _streams(k, v, n_elem, seed):
    B = np.zeros((n_elem, k))
    C = np.zeros((n_elem, k), dtype=np.int64)
    for i in range(n_elem):
        B[i], C[i] = oracle.arrivals(i, v, k, seed)
    return B, C


def pin_order_statistics(k=12, v=0.5, n_elem=6000, seed=3):
    """Eq. biz_dis: b_(z) v is the z-th order statistic of k iid Exp(1) (Renyi).

    E[b_(z) v] = H_k - H_{k-z}, Var = sum_{l=k-z+1}^{k} 1/l^2 (1-based z); the
    pooled values are iid Exp(1); the servers of a full stream are a permutation.
    """
    fails = []
    B, C = _streams(k, v, n_elem, seed)
    X = B * v
    for z in range(k):  # 0-based step z is order statistic z+1
        mean = sum(1.0 / (k - l) for l in range(z + 1))
        var = sum(1.0 / (k - l) ** 2 for l in range(z + 1))
        se = math.sqrt(var / n_elem)
        if abs(X[:, z].mean() - mean) > 5 * se:
            fails.append("order stat %d: mean %.4f want %.4f" % (z, X[:, z].mean(), mean))
        if abs(X[:, z].var() / var - 1.0) > 0.15:
            fails.append("order stat %d: var %.4f want %.4f" % (z, X[:, z].var(), var))
    if np.any(np.diff(B, axis=1) < 0):
        fails.append("arrival times not ascending")
    if not all(sorted(row) == list(range(k)) for row in C[:200].tolist()):
        fails.append("servers of a full stream are not a permutation")
    p = stats.kstest(X.ravel()[::7], "expon").pvalue
    if p < P_MIN:
        fails.append("pooled b*v not Exp(1): p=%g" % p)
    return fails


def pin_server_uniformity(k=8, n_elem=20000, seed=5):
    """Fisher-Yates (Sec. 2.2): the server at any step is uniform over k, and the
    first two servers are a uniform ordered pair of distinct servers."""
    fails = []
    C = np.zeros((n_elem, 3), dtype=np.int64)
    for i in range(n_elem):
        _, c = oracle.arrivals(i, 1.0, k, seed, n_steps=3)
        C[i] = c
    for z in range(3):
        counts = np.bincount(C[:, z], minlength=k)
        p = stats.chisquare(counts).pvalue
        if p < P_MIN:
            fails.append("server at step %d not uniform: p=%g counts=%s" % (z, p, counts.tolist()))
    if np.any(C[:, 0] == C[:, 1]):
        fails.append("a server was visited twice")
    pair = C[:, 0] * k + C[:, 1]
    counts = np.bincount(pair, minlength=k * k).reshape(k, k)
    off = counts[~np.eye(k, dtype=bool)]
    p = stats.chisquare(off).pvalue
    if p < P_MIN:
        fails.append("ordered server pairs not uniform: p=%g" % p)
    return fails


def pin_brute_force(seed=7):
    """P10: tiny vectors; the full arrival matrix (k arrivals of every element,
    placed by server) and its column minima (Eq. sjv / yjpi) give the sketch, and
    the second entry of each column in (time, id) order its runner-up."""
    fails = []
    rng = np.random.default_rng(seed)
    for trial in range(60):
        k = int(rng.integers(1, 5))
        n = int(rng.integers(1, 5))
        ids = np.sort(rng.choice(50, size=n, replace=False)).astype(np.int32)
        w = rng.random(n) + 0.05
        w[rng.random(n) < 0.2] = 0.0
        M = np.full((n, k), np.inf)
        for a in range(n):
            if w[a] > 0:
                b, c = oracle.arrivals(int(ids[a]), float(w[a]), k, 99)
                M[a, c] = b
        want_y = M.min(axis=0)
        want_s = np.array([int(ids[np.flatnonzero(M[:, j] == want_y[j])].min()) if np.isfinite(want_y[j]) else -1
                           for j in range(k)])
        want_y2, want_s2 = np.full(k, np.inf), np.full(k, -1)
        for j in range(k):
            cand = sorted((M[a, j], int(ids[a])) for a in range(n) if np.isfinite(M[a, j]))
            if len(cand) >= 2:
                want_y2[j], want_s2[j] = cand[1]
        s, y, y2, s2 = oracle.sketch([0, n], ids, w, k, 99, runner_up=True)
        if not (np.array_equal(s[0], want_s) and np.array_equal(y[0], want_y)):
            fails.append("brute force trial %d: %s %s vs %s %s" % (trial, s[0], y[0], want_s, want_y))
        if not (np.array_equal(s2[0], want_s2) and np.array_equal(y2[0], want_y2)):
            fails.append("brute force runner-up trial %d: %s %s vs %s %s" % (trial, s2[0], y2[0], want_s2, want_y2))
    return fails


# --------------------------------------------------------------------------- sketch statistics
def pin_argmax_distribution(n_rows=20000, k=16, seed=1):
    """P(s_j = i) = v_i / sum v (Sec. 1), chi-square over independent copies."""
    fails = []
    v = np.array([0.5, 1.0, 1.5, 2.0, 3.0])
    X = _blocks(v, n_rows)
    s, y = oracle.sketch(X.row_ptr, X.ids, X.w, k, seed)
    for j in (0, k // 2):
        idx = s[:, j] - np.arange(n_rows) * v.size
        counts = np.bincount(idx, minlength=v.size)
        p = stats.chisquare(counts, n_rows * v / v.sum()).pvalue
        if p < P_MIN:
            fails.append("argmax distribution register %d: p=%g counts=%s" % (j, p, counts.tolist()))
    return fails


def pin_register_law(n_rows=8000, k=16, seed=2):
    """y_j ~ Exp(sum v) (Sec. 1): KS on y_j * sum v; and the max over registers
    y* sum v has CDF (1 - e^-t)^k, mean H_k (Sec. 2.3 Time Complexity)."""
    fails = []
    v = np.array([0.2, 0.7, 1.1, 0.05, 2.5])
    X = _blocks(v, n_rows)
    s, y = oracle.sketch(X.row_ptr, X.ids, X.w, k, seed)
    Y = y * v.sum()
    for j in (0, 5, k - 1):
        p = stats.kstest(Y[:, j], "expon").pvalue
        if p < P_MIN:
            fails.append("register %d not Exp(sum v): p=%g" % (j, p))
    ystar = Y.max(axis=1)
    p = stats.kstest(ystar, lambda t: (1.0 - np.exp(-np.maximum(t, 0))) ** k).pvalue
    if p < P_MIN:
        fails.append("y* law: p=%g" % p)
    hk = _harmonic(k)
    se = math.sqrt(sum(1.0 / m ** 2 for m in range(1, k + 1)) / n_rows)
    if abs(ystar.mean() - hk) > 5 * se:
        fails.append("E[y* sum v] %.4f vs H_k %.4f" % (ystar.mean(), hk))
    return fails


def pin_cardinality(n_rows=6000, k=16, seed=4):
    """(k-1)/sum_j y_j is unbiased for sum v (Lemiesz; Sec. 2.4 theorem), and
    from the Gamma(k, c) law of sum_j y_j its relative variance is exactly 1/(k-2)."""
    fails = []
    v = np.array([0.3, 0.9, 1.7, 0.4])
    c = v.sum()
    X = _blocks(v, n_rows)
    _, y = oracle.sketch(X.row_ptr, X.ids, X.w, k, seed)
    est = oracle.cardinality(y)
    sigma = c / math.sqrt((k - 2) * n_rows)
    if abs(est.mean() - c) > 4 * sigma:
        fails.append("cardinality mean %.4f vs %.4f (sigma %.4f)" % (est.mean(), c, sigma))
    rel_var = est.var() / c ** 2
    if abs(rel_var * (k - 2) - 1.0) > 0.15:
        fails.append("cardinality rel. variance %.4f vs 1/(k-2)=%.4f" % (rel_var, 1.0 / (k - 2)))
    return fails


def jaccard_probability(u, v):
    """Probability Jaccard J_P (Sec. 1), straight from its definition."""
    u = np.asarray(u, float)
    v = np.asarray(v, float)
    total = 0.0
    for i in range(u.size):
        if u[i] > 0 and v[i] > 0:
            total += 1.0 / np.sum(np.maximum(u / u[i], v / v[i]))
    return total


def pin_jaccard_collision(n_pairs=3000, k=32, seed=6):
    """E[(1/k) sum 1(s_j(u)=s_j(v))] = J_P(u, v), Var = J(1-J)/k (Sec. 2.4 theorem)."""
    fails = []
    u = np.array([1.0, 2.0, 0.0, 3.0, 0.5, 1.0])
    v = np.array([2.0, 1.0, 1.0, 0.0, 0.5, 1.5])
    J = jaccard_probability(u, v)
    A = _blocks(u, n_pairs)
    B = _blocks(v, n_pairs)
    sa, _ = oracle.sketch(A.row_ptr, A.ids, A.w, k, seed)
    sb, _ = oracle.sketch(B.row_ptr, B.ids, B.w, k, seed)
    est = oracle.jaccard(sa, sb)
    se = math.sqrt(J * (1 - J) / (k * n_pairs))
    if abs(est.mean() - J) > 5 * se:
        fails.append("collision rate %.4f vs J_P %.4f (se %.4f)" % (est.mean(), J, se))
    if abs(est.var() / (J * (1 - J) / k) - 1.0) > 0.15:
        fails.append("collision variance %.5f vs J(1-J)/k %.5f" % (est.var(), J * (1 - J) / k))
    return fails


def pin_merge_and_scale(seed=8):
    """Sec. 2.3 Mergeability: the register-wise min of two sketches is the sketch
    of the union; scaling v by 2 halves y exactly and keeps s (the sketch of v and
    of its normalised vector agree, Sec. 2.3 Time Complexity); ties in a merge
    go to the smaller id."""
    fails = []
    rng = np.random.default_rng(seed)
    k = 24
    for trial in range(8):
        ids = np.sort(rng.choice(5000, size=60, replace=False)).astype(np.int32)
        w = rng.exponential(size=60)
        a = rng.random(60) < 0.5
        sA, yA = oracle.sketch([0, int(a.sum())], ids[a], w[a], k, seed)
        sB, yB = oracle.sketch([0, int((~a).sum())], ids[~a], w[~a], k, seed)
        sU, yU = oracle.sketch([0, 60], ids, w, k, seed)
        sM, yM = oracle.merge(sA, yA, sB, yB)
        if not (np.array_equal(sM, sU) and np.array_equal(yM, yU)):
            fails.append("merge != sketch of union (trial %d)" % trial)
        s2, y2 = oracle.sketch([0, 60], ids, 2.0 * w, k, seed)
        if not (np.array_equal(s2, sU) and np.array_equal(2.0 * y2, yU)):
            fails.append("scaling by 2 changed the sketch (trial %d)" % trial)
    s, y = oracle.merge(np.array([5, 9], np.int32), np.array([1.0, 2.0]),
                        np.array([3, 9], np.int32), np.array([1.0, 1.5]))
    if s.tolist() != [3, 9] or y.tolist() != [1.0, 1.5]:
        fails.append("merge tie/min rule: %s %s" % (s, y))
    return fails


def pin_empty_and_zero():
    fails = []
    s, y = oracle.sketch([0, 0, 3], np.array([4, 8, 9], np.int32), np.array([0.0, 0.0, 0.0]), 5, 1)
    if not (np.all(s == -1) and np.all(np.isinf(y))):
        fails.append("empty / all-zero rows must be unfilled")
    s1, y1 = oracle.sketch([0, 3], np.array([4, 8, 9], np.int32), np.array([0.0, 1.0, 0.0]), 5, 1)
    s2, y2 = oracle.sketch([0, 1], np.array([8], np.int32), np.array([1.0]), 5, 1)
    if not (np.array_equal(s1, s2) and np.array_equal(y1, y2)):
        fails.append("zero weights must not take part")
    return fails


# --------------------------------------------------------------------------- Algorithms 1 and 2
def pin_fastsearch_budgets():
    with open(os.path.join(GOLDEN, "fastsearch_budgets_example.txt")) as f:
        rec = {ln.split()[0]: ln.split()[1:] for ln in f if ln.strip() and not ln.startswith("#")}
    v = np.array([float(x) for x in rec["v"]])
    R = int(rec["R"][0])
    k = int(rec["k"][0])
    fails = []
    if R != math.ceil(k * math.log(k)):
        fails.append("R != ceil(k ln k)")
    got = oracle.fastsearch_budgets(v, R)
    if got.tolist() != [int(x) for x in rec["R_i"]] or int(got.sum()) != int(rec["sum"][0]):
        fails.append("budgets %s (sum %d)" % (got.tolist(), got.sum()))
    return fails


def pin_alg1_equals_full_stream(seed=9):
    """Pruning never changes a register (Sec. 1, Sec. 2.2): Algorithm 1 returns
    exactly the unpruned sketch, with far fewer arrivals than k n+."""
    fails = []
    rng = np.random.default_rng(seed)
    for trial, (n, k) in enumerate([(1, 8), (3, 16), (40, 8), (300, 64), (1000, 128), (60, 256)]):
        ids = np.sort(rng.choice(100000, size=n, replace=False)).astype(np.int32)
        w = rng.random(n) if trial % 2 else rng.exponential(size=n)
        s0, y0 = oracle.sketch([0, n], ids, w, k, seed)
        s1, y1, arr = oracle.fastgm_alg1(ids, w, k, seed)
        if not (np.array_equal(s0[0], s1) and np.array_equal(y0[0], y1)):
            fails.append("Algorithm 1 != unpruned (n=%d k=%d)" % (n, k))
        if n * k >= 10000 and arr > 0.5 * n * k:
            fails.append("Algorithm 1 generated %d of %d arrivals" % (arr, n * k))
    return fails


def pin_stream_fastgm(seed=10):
    """Algorithm 2 over a stream with repeats equals the sketch of its distinct set (Sec. 3)."""
    fails = []
    rng = np.random.default_rng(seed)
    for trial in range(5):
        k = [16, 64, 128, 32, 8][trial]
        n = int(rng.integers(5, 400))
        ids = rng.choice(100000, size=n, replace=False).astype(np.int32)
        w = rng.random(n) + 0.01
        pick = rng.integers(0, n, size=3 * n)
        s0, y0 = oracle.sketch([0, n], ids[np.argsort(ids)], w[np.argsort(ids)], k, seed)
        s1, y1, _ = oracle.stream_fastgm(ids[pick], w[pick], k, seed)
        present = np.unique(pick)
        sD, yD = oracle.sketch([0, present.size], ids[present], w[present], k, seed)
        if not (np.array_equal(sD[0], s1) and np.array_equal(yD[0], y1)):
            fails.append("Stream-FastGM != sketch of the distinct set (trial %d)" % trial)
    return fails


ALL_PINS = [pin_philox_kat, pin_uniform_and_randint, pin_exact_sum, pin_order_statistics,
            pin_server_uniformity, pin_brute_force, pin_argmax_distribution, pin_register_law,
            pin_cardinality, pin_jaccard_collision, pin_merge_and_scale, pin_empty_and_zero,
            pin_fastsearch_budgets, pin_alg1_equals_full_stream, pin_stream_fastgm]
