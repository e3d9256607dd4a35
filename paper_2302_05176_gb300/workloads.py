"""Seeded synthetic CSR workloads.

This module holds no arithmetic of the sketch: it only draws inputs.  Both the
CUDA path and the CPU oracle are fed from here, so that the two sides see the
same vectors.  All draws use numpy's PCG64 generator, which gives the same
numbers on x86-64 and aarch64.

The shapes follow the paper's synthetic settings (Sec. 4: weights UNI(0,1) or
EXP(1), n+ from 10^2 to 10^6, k from 2^6 to 2^12) at the sizes of the five
benchmark configurations:

* ``single_vector``   -- one row, n = 10,000 dims, n+ = 1,000 positive entries at
  uniformly random ids, weights Uniform(0, 1], k = 128.
* ``lognormal_batch`` -- 4,096 rows, n+ ~ LogNormal(ln 2000, 1) clipped to
  [10, 200,000], ids uniform without replacement in [0, 2^24) and sorted within
  the row, weights Exp(1).
* ``pareto_heavy``    -- 16 rows of n+ = 1,000,000, weights Pareto(alpha=1.2,
  x_min=1e-3).
* ``serving_requests`` -- a Poisson request stream, n+ log-uniform in
  [100, 5e6], weights an equal mixture of Exp(1) and Pareto(1.5), k uniform in
  {256, 1024, 4096}.
* ``jaccard_pairs``   -- pairs of rows sharing a fraction of their ids, the
  shared weights multiplied by a log-normal perturbation.
"""
from dataclasses import dataclass

import numpy as np

ID_SPACE = 1 << 24


@dataclass
class CSR:
    row_ptr: np.ndarray  # int64 [n_rows + 1]
    ids: np.ndarray      # int32 [nnz]
    w: np.ndarray        # float64 [nnz]

    @property
    def n_rows(self) -> int:
        return int(self.row_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, r):
        lo, hi = int(self.row_ptr[r]), int(self.row_ptr[r + 1])
        return self.ids[lo:hi], self.w[lo:hi]

    def take_rows(self, rows) -> "CSR":
        rows = np.asarray(rows, dtype=np.int64)
        lens = self.row_ptr[rows + 1] - self.row_ptr[rows]
        rp = np.zeros(rows.size + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        ids = np.concatenate([self.row(r)[0] for r in rows]) if rows.size else np.zeros(0, np.int32)
        w = np.concatenate([self.row(r)[1] for r in rows]) if rows.size else np.zeros(0, np.float64)
        return CSR(rp, ids.astype(np.int32), w.astype(np.float64))


def _distinct_ids(rng, n, space):
    """n distinct ids drawn uniformly from [0, space), sorted."""
    if n > space:
        raise ValueError("more ids than the id space")
    if n * 4 > space:
        return np.sort(rng.permutation(space)[:n]).astype(np.int32)
    got = np.unique(rng.integers(0, space, size=int(n * 1.1) + 16))
    while got.size < n:
        got = np.unique(np.concatenate([got, rng.integers(0, space, size=n)]))
    if got.size > n:
        got = np.sort(rng.choice(got, size=n, replace=False))
    return got.astype(np.int32)


def from_rows(rows) -> CSR:
    """Build a CSR from a list of (ids, weights) pairs."""
    lens = np.array([len(r[0]) for r in rows], dtype=np.int64)
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    ids = np.concatenate([np.asarray(r[0], np.int32) for r in rows]) if rows else np.zeros(0, np.int32)
    w = np.concatenate([np.asarray(r[1], np.float64) for r in rows]) if rows else np.zeros(0, np.float64)
    return CSR(rp, ids.astype(np.int32), w.astype(np.float64))


def single_vector(seed=1, n_dims=10_000, n_pos=1_000) -> CSR:
    rng = np.random.default_rng(seed)
    ids = np.sort(rng.choice(n_dims, size=n_pos, replace=False)).astype(np.int32)
    w = 1.0 - rng.random(n_pos)  # Uniform(0, 1]
    return from_rows([(ids, w)])


def lognormal_lengths(rng, n_rows, median=2000.0, sigma=1.0, lo=10, hi=200_000):
    n = np.rint(rng.lognormal(np.log(median), sigma, size=n_rows)).astype(np.int64)
    return np.clip(n, lo, hi)


def lognormal_batch(seed=1, n_rows=4096, median=2000.0, sigma=1.0, lo=10, hi=200_000) -> CSR:
    rng = np.random.default_rng(seed)
    lens = lognormal_lengths(rng, n_rows, median, sigma, lo, hi)
    rows = []
    for n in lens:
        ids = _distinct_ids(rng, int(n), ID_SPACE)
        w = rng.standard_exponential(int(n))
        rows.append((ids, w))
    return from_rows(rows)


def lognormal_batch_device(seed, n_rows=4096, median=2000.0, sigma=1.0, lo=10, hi=200_000, device="cuda"):
    """The lognormal_batch distribution drawn on the device (torch's Philox
    generator), for training sets of many thousands of rows.  Row lengths and
    weights follow lognormal_batch; the ids of row r are the arithmetic
    progression (a_r + i s_r) mod 2^24 with a random start a_r and a random odd
    step s_r, so they are distinct within the row.  Returns device tensors
    (row_ptr int64, ids int32, w float64)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    z = torch.randn(n_rows, generator=g, device=device, dtype=torch.float64)
    lens = torch.exp(np.log(median) + sigma * z).round().clamp_(lo, hi).to(torch.int64)
    row_ptr = torch.zeros(n_rows + 1, dtype=torch.int64, device=device)
    torch.cumsum(lens, 0, out=row_ptr[1:])
    nnz = int(row_ptr[-1].item())
    row = torch.repeat_interleave(torch.arange(n_rows, device=device), lens, output_size=nnz)
    pos = torch.arange(nnz, device=device, dtype=torch.int64) - row_ptr[row]
    start = torch.randint(0, ID_SPACE, (n_rows,), generator=g, device=device, dtype=torch.int64)
    step = torch.randint(0, ID_SPACE // 2, (n_rows,), generator=g, device=device, dtype=torch.int64) * 2 + 1
    ids = ((start[row] + pos * step[row]) % ID_SPACE).to(torch.int32)
    w = torch.empty(nnz, dtype=torch.float64, device=device).exponential_(1.0, generator=g)
    return row_ptr, ids, w


def single_vector_batch_device(seed, n_rows=4096, n_dims=10_000, n_pos=1_000, device="cuda"):
    """Rows of the single_vector law drawn on the device: n_pos positive entries of
    n_dims dimensions, weights Uniform(0, 1].  The ids of row r are the progression
    (a_r + i s_r) mod n_dims with a random start and a random step coprime to
    n_dims (so distinct within the row); the sketch keys its random numbers on the
    id, so this structure is immaterial.  Returns device tensors (row_ptr int64,
    ids int32, w float64)."""
    import math
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    units = torch.tensor([s for s in range(1, n_dims) if math.gcd(s, n_dims) == 1], dtype=torch.int64,
                         device=device)
    row_ptr = torch.arange(n_rows + 1, dtype=torch.int64, device=device) * n_pos
    start = torch.randint(0, n_dims, (n_rows, 1), generator=g, device=device, dtype=torch.int64)
    step = units[torch.randint(0, units.numel(), (n_rows, 1), generator=g, device=device)]
    pos = torch.arange(n_pos, dtype=torch.int64, device=device)[None, :]
    ids = ((start + pos * step) % n_dims).reshape(-1).to(torch.int32)
    w = 1.0 - torch.rand(n_rows * n_pos, generator=g, device=device, dtype=torch.float64)
    return row_ptr, ids, w


def pareto_weights(rng, n, alpha, x_min):
    return x_min * (1.0 + rng.pareto(alpha, size=n))


def pareto_heavy(seed=1, n_rows=16, n_pos=1_000_000, alpha=1.2, x_min=1e-3) -> CSR:
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n_rows):
        ids = _distinct_ids(rng, n_pos, ID_SPACE)
        rows.append((ids, pareto_weights(rng, n_pos, alpha, x_min)))
    return from_rows(rows)


def uniform_rows(seed, n_rows, n_pos, space=ID_SPACE, weight="uniform") -> CSR:
    """Rows of fixed length n_pos (int or array) with Uniform(0,1] or Exp(1) weights."""
    rng = np.random.default_rng(seed)
    lens = np.broadcast_to(np.asarray(n_pos, dtype=np.int64), (n_rows,))
    rows = []
    for n in lens:
        ids = _distinct_ids(rng, int(n), space)
        w = (1.0 - rng.random(int(n))) if weight == "uniform" else rng.standard_exponential(int(n))
        rows.append((ids, w))
    return from_rows(rows)


def jaccard_pairs(seed, n_pairs, n_pos, shared=0.5, sigma=0.2, space=ID_SPACE):
    """Two CSR batches A, B: row p of B shares a fraction `shared` of row p of A's ids.

    Shared entries get the A weight times exp(N(0, sigma^2)); the rest are fresh ids
    with Exp(1) weights.
    """
    rng = np.random.default_rng(seed)
    ra, rb = [], []
    for _ in range(n_pairs):
        ids = _distinct_ids(rng, 2 * n_pos, space)
        rng.shuffle(ids)
        a_ids = ids[:n_pos]
        n_sh = int(round(shared * n_pos))
        b_ids = np.concatenate([a_ids[:n_sh], ids[n_pos:2 * n_pos - n_sh]])
        a_w = rng.standard_exponential(n_pos)
        b_w = np.concatenate([a_w[:n_sh] * np.exp(rng.normal(0.0, sigma, n_sh)),
                              rng.standard_exponential(n_pos - n_sh)])
        oa, ob = np.argsort(a_ids), np.argsort(b_ids)
        ra.append((a_ids[oa], a_w[oa]))
        rb.append((b_ids[ob], b_w[ob]))
    return from_rows(ra), from_rows(rb)


@dataclass
class Request:
    t_arrive: float
    kind: str        # "sketch" | "jaccard" | "cardinality"
    k: int
    csr: CSR = None
    pair: tuple = None   # (handle_a, handle_b) for jaccard
    handle: int = -1     # for cardinality


def _progression_ids(rng, n, space=ID_SPACE):
    """n distinct ids in [0, space): (a + i s) mod space with a random start and a
    random odd step (space a power of two).  O(n), for large request streams; the
    sketch keys its random numbers on the id, so the structure is immaterial."""
    a = int(rng.integers(0, space))
    st = int(rng.integers(0, space // 2)) * 2 + 1
    return ((a + np.arange(n, dtype=np.int64) * st) % space).astype(np.int32)


def serving_requests(seed=1, n_requests=2000, rate=20_000.0, n_lo=100, n_hi=5_000_000,
                     ks=(256, 1024, 4096), query_frac=0.3, pair_frac=0.5, shared=0.5, sigma=0.2,
                     max_nnz=None, n_vectors=None):
    """A Poisson stream of sketch requests plus Jaccard / cardinality queries.

    Sketch sizes n+ are log-uniform in [n_lo, n_hi], weights Exp(1) or
    Pareto(1.5) (an equal mixture), k uniform over ``ks``.  A fraction
    ``pair_frac`` of the sketch requests are partners of an earlier request: they
    keep ``shared`` of its ids with the weights multiplied by exp(N(0, sigma^2)),
    add fresh ids for the rest, and use its k; the Jaccard queries are over such
    pairs, the cardinality queries over any earlier sketch.  Queries refer to
    sketch requests by their index in the stream.  ``max_nnz`` caps n+.  With
    ``n_vectors``, once that many distinct vectors exist every later sketch
    request sketches one of them again (chosen uniformly, k drawn afresh), so a
    long stream needs only that many vectors in host memory.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    hi = n_hi if max_nnz is None else min(n_hi, max_nnz)
    reqs, sketch_idx, pairs = [], [], []
    distinct = []
    for q in range(n_requests):
        if sketch_idx and rng.random() < query_frac:
            if pairs and rng.random() < 0.5:
                a, b = pairs[int(rng.integers(len(pairs)))]
                reqs.append(Request(float(t[q]), "jaccard", reqs[a].k, pair=(a, b)))
            else:
                h = int(rng.choice(sketch_idx))
                reqs.append(Request(float(t[q]), "cardinality", reqs[h].k, handle=h))
            continue
        if n_vectors is not None and len(distinct) >= n_vectors:
            a = distinct[int(rng.integers(len(distinct)))]
            reqs.append(Request(float(t[q]), "sketch", int(rng.choice(ks)), csr=reqs[a].csr))
            sketch_idx.append(q)
            continue
        if sketch_idx and rng.random() < pair_frac:
            a = int(rng.choice(sketch_idx))
            base = reqs[a].csr
            n = base.nnz
            keep = rng.random(n) < shared
            n_fresh = n - int(keep.sum())
            # fresh ids from a block of their own above the base ids' range, so
            # they never repeat a kept id (blocks of 2^23 ids, reused cyclically)
            block = 2 + len(pairs) % 254
            fresh = (block << 23) + _progression_ids(rng, n_fresh, 1 << 23).astype(np.int64)
            ids = np.concatenate([base.ids[keep].astype(np.int64), fresh])
            w = np.concatenate([base.w[keep] * np.exp(rng.normal(0.0, sigma, n - n_fresh)),
                                rng.standard_exponential(n_fresh)])
            if len(pairs) >= 254:  # a reused block may meet a partner's kept ids
                ids, first = np.unique(ids, return_index=True)
                w = w[first]
            reqs.append(Request(float(t[q]), "sketch", reqs[a].k, csr=CSR(np.array([0, ids.size], dtype=np.int64),
                                                                       ids.astype(np.int32), w)))
            pairs.append((a, q))
            sketch_idx.append(q)
            distinct.append(q)
            continue
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(hi))))
        ids = _progression_ids(rng, n)
        w = rng.standard_exponential(n) if rng.random() < 0.5 else pareto_weights(rng, n, 1.5, 1.0)
        k = int(rng.choice(ks))
        reqs.append(Request(float(t[q]), "sketch", k, csr=CSR(np.array([0, n], dtype=np.int64), ids, w)))
        sketch_idx.append(q)
        distinct.append(q)
    return reqs
