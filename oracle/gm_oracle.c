/*
 * gm_oracle.c -- plain, slow CPU oracle for the k-register Gumbel-Max sketch.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline
 * / reference leg use it.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only through the seeded input generators.
 *
 * What it computes (paper: Zhang et al., "Fast Gumbel-Max Sketch and its
 * Applications", arXiv 2302.05176):
 *
 *   For a non-negative vector v and k registers, register j holds
 *       y_j = min_{i: v_i > 0} b_{i,j}      s_j = argmin (ties: smallest id)
 *   (Eq. sjv and Eq. yjpi, Sec. 1), where element i's k variables are produced
 *   in ascending order as the exponential order statistics of Eq. biz_dis
 *   (Sec. 2.2, "Generating Ascending Exponential Random Variables"):
 *       b_{i,(z)} = (1/v_i) * sum_{n=1}^{z} (-ln u_{i,n}) / (k - n + 1)
 *   and the z-th of them is handed to server pi_{i,z} of a Fisher-Yates shuffle
 *   (same section).  The oracle is the UNPRUNED full stream: all k arrivals of
 *   every positive element, so it needs no pruning argument at all.
 *
 * Readings of the paper fixed here (the paper leaves them open):
 *   R1  RandUNI / RandInt (Algorithm 1) are one Philox4x32-10 call (Salmon et al.,
 *       SC'11) per arrival: key = (seed_lo, seed_hi), counter = (id, z, 0, 0)
 *       with z the 0-based step.  Words 0,1 give the 52-bit m = (w1:w0) >> 12
 *       and u = (2m+1) * 2^-53: exact in double (2m+1 < 2^53) and never 0 or 1,
 *       the open-interval uniform RandUNI(0,1) asks for.  Words 2,3 give the 64-bit
 *       r and RandInt(z, k) = z + floor(r * (k - z) / 2^64).
 *   R2  Rounding: E = RN(-ln u) (here: libm log), C_z = RN(1/(k-z)),
 *       t_z = RN(E * C_z), S_z = RN(t_0 + ... + t_z) with the sum formed
 *       EXACTLY and rounded once (an exact fixed-point accumulator below),
 *       R = RN(1/v), b_z = RN(S_z * R).  All roundings are to nearest-even.
 *   R3  Ties in a register go to the smallest element id.
 *   R4  An unfilled register is y = +inf, s = -1 (the paper uses y = -1).
 *       An arrival that is not finite never enters a register.
 *
 * Compile with -O2 -ffp-contract=off so that no product is fused into a sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GMO_OK 0
#define GMO_EINVAL 1
#define GMO_ENOMEM 2
#define GMO_ERANGE 3

/* ---- planted-mistake switch: tests set it to show that the pins catch errors --- */
static int g_mutation = 0;
void gmo_set_mutation(int m) { g_mutation = m; }
int gmo_get_mutation(void) { return g_mutation; }

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box, the key bumped by
 * the Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
void gmo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The four Philox words of arrival z of element id (reading R1). */
static void arrival_words(uint64_t seed, int32_t id, uint32_t z, uint32_t w[4]) {
  uint32_t ctr[4] = {(uint32_t)id, z, 0u, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  gmo_philox4x32_10(ctr, key, w);
}

/* u in (0,1) from words 0,1 (reading R1); exact in double. */
double gmo_uniform_from_words(uint32_t w0, uint32_t w1) {
  uint64_t x = ((uint64_t)w1 << 32) | (uint64_t)w0;
  uint64_t m = x >> 12;
  if (g_mutation == 5) m = x >> 13; /* planted: drop a bit of the uniform */
  return ldexp((double)(2 * m + 1), -53);
}

/* RandInt(z, k) from words 2,3 (reading R1): uniform in [z, k). */
int32_t gmo_randint_from_words(uint32_t w2, uint32_t w3, int32_t z, int32_t k) {
  uint64_t r = ((uint64_t)w3 << 32) | (uint64_t)w2;
  unsigned __int128 prod = (unsigned __int128)r * (unsigned __int128)(uint64_t)(k - z);
  return z + (int32_t)(uint64_t)(prod >> 64);
}

/* ---------------------------------------------------------------------------
 * Exact accumulator for reading R2.  value = sum_i limb[i] * 2^(64 i - 160).
 * It holds exactly any sum of non-negative doubles whose lowest mantissa bit is
 * at least 2^-160 and whose total stays below 2^90.  The method's terms lie in
 * [2^-70, 2^6) (E >= 2^-53, C >= 2^-16) and a stream sums at most 65536 of them,
 * so every prefix sum the method forms is exact here.
 * ------------------------------------------------------------------------- */
typedef struct {
  uint64_t limb[4];
} gmo_acc;

static void acc_zero(gmo_acc* a) { memset(a, 0, sizeof(*a)); }

/* Add the 64-bit word x at limb position li, carrying upwards. */
static int acc_add_word(gmo_acc* a, int li, uint64_t x) {
  while (x != 0) {
    if (li > 3) return GMO_ERANGE;
    uint64_t before = a->limb[li];
    a->limb[li] = before + x;
    x = (a->limb[li] < before) ? 1u : 0u; /* carry out */
    ++li;
  }
  return GMO_OK;
}

static int acc_add(gmo_acc* a, double t) {
  if (t == 0.0) return GMO_OK;
  if (!(t > 0.0) || !isfinite(t)) return GMO_ERANGE;
  int e;
  double fr = frexp(t, &e);                  /* t = fr * 2^e, fr in [0.5, 1) */
  uint64_t M = (uint64_t)ldexp(fr, 53);     /* exact: t = M * 2^(e - 53)    */
  int off = e - 53 + 160;                   /* bit index of M's lowest bit  */
  if (off < 0 || off + 53 > 250) return GMO_ERANGE;
  int li = off / 64, sh = off % 64;
  uint64_t lo = M << sh;
  uint64_t hi = sh ? (M >> (64 - sh)) : 0;
  int rc = acc_add_word(a, li, lo);
  if (rc == GMO_OK && hi) rc = acc_add_word(a, li + 1, hi);
  return rc;
}

static int acc_bit(const gmo_acc* a, int pos) {
  if (pos < 0) return 0;
  return (int)((a->limb[pos / 64] >> (pos % 64)) & 1u);
}

/* Is any bit strictly below position pos set? */
static int acc_any_below(const gmo_acc* a, int pos) {
  if (pos <= 0) return 0;
  int li = pos / 64, sh = pos % 64;
  for (int i = 0; i < li; ++i)
    if (a->limb[i]) return 1;
  if (sh && (a->limb[li] & ((((uint64_t)1) << sh) - 1))) return 1;
  return 0;
}

/* Bits [lsb, lsb + 53) as an integer. */
static uint64_t acc_bits53(const gmo_acc* a, int lsb) {
  uint64_t v = 0;
  for (int b = 52; b >= 0; --b) v = (v << 1) | (uint64_t)acc_bit(a, lsb + b);
  return v;
}

/* Round the exact value to the nearest double (ties to even). */
static double acc_round(const gmo_acc* a) {
  int top = 3;
  while (top >= 0 && a->limb[top] == 0) --top;
  if (top < 0) return 0.0;
  int p = top * 64 + 63 - __builtin_clzll(a->limb[top]); /* highest set bit */
  if (p <= 52) return ldexp((double)a->limb[0], -160);   /* fits 53 bits: exact */
  int lsb = p - 52;
  uint64_t mant = acc_bits53(a, lsb);
  int round_bit = acc_bit(a, lsb - 1);
  int sticky = acc_any_below(a, lsb - 1);
  if (round_bit && (sticky || (mant & 1u))) mant += 1; /* may reach 2^53: still exact */
  return ldexp((double)mant, lsb - 160);
}

/* Testing hook: the exactly rounded sum of n non-negative doubles. */
int gmo_exact_sum(const double* t, int64_t n, double* out) {
  gmo_acc a;
  acc_zero(&a);
  for (int64_t i = 0; i < n; ++i) {
    int rc = acc_add(&a, t[i]);
    if (rc) return rc;
  }
  *out = acc_round(&a);
  return GMO_OK;
}

/* ---------------------------------------------------------------------------
 * One element's arrival stream (Eq. biz_dis / Eq. biz_biz-1 plus the
 * Fisher-Yates server assignment, Sec. 2.2), unpruned.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t id, k;
  uint64_t seed;
  double r;        /* R = RN(1/v) */
  int32_t z;       /* next 0-based step */
  gmo_acc acc;     /* exact sum of the terms so far */
  int32_t* perm;   /* Fisher-Yates array, k entries */
} gmo_stream;

static int stream_init(gmo_stream* st, int32_t id, double v, int32_t k, uint64_t seed) {
  st->id = id;
  st->k = k;
  st->seed = seed;
  st->r = 1.0 / v;
  st->z = 0;
  acc_zero(&st->acc);
  st->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  if (!st->perm) return GMO_ENOMEM;
  for (int32_t j = 0; j < k; ++j) st->perm[j] = j;
  return GMO_OK;
}

static void stream_free(gmo_stream* st) {
  free(st->perm);
  st->perm = NULL;
}

/* Produce the next arrival: time *b and server *c.  Returns GMO_OK or an error. */
static int stream_next(gmo_stream* st, double* b, int32_t* c) {
  const int32_t z = st->z, k = st->k;
  uint32_t w[4];
  arrival_words(st->seed, st->id, (uint32_t)z, w);
  double u = gmo_uniform_from_words(w[0], w[1]);
  double E = -log(u);
  double Cz = 1.0 / (double)(k - z);
  if (g_mutation == 1) Cz = 1.0 / (double)k;           /* planted: no order statistics */
  if (g_mutation == 2) Cz = 1.0 / (double)(k - z + 1);  /* planted: off-by-one divisor */
  double t = E * Cz;
  int rc = acc_add(&st->acc, t);
  if (rc) return rc;
  double S = acc_round(&st->acc);
  *b = S * st->r;
  int32_t J = gmo_randint_from_words(w[2], w[3], z, k);
  if (g_mutation == 3) J = z; /* planted: no shuffle */
  int32_t tmp = st->perm[z];
  st->perm[z] = st->perm[J];
  st->perm[J] = tmp;
  *c = st->perm[z];
  if (g_mutation == 4) *c = st->perm[J]; /* planted: wrong slot read after the swap */
  st->z = z + 1;
  return GMO_OK;
}

/* Testing hook: the first n_steps arrivals (time, server) of element (id, v). */
int gmo_arrivals(int32_t id, double v, int32_t k, uint64_t seed, int32_t n_steps, double* b_out,
                 int32_t* c_out) {
  if (k < 1 || n_steps < 0 || n_steps > k || id < 0 || !(v > 0.0) || !isfinite(v)) return GMO_EINVAL;
  gmo_stream st;
  int rc = stream_init(&st, id, v, k, seed);
  if (rc) return rc;
  for (int32_t z = 0; z < n_steps && rc == GMO_OK; ++z) rc = stream_next(&st, &b_out[z], &c_out[z]);
  stream_free(&st);
  return rc;
}

/* Register update (reading R3): lexicographic min of (time, id). */
static int better(double b, int32_t id, double y, int32_t s) {
  if (g_mutation == 6) return b < y || (b == y && id > s); /* planted: ties to largest id */
  return b < y || (b == y && id < s);
}

static int check_weight(double v) {
  if (v != v || v < 0.0 || !isfinite(v)) return GMO_EINVAL;
  return GMO_OK;
}

/* ---------------------------------------------------------------------------
 * The unpruned sketch of CSR rows.  y2_out and s2_out (nullable) receive, per
 * register, the runner-up: the second candidate in the register's (time, id)
 * order over distinct elements, so that a caller can tell which registers are
 * decided by a near-tie and which element would win it the other way
 * (+inf / -1 when fewer than two elements reach the register).
 * Unfilled registers: y = +inf, s = -1.
 * ------------------------------------------------------------------------- */
int gmo_sketch_rows(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                    int32_t k, uint64_t seed, int32_t* s_out, double* y_out, double* y2_out,
                    int32_t* s2_out) {
  if (n_rows < 0 || k < 1) return GMO_EINVAL;
  for (int32_t row = 0; row < n_rows; ++row) {
    int32_t* s = s_out + (int64_t)row * k;
    double* y = y_out + (int64_t)row * k;
    double* y2 = y2_out ? y2_out + (int64_t)row * k : NULL;
    int32_t* s2 = s2_out ? s2_out + (int64_t)row * k : NULL;
    for (int32_t j = 0; j < k; ++j) {
      s[j] = INT32_MAX;
      y[j] = INFINITY;
      if (y2) y2[j] = INFINITY;
      if (s2) s2[j] = INT32_MAX;
    }
    if (row_ptr[row + 1] < row_ptr[row]) return GMO_EINVAL;
    for (int64_t e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
      double v = w[e];
      int32_t id = ids[e];
      if (check_weight(v) || id < 0) return GMO_EINVAL;
      if (v == 0.0) continue; /* only positive elements take part (N^+, Sec. 1) */
      gmo_stream st;
      int rc = stream_init(&st, id, v, k, seed);
      if (rc) return rc;
      for (int32_t z = 0; z < k; ++z) {
        double b;
        int32_t c;
        rc = stream_next(&st, &b, &c);
        if (rc) break;
        if (!isfinite(b)) continue; /* reading R4 */
        if (better(b, id, y[c], s[c])) {
          if (y2) y2[c] = y[c];
          if (s2) s2[c] = s[c];
          y[c] = b;
          s[c] = id;
        } else if (y2 && better(b, id, y2[c], s2 ? s2[c] : INT32_MAX)) {
          y2[c] = b;
          if (s2) s2[c] = id;
        }
      }
      stream_free(&st);
      if (rc) return rc;
    }
    for (int32_t j = 0; j < k; ++j) {
      if (s[j] == INT32_MAX) s[j] = -1;
      if (s2 && s2[j] == INT32_MAX) s2[j] = -1;
    }
  }
  return GMO_OK;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 (FastGM) on one vector, as a host cross-check of the pruning
 * logic.  Same arrivals as above; FastSearch releases ceil(R * v_i / sum v)
 * arrivals per element with R growing by delta until every register is filled;
 * FastPrune then streams each element until its arrival exceeds y* = max_j y_j
 * (or its k arrivals are spent), refreshing y* whenever the register holding
 * the maximum improves.  arrivals_out counts the arrivals generated.
 * ------------------------------------------------------------------------- */
int gmo_fastsearch_budgets(const double* v, int64_t n, int64_t R, int64_t* out) {
  double sum = 0.0;
  for (int64_t i = 0; i < n; ++i) sum += v[i];
  for (int64_t i = 0; i < n; ++i) out[i] = (int64_t)ceil((double)R * (v[i] / sum));
  return GMO_OK;
}

static double max_register(const double* y, int32_t k, int32_t* jmax) {
  double m = -INFINITY;
  *jmax = 0;
  for (int32_t j = 0; j < k; ++j)
    if (y[j] > m) {
      m = y[j];
      *jmax = j;
    }
  return m;
}

int gmo_fastgm_alg1(const int32_t* ids, const double* w, int64_t n, int32_t k, uint64_t seed,
                    int32_t delta, int32_t* s, double* y, int64_t* arrivals_out, int64_t* search_R_out,
                    int64_t* search_arrivals_out) {
  if (k < 1 || n < 0 || delta < 1) return GMO_EINVAL;
  for (int32_t j = 0; j < k; ++j) {
    s[j] = INT32_MAX;
    y[j] = INFINITY;
  }
  /* the positive elements N^+ and their sum (for the normalised weights v*) */
  int64_t np = 0;
  double sum = 0.0;
  for (int64_t e = 0; e < n; ++e) {
    if (check_weight(w[e]) || ids[e] < 0) return GMO_EINVAL;
    if (w[e] > 0.0) {
      ++np;
      sum += w[e];
    }
  }
  gmo_stream* st = (gmo_stream*)calloc((size_t)(np ? np : 1), sizeof(gmo_stream));
  double* vstar = (double*)calloc((size_t)(np ? np : 1), sizeof(double));
  if (!st || !vstar) {
    free(st);
    free(vstar);
    return GMO_ENOMEM;
  }
  int rc = GMO_OK;
  int64_t q = 0;
  for (int64_t e = 0; e < n && rc == GMO_OK; ++e)
    if (w[e] > 0.0) {
      vstar[q] = w[e] / sum;
      rc = stream_init(&st[q++], ids[e], w[e], k, seed);
    }
  int64_t arrivals = 0;
  int32_t unfilled = k;
  int64_t R = 0;
  /* FastSearch: release ceil(R v*_i) arrivals of every queue, R += delta, until no server is empty */
  while (rc == GMO_OK && unfilled > 0 && np > 0) {
    R += delta;
    for (int64_t i = 0; i < np && rc == GMO_OK; ++i) {
      gmo_stream* S = &st[i];
      int64_t Ri = (int64_t)ceil((double)R * vstar[i]);
      while (S->z < Ri && S->z < k) {
        double b;
        int32_t c;
        rc = stream_next(S, &b, &c);
        if (rc) break;
        ++arrivals;
        if (!isfinite(b)) continue;
        if (better(b, S->id, y[c], s[c])) {
          if (y[c] == INFINITY) --unfilled;
          y[c] = b;
          s[c] = S->id;
        }
      }
    }
  }
  if (search_R_out) *search_R_out = R;                 /* the budget at which no server was empty */
  if (search_arrivals_out) *search_arrivals_out = arrivals;
  /* FastPrune: stream every queue until its next arrival exceeds y* (or its k arrivals are spent) */
  if (rc == GMO_OK && np > 0) {
    int32_t jstar;
    double ystar = max_register(y, k, &jstar);
    for (int64_t i = 0; i < np && rc == GMO_OK; ++i) {
      gmo_stream* S = &st[i];
      while (S->z < k) {
        double b;
        int32_t c;
        rc = stream_next(S, &b, &c);
        if (rc) break;
        ++arrivals;
        if (b > ystar) break;
        if (better(b, S->id, y[c], s[c])) {
          y[c] = b;
          s[c] = S->id;
          if (c == jstar) ystar = max_register(y, k, &jstar);
        }
      }
    }
  }
  for (int64_t i = 0; i < q; ++i) stream_free(&st[i]);
  free(st);
  free(vstar);
  for (int32_t j = 0; j < k; ++j)
    if (s[j] == INT32_MAX) s[j] = -1;
  if (arrivals_out) *arrivals_out = arrivals;
  return rc;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2 (Stream-FastGM): one pass over a stream in which an element may
 * occur many times.  Before every register is filled an element's whole stream
 * is generated; afterwards it stops at its first arrival above y*.
 * ------------------------------------------------------------------------- */
int gmo_stream_fastgm(const int32_t* ids, const double* w, int64_t n, int32_t k, uint64_t seed,
                      int32_t* s, double* y, int64_t* arrivals_out) {
  if (k < 1 || n < 0) return GMO_EINVAL;
  for (int32_t j = 0; j < k; ++j) {
    s[j] = INT32_MAX;
    y[j] = INFINITY;
  }
  int64_t arrivals = 0;
  int32_t unfilled = k, jstar = 0;
  int prune = 0;
  double ystar = INFINITY;
  int rc = GMO_OK;
  for (int64_t e = 0; e < n && rc == GMO_OK; ++e) {
    if (check_weight(w[e]) || ids[e] < 0) return GMO_EINVAL;
    if (!(w[e] > 0.0)) continue;
    gmo_stream st;
    rc = stream_init(&st, ids[e], w[e], k, seed);
    if (rc) break;
    for (int32_t z = 0; z < k; ++z) {
      double b;
      int32_t c;
      rc = stream_next(&st, &b, &c);
      if (rc) break;
      ++arrivals;
      if (prune && b > ystar) break;
      if (!isfinite(b)) continue;
      int was_empty = (y[c] == INFINITY);
      if (better(b, st.id, y[c], s[c])) {
        y[c] = b;
        s[c] = st.id;
        if (!prune && was_empty && --unfilled == 0) {
          prune = 1;
          ystar = max_register(y, k, &jstar);
        } else if (prune && c == jstar) {
          ystar = max_register(y, k, &jstar);
        }
      }
    }
    stream_free(&st);
  }
  for (int32_t j = 0; j < k; ++j)
    if (s[j] == INT32_MAX) s[j] = -1;
  if (arrivals_out) *arrivals_out = arrivals;
  return rc;
}

/* ---------------------------------------------------------------------------
 * Estimators and the union (Sec. 1 and Sec. 2.3).
 * ------------------------------------------------------------------------- */

/* Probability-Jaccard estimate (1/k) sum_j 1(s_j(a) = s_j(b)); unfilled registers never match. */
int gmo_jaccard(const int32_t* sa, const int32_t* sb, int64_t n_pairs, int32_t k, double* out) {
  if (k < 1 || n_pairs < 0) return GMO_EINVAL;
  for (int64_t p = 0; p < n_pairs; ++p) {
    int64_t hits = 0;
    for (int32_t j = 0; j < k; ++j) {
      int32_t a = sa[p * k + j], b = sb[p * k + j];
      if (a >= 0 && a == b) ++hits;
    }
    out[p] = (double)hits / (double)k;
  }
  return GMO_OK;
}

/* Weighted-cardinality estimate (k - 1) / sum_j y_j (Lemiesz; Sec. 1, Eq. yjpi), left-to-right sum. */
int gmo_cardinality(const double* y, int32_t n_rows, int32_t k, double* out) {
  if (k < 2 || n_rows < 0) return GMO_EINVAL;
  for (int32_t r = 0; r < n_rows; ++r) {
    double sum = 0.0;
    for (int32_t j = 0; j < k; ++j) sum += y[(int64_t)r * k + j];
    out[r] = (double)(k - 1) / sum;
  }
  return GMO_OK;
}

/* Union of sketches (Sec. 2.3, Mergeability): register-wise min of (y, s). */
int gmo_merge(const int32_t* sa, const double* ya, const int32_t* sb, const double* yb, int64_t n_regs,
              int32_t* s_out, double* y_out) {
  for (int64_t j = 0; j < n_regs; ++j) {
    int32_t ia = sa[j] < 0 ? INT32_MAX : sa[j];
    int32_t ib = sb[j] < 0 ? INT32_MAX : sb[j];
    if (better(yb[j], ib, ya[j], ia)) {
      y_out[j] = yb[j];
      s_out[j] = sb[j];
    } else {
      y_out[j] = ya[j];
      s_out[j] = sa[j];
    }
  }
  return GMO_OK;
}
