/* Drives every routine of the CPU oracle (oracle/gm_oracle.c) on small seeded
 * inputs, including empty rows, zero weights, repeated ids and extreme weights,
 * for a build with -fsanitize=address,undefined.  Exit 0 when every call
 * returns its documented status; the sanitizers abort on any memory or
 * undefined-behaviour error.  Test infrastructure only. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void gmo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double gmo_uniform_from_words(uint32_t w0, uint32_t w1);
int gmo_exact_sum(const double* t, int64_t n, double* out);
int gmo_arrivals(int32_t id, double v, int32_t k, uint64_t seed, int32_t n_steps, double* b_out, int32_t* c_out);
int gmo_sketch_rows(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int32_t k,
                    uint64_t seed, int32_t* s_out, double* y_out, double* y2_out, int32_t* s2_out);
int gmo_fastsearch_budgets(const double* v, int64_t n, int64_t R, int64_t* out);
int gmo_fastgm_alg1(const int32_t* ids, const double* w, int64_t n, int32_t k, uint64_t seed, int32_t delta,
                    int32_t* s, double* y, int64_t* arrivals_out, int64_t* search_R_out,
                    int64_t* search_arrivals_out);
int gmo_stream_fastgm(const int32_t* ids, const double* w, int64_t n, int32_t k, uint64_t seed, int32_t* s,
                      double* y, int64_t* arrivals_out);
int gmo_jaccard(const int32_t* sa, const int32_t* sb, int64_t n_pairs, int32_t k, double* out);
int gmo_cardinality(const double* y, int32_t n_rows, int32_t k, double* out);
int gmo_merge(const int32_t* sa, const double* ya, const int32_t* sb, const double* yb, int64_t n_regs,
              int32_t* s_out, double* y_out);

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64(void) { /* splitmix64 */
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double unit(void) { return ((double)(next_u64() >> 11) + 0.5) * 0x1p-53; }

#define CHECK(x)                                                     \
  do {                                                               \
    if ((x) != 0) {                                                  \
      fprintf(stderr, "%s:%d: %s failed\n", __FILE__, __LINE__, #x); \
      return 1;                                                      \
    }                                                                \
  } while (0)

int main(void) {
  uint32_t ctr[4] = {1, 2, 3, 4}, key[2] = {5, 6}, out[4];
  gmo_philox4x32_10(ctr, key, out);
  if (!(gmo_uniform_from_words(0u, 0u) > 0.0) || !(gmo_uniform_from_words(~0u, ~0u) < 1.0)) return 1;
  const int ks[3] = {1, 7, 64};
  for (int ki = 0; ki < 3; ++ki) {
    const int32_t k = ks[ki];
    /* rows: empty, one element, zeros only, a repeated id, extreme weights, random */
    const int32_t n_rows = 6;
    int64_t row_ptr[7] = {0, 0, 1, 3, 5, 8, 48};
    int32_t ids[48];
    double w[48];
    for (int i = 0; i < 48; ++i) {
      ids[i] = (int32_t)(next_u64() % (1u << 24));
      w[i] = -log(unit());
    }
    w[1] = 0.0;
    w[2] = 0.0;
    ids[4] = ids[3];
    w[5] = 5e-324;
    w[6] = 1e300;
    w[7] = 1.0;
    int32_t s[6 * 64], s2[6 * 64];
    double y[6 * 64], y2[6 * 64], ym[6 * 64], card[6], jac[6];
    CHECK(gmo_sketch_rows(row_ptr, ids, w, n_rows, k, 11, s, y, y2, s2));
    CHECK(gmo_sketch_rows(row_ptr, ids, w, n_rows, k, 12, s2, ym, NULL, NULL));
    CHECK(gmo_jaccard(s, s2, n_rows, k, jac));
    if (k >= 2) CHECK(gmo_cardinality(y, n_rows, k, card));
    CHECK(gmo_merge(s, y, s2, ym, (int64_t)n_rows * k, s2, ym));
    int64_t arr = 0, sR = 0, sA = 0;
    int32_t sa[64];
    double ya[64];
    CHECK(gmo_fastgm_alg1(ids + 8, w + 8, 40, k, 3, k, sa, ya, &arr, &sR, &sA));
    CHECK(gmo_fastgm_alg1(ids, w, 0, k, 3, k, sa, ya, &arr, NULL, NULL));
    int32_t rep_ids[80];
    double rep_w[80];
    for (int i = 0; i < 80; ++i) {
      rep_ids[i] = ids[8 + i % 40];
      rep_w[i] = w[8 + i % 40];
    }
    CHECK(gmo_stream_fastgm(rep_ids, rep_w, 80, k, 3, sa, ya, &arr));
    double b[64];
    int32_t c[64];
    CHECK(gmo_arrivals(ids[10], w[10], k, 9, k, b, c));
    int64_t budgets[40];
    CHECK(gmo_fastsearch_budgets(w + 8, 40, 10 * k, budgets));
    double tot;
    CHECK(gmo_exact_sum(w + 8, 40, &tot));
  }
  return 0;
}
