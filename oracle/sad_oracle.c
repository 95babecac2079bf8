/*
 * CPU oracle for the Sample-Align-D decomposition step (k-mer count vectors,
 * k-mer rank, regular-sampling partition).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference the CUDA
 * library is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it; the product path
 * never does. It shares no code, header or table with the CUDA library.
 *
 * Every function follows the paper (Saeed & Khokhar, "Sample-Align-D", arXiv
 * 0905.1744) as cited beside it, in the paper's order and notation:
 *
 *   count      Sec. 3 "k-mer Rank": c^X = (c^X_1..c^X_eps), eps = c^k, the number
 *              of occurrences of every k-letter word in X.
 *   similarity Eq. 1: F(X,Y) = sum_i min(c^X_i, c^Y_i) / (min(n,m) - k + 1).
 *              (The printed subscript c^Y_j is read as c^Y_i.)
 *   rank       Eq. 3: R_i = (1/N) sum_{j=1..N} F(i,j): the mean of F over the
 *              whole set, j = i included. The paper averages the distance form
 *              of Eq. 2; the rank here is the mean of F itself, and the
 *              distance form is sad_oracle_rank_dist below.
 *              The key carried for each sequence is the 128-bit fixed-point sum
 *              key_i = sum_j floor(S_ij * 2^64 / D_ij), S_ij the Eq. 1 numerator
 *              and D_ij its denominator; the float view is
 *              rank_i = (hi + lo * 2^-64) / N.
 *   partition  Sec. 3.1.2 and Algorithm 2 steps 7-11: sort p blocks, take p-1
 *              regularly spaced samples per block, sort the p(p-1) samples,
 *              pick pivots Y_{p/2}, Y_{p+p/2}, ..., Y_{(p-2)p+p/2}, and send the
 *              keys in (y_{i-1}, y_i] to bucket i (Sec. 3.3.2).
 *
 * Status codes returned: 0 ok, 1 invalid argument, 6 bad input data.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_INVALID = 1, OR_BAD_INPUT = 6 };

static int64_t ipow(int64_t a, int32_t k) {
  int64_t r = 1;
  for (int32_t i = 0; i < k; ++i) r *= a;
  return r;
}

/* ---------------------------------------------------------------- count --- */

/* Sec. 3 "k-mer Rank": counts[x * eps + tau] = occurrences of word tau in
 * sequence x. Word index tau = sum_r a_{i+r} * c^(k-1-r) (first letter most
 * significant). A letter code >= alphabet or a sequence shorter than k is bad
 * input. */
int sad_oracle_kmer_count(const uint8_t *codes, const int64_t *offsets, int32_t n,
                          int32_t k, int32_t alphabet, int32_t *counts) {
  if (n < 0 || k < 1 || alphabet < 1) return OR_INVALID;
  int64_t eps = ipow(alphabet, k);
  memset(counts, 0, sizeof(int32_t) * (size_t)eps * (size_t)n);
  for (int32_t x = 0; x < n; ++x) {
    int64_t start = offsets[x], len = offsets[x + 1] - offsets[x];
    if (len < k) return OR_BAD_INPUT;
    for (int64_t i = 0; i + k <= len; ++i) {
      int64_t tau = 0;
      for (int32_t r = 0; r < k; ++r) {
        uint8_t a = codes[start + i + r];
        if (a >= alphabet) return OR_BAD_INPUT;
        tau = tau * alphabet + a;
      }
      counts[(int64_t)x * eps + tau] += 1;
    }
  }
  return OR_OK;
}

/* ----------------------------------------------------------- similarity --- */

/* Eq. 1 numerator: S(X,Y) = sum over all eps words of min(c^X_i, c^Y_i). */
int64_t sad_oracle_shared_count(const int32_t *cx, const int32_t *cy, int64_t eps) {
  int64_t s = 0;
  for (int64_t i = 0; i < eps; ++i) s += cx[i] < cy[i] ? cx[i] : cy[i];
  return s;
}

/* floor(S * 2^64 / D) as (hi, lo): one pair's F(X,Y) = S/D in 64.64 fixed point. */
void sad_oracle_term(uint64_t s, uint64_t d, uint64_t *hi, uint64_t *lo) {
  u128 t = ((u128)s << 64) / (u128)d;
  *hi = (uint64_t)(t >> 64);
  *lo = (uint64_t)t;
}

typedef struct {
  const int32_t *counts;
  const int64_t *m;      /* number of k-mers per sequence, L - k + 1 */
  int32_t n;
  int64_t eps;
  const int32_t *rows;   /* rows to evaluate */
  int32_t n_rows;
  const int32_t *ref;    /* reference sequences of the rank (NULL: all n) */
  int32_t n_ref;
  uint64_t *key_hi, *key_lo;
  double *rank;
  double *rank_fp64;
  int32_t next;          /* shared row cursor */
  pthread_mutex_t lock;
} rank_job;

/* Eq. 3 for one sequence i: key_i = sum_{j=1..N} floor(S_ij 2^64 / D_ij),
 * D_ij = min(n_i, n_j) - k + 1 (Eq. 1 denominator), j = i included. With a
 * reference list the sum runs over its entries instead (the globalised rank of
 * Sec. 3.1.1: the k x p samples, Algorithm 2 step 6). Also the independent FP64
 * mean of S_ij / D_ij with Neumaier compensation. */
static void rank_row(const rank_job *J, int32_t out, int32_t i) {
  const int32_t *ci = J->counts + (int64_t)i * J->eps;
  u128 key = 0;
  double sum = 0.0, comp = 0.0;
  for (int32_t r = 0; r < J->n_ref; ++r) {
    const int32_t j = J->ref ? J->ref[r] : r;
    const int32_t *cj = J->counts + (int64_t)j * J->eps;
    int64_t s = sad_oracle_shared_count(ci, cj, J->eps);
    int64_t d = J->m[i] < J->m[j] ? J->m[i] : J->m[j];
    key += ((u128)s << 64) / (u128)d;
    double f = (double)s / (double)d;
    double t = sum + f;
    if (fabs(sum) >= fabs(f)) comp += (sum - t) + f; else comp += (f - t) + sum;
    sum = t;
  }
  uint64_t hi = (uint64_t)(key >> 64), lo = (uint64_t)key;
  J->key_hi[out] = hi;
  J->key_lo[out] = lo;
  /* rank_i = (hi + lo * 2^-64) / N, each operation rounded to nearest. */
  volatile double whole = (double)hi;
  volatile double frac = ldexp((double)lo, -64);
  volatile double total = whole + frac;
  J->rank[out] = total / (double)J->n_ref;
  if (J->rank_fp64) J->rank_fp64[out] = (sum + comp) / (double)J->n_ref;
}

static void *rank_worker(void *arg) {
  rank_job *J = (rank_job *)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int32_t r = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (r >= J->n_rows) break;
    rank_row(J, r, J->rows ? J->rows[r] : r);
  }
  return NULL;
}

/* Keys and rank views for rows[0..n_rows) (all rows when rows == NULL; then
 * n_rows must be n). lengths are the sequence lengths L (residues). */
int sad_oracle_kmer_rank(const int32_t *counts, const int64_t *lengths, int32_t n,
                         int32_t k, int32_t alphabet, const int32_t *rows,
                         int32_t n_rows, uint64_t *key_hi, uint64_t *key_lo,
                         double *rank, double *rank_fp64, int32_t threads) {
  if (n < 0 || k < 1 || alphabet < 1 || n_rows < 0) return OR_INVALID;
  if (!rows && n_rows != n) return OR_INVALID;
  int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t x = 0; x < n; ++x) {
    m[x] = lengths[x] - k + 1;
    if (m[x] < 1) { free(m); return OR_BAD_INPUT; }
  }
  for (int32_t r = 0; rows && r < n_rows; ++r)
    if (rows[r] < 0 || rows[r] >= n) { free(m); return OR_INVALID; }
  rank_job J = {counts, m, n, ipow(alphabet, k), rows, n_rows, NULL, n,
                key_hi, key_lo, rank, rank_fp64, 0, PTHREAD_MUTEX_INITIALIZER};
  if (threads < 1) threads = 1;
  if (threads > 1024) threads = 1024;
  pthread_t tid[1024];
  for (int32_t t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, rank_worker, &J);
  for (int32_t t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(m);
  return OR_OK;
}

/* Globalised rank (Sec. 3.1.1, Algorithm 2 step 6): every sequence against the
 * reference multiset ref[0..n_ref) (input indices; an index listed twice counts
 * twice): key_i = sum_r floor(S_{i,ref_r} 2^64 / (min(n_i, n_ref_r) - k + 1)),
 * rank_i = key_i / (n_ref 2^64). */
int sad_oracle_rank_vs(const int32_t *counts, const int64_t *lengths, int32_t n, int32_t k,
                       int32_t alphabet, const int32_t *ref, int32_t n_ref, uint64_t *key_hi,
                       uint64_t *key_lo, double *rank, int32_t threads) {
  if (n < 0 || k < 1 || alphabet < 1 || n_ref < 1 || !ref) return OR_INVALID;
  for (int32_t r = 0; r < n_ref; ++r)
    if (ref[r] < 0 || ref[r] >= n) return OR_INVALID;
  int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t x = 0; x < n; ++x) {
    m[x] = lengths[x] - k + 1;
    if (m[x] < 1) { free(m); return OR_BAD_INPUT; }
  }
  rank_job J = {counts, m, n, ipow(alphabet, k), NULL, n, ref, n_ref,
                key_hi, key_lo, rank, NULL, 0, PTHREAD_MUTEX_INITIALIZER};
  if (threads < 1) threads = 1;
  if (threads > 1024) threads = 1024;
  pthread_t tid[1024];
  for (int32_t t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, rank_worker, &J);
  for (int32_t t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(m);
  return OR_OK;
}

/* ------------------------------------------------ distance-form rank ------ */

/* floor(ln 2 * 2^64), from the decimal expansion ln 2 = 0.693147180559945309417... */
#define OR_LN2_Q64 0xB17217F7D1CF79ABull

/* ln(x) * 2^32 for an integer x >= 1, as a deterministic fixed-point value: the
 * binary logarithm by repeated squaring (x = 2^e m, m in [1, 2); squaring m gives
 * the next fraction bit of log2 m, halving it when it reaches 2), 40 fraction
 * bits with a 64-bit mantissa, then times ln 2. */
int64_t sad_oracle_ln_q(uint64_t x) {
  if (x == 0) return 0;
  int e = 63;
  while (!((x >> e) & 1u)) --e;
  uint64_t y = x << (63 - e);            /* m = y / 2^63 */
  uint64_t f = 0;
  for (int i = 1; i <= 40; ++i) {
    u128 t = ((u128)y * (u128)y) >> 63;  /* m^2 in [1, 4) */
    if (t >> 64) {
      t >>= 1;
      f |= (uint64_t)1 << (40 - i);
    }
    y = (uint64_t)t;
  }
  const u128 l2 = ((u128)(uint64_t)e << 40) | f;  /* log2 x, 40 fraction bits */
  return (int64_t)((l2 * (u128)OR_LN2_Q64) >> 72);
}

/* Eq. 2 and Eq. 3 literally: R_i = (1/N) sum_j d(i, j), d = -ln(Delta + F(i, j)),
 * with Delta = 1 / delta_den. With F = S / D, Delta + F = (D + b S) / (b D), so
 * the per-pair value is q_ij = ln_q(b D) - ln_q(D + b S) (ln times 2^32) and
 * key_i = sum_j q_ij (j = i included), rank_i = key_i 2^-32 / N (each step rounded
 * to nearest). rank_fp64: the FP64 mean of -log(1/b + S/D) with Neumaier
 * compensation, as an independent check. */
typedef struct {
  const int32_t *counts;
  const int64_t *m;
  int32_t n;
  int64_t eps;
  int64_t b;
  const int32_t *ref;    /* reference multiset (NULL: all n) */
  int32_t n_ref;
  int64_t *key;
  double *rank, *rank_fp64;
  int32_t next;
  pthread_mutex_t lock;
} dist_job;

static void *dist_worker(void *arg) {
  dist_job *J = (dist_job *)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int32_t i = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (i >= J->n) break;
    const int32_t *ci = J->counts + (int64_t)i * J->eps;
    int64_t key = 0;
    double sum = 0.0, comp = 0.0;
    for (int32_t r = 0; r < J->n_ref; ++r) {
      const int32_t j = J->ref ? J->ref[r] : r;
      const int64_t s = sad_oracle_shared_count(ci, J->counts + (int64_t)j * J->eps, J->eps);
      const int64_t d = J->m[i] < J->m[j] ? J->m[i] : J->m[j];
      key += sad_oracle_ln_q((uint64_t)(J->b * d)) - sad_oracle_ln_q((uint64_t)(d + J->b * s));
      const double f = -log(1.0 / (double)J->b + (double)s / (double)d);
      const double t = sum + f;
      if (fabs(sum) >= fabs(f)) comp += (sum - t) + f; else comp += (f - t) + sum;
      sum = t;
    }
    J->key[i] = key;
    volatile double k64 = (double)key;
    volatile double nats = k64 * ldexp(1.0, -32);
    J->rank[i] = nats / (double)J->n_ref;
    if (J->rank_fp64) J->rank_fp64[i] = (sum + comp) / (double)J->n_ref;
  }
  return NULL;
}

int sad_oracle_rank_dist(const int32_t *counts, const int64_t *lengths, int32_t n, int32_t k,
                         int32_t alphabet, int32_t delta_den, int64_t *key, double *rank,
                         double *rank_fp64, int32_t threads) {
  if (n < 0 || k < 1 || alphabet < 1 || delta_den < 1) return OR_INVALID;
  int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t x = 0; x < n; ++x) {
    m[x] = lengths[x] - k + 1;
    if (m[x] < 1) { free(m); return OR_BAD_INPUT; }
  }
  dist_job J = {counts, m, n, ipow(alphabet, k), delta_den, NULL, n, key, rank, rank_fp64, 0,
                PTHREAD_MUTEX_INITIALIZER};
  if (threads < 1) threads = 1;
  if (threads > 1024) threads = 1024;
  pthread_t tid[1024];
  for (int32_t t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, dist_worker, &J);
  for (int32_t t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(m);
  return OR_OK;
}

/* The distance form against a reference multiset ref[0..n_ref) (the globalised
 * rank of Sec. 3.1.1 on Eq. 2): key_i = sum_r q_{i, ref_r}, rank_i = key_i 2^-32 / n_ref. */
int sad_oracle_rank_vs_dist(const int32_t *counts, const int64_t *lengths, int32_t n, int32_t k,
                            int32_t alphabet, int32_t delta_den, const int32_t *ref,
                            int32_t n_ref, int64_t *key, double *rank, int32_t threads) {
  if (n < 0 || k < 1 || alphabet < 1 || delta_den < 1 || n_ref < 1 || !ref) return OR_INVALID;
  for (int32_t r = 0; r < n_ref; ++r)
    if (ref[r] < 0 || ref[r] >= n) return OR_INVALID;
  int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t x = 0; x < n; ++x) {
    m[x] = lengths[x] - k + 1;
    if (m[x] < 1) { free(m); return OR_BAD_INPUT; }
  }
  dist_job J = {counts, m, n, ipow(alphabet, k), delta_den, ref, n_ref, key, rank, NULL, 0,
                PTHREAD_MUTEX_INITIALIZER};
  if (threads < 1) threads = 1;
  if (threads > 1024) threads = 1024;
  pthread_t tid[1024];
  for (int32_t t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, dist_worker, &J);
  for (int32_t t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(m);
  return OR_OK;
}

/* ------------------------------------------------------------ partition --- */

typedef struct { uint64_t hi, lo; int32_t idx; } item;

/* Order of the rank keys: by value, ties by input index (so all items differ). */
static int item_less(const item *a, const item *b) {
  if (a->hi != b->hi) return a->hi < b->hi;
  if (a->lo != b->lo) return a->lo < b->lo;
  return a->idx < b->idx;
}

static int item_cmp(const void *pa, const void *pb) {
  const item *a = (const item *)pa, *b = (const item *)pb;
  if (item_less(a, b)) return -1;
  if (item_less(b, a)) return 1;
  return 0;
}

/* Sec. 3.1.2 / Algorithm 2 steps 7-11 on one device, p virtual processors.
 *   step 1/7: processor b holds the contiguous block [floor(bN/p), floor((b+1)N/p))
 *             and sorts it by rank;
 *   step 8:   it picks p-1 evenly spaced samples, positions floor(j w_b / p),
 *             j = 1..p-1 (0-based within the sorted block of size w_b);
 *   step 9:   the p(p-1) samples Y are sorted and y_i = Y_{(i-1)p + floor(p/2)}
 *             (1-based), i = 1..p-1, are the pivots;
 *   step 11:  bucket i (1-based) receives the keys in (y_{i-1}, y_i] (Sec. 3.3.2),
 *             i.e. the 0-based bucket of x is the number of pivots below x; each
 *             block sends its sub-blocks, and a bucket lists its members in
 *             ascending (key, index) order.
 * Outputs: bucket_offsets[p+1] (CSR), members[n] (input indices),
 * pivot_idx[p-1] (input index of each pivot; may be NULL). Requires 1 <= p <= n
 * (so that no block is empty), or n == 0. */
int sad_oracle_partition(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n,
                         int32_t p, int32_t *bucket_offsets, int32_t *members,
                         int32_t *pivot_idx) {
  if (p < 1 || n < 0) return OR_INVALID;
  if (n == 0) {
    for (int32_t b = 0; b <= p; ++b) bucket_offsets[b] = 0;
    return OR_OK;
  }
  if (p > n) return OR_INVALID;
  item *blk = (item *)malloc(sizeof(item) * (size_t)n);
  for (int32_t x = 0; x < n; ++x) { blk[x].hi = key_hi[x]; blk[x].lo = key_lo[x]; blk[x].idx = x; }

  /* local sorts (steps 1, 7) */
  int64_t nsamp = (int64_t)p * (p - 1);
  item *Y = (item *)malloc(sizeof(item) * (size_t)(nsamp > 0 ? nsamp : 1));
  int64_t ny = 0;
  for (int32_t b = 0; b < p; ++b) {
    int64_t lo = (int64_t)b * n / p, hi = (int64_t)(b + 1) * n / p;
    int64_t w = hi - lo;
    qsort(blk + lo, (size_t)w, sizeof(item), item_cmp);
    /* regular samples (step 8) */
    for (int32_t j = 1; j < p; ++j) Y[ny++] = blk[lo + (int64_t)j * w / p];
  }
  /* sort the samples and choose pivots (step 9) */
  qsort(Y, (size_t)ny, sizeof(item), item_cmp);
  item *piv = (item *)malloc(sizeof(item) * (size_t)(p > 1 ? p - 1 : 1));
  for (int32_t i = 1; i < p; ++i) {
    int64_t one_based = (int64_t)(i - 1) * p + p / 2;
    piv[i - 1] = Y[one_based - 1];
    if (pivot_idx) pivot_idx[i - 1] = piv[i - 1].idx;
  }

  /* bucket of every item = number of pivots strictly below it (step 11) */
  int32_t *bucket = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t b = 0; b <= p; ++b) bucket_offsets[b] = 0;
  for (int32_t x = 0; x < n; ++x) {
    int32_t c = 0;
    for (int32_t i = 0; i < p - 1; ++i) c += item_less(&piv[i], &blk[x]);
    bucket[x] = c;
    bucket_offsets[c + 1] += 1;
  }
  for (int32_t b = 0; b < p; ++b) bucket_offsets[b + 1] += bucket_offsets[b];

  /* redistribution: block 0's sub-block first, then block 1's, ... */
  item *out = (item *)malloc(sizeof(item) * (size_t)n);
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
  for (int32_t b = 0; b < p; ++b) fill[b] = bucket_offsets[b];
  for (int32_t x = 0; x < n; ++x) out[fill[bucket[x]]++] = blk[x];
  /* each processor orders what it received */
  for (int32_t b = 0; b < p; ++b)
    qsort(out + bucket_offsets[b], (size_t)(bucket_offsets[b + 1] - bucket_offsets[b]),
          sizeof(item), item_cmp);
  for (int32_t x = 0; x < n; ++x) members[x] = out[x].idx;

  free(fill); free(out); free(bucket); free(piv); free(Y); free(blk);
  return OR_OK;
}

/* Library identity for the loader. */
/* Algorithm 2 steps 3-4: each of the p contiguous blocks b = [floor(bN/p),
 * floor((b+1)N/p)) of sequences (w_b of them) is sorted by its local key (ties by
 * input index), and ks evenly spaced samples are taken at the 0-based positions
 * floor(j w_b / (ks + 1)), j = 1..ks (the spacing of the regular sampling of
 * Sec. 3.1.2 with ks + 1 parts). Output: input indices, block-major. Every block
 * must hold a sequence (N >= p). */
int sad_oracle_local_samples(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n,
                             int32_t p, int32_t ks, int32_t *sample_idx) {
  if (p < 1 || ks < 1 || n < p) return OR_INVALID;
  item *it = (item *)malloc(sizeof(item) * (size_t)n);
  for (int32_t x = 0; x < n; ++x) {
    it[x].hi = key_hi[x];
    it[x].lo = key_lo[x];
    it[x].idx = x;
  }
  for (int32_t b = 0; b < p; ++b) {
    const int64_t lo = (int64_t)b * n / p, hi = (int64_t)(b + 1) * n / p, w = hi - lo;
    qsort(it + lo, (size_t)w, sizeof(item), item_cmp);
    for (int32_t j = 1; j <= ks; ++j)
      sample_idx[(int64_t)b * ks + (j - 1)] = it[lo + (int64_t)j * w / (ks + 1)].idx;
  }
  free(it);
  return OR_OK;
}

const char *sad_oracle_version(void) { return "sad-oracle-1"; }
