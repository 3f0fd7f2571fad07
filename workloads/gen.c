/*
 * Seeded synthetic sparse workloads for the load-balanced SpMV path.
 *
 * This module only draws random numbers and lays out CSR arrays (row lengths,
 * sorted distinct column indices, values, dense vectors).  It holds none of the
 * method's arithmetic: no products, no sums, no partitioning, no transposes.
 * Both the CUDA path and the CPU oracle consume what it produces.
 *
 * Random numbers: splitmix64 (seeding) feeding xoshiro256** (Blackman & Vigna,
 * "Scrambled linear pseudorandom number generators", 2021).  Every logical
 * stream (one per row, per vector block, per R-MAT edge block) is seeded from
 * (seed, tag, stream index), so output never depends on the thread count.
 *
 * Values: U(-1,1) = (m - 2^23) / 2^23 with m a 24-bit draw (exact in FP32);
 * U(0,1) = m / 2^24; N(0,1) by Box-Muller in double, rounded to float.
 * Zipf(s=2) on {1..200000} by inverse CDF over a precomputed table.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PRNG -- */

typedef struct { uint64_t s[4]; } wl_rng;

static inline uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(wl_rng* r) {
  uint64_t* s = r->s;
  const uint64_t out = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

static void rng_init(wl_rng* r, uint64_t seed, uint64_t tag, uint64_t stream) {
  uint64_t x = seed;
  uint64_t a = splitmix64(&x);
  x = a ^ (tag * 0xD1B54A32D192ED03ULL);
  uint64_t b = splitmix64(&x);
  x = b ^ (stream * 0x9E3779B97F4A7C15ULL) ^ 0x632BE59BD9B4E019ULL;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* uniform integer in [0, n), n >= 1 (Lemire's multiply-shift with rejection) */
static inline uint32_t rng_below(wl_rng* r, uint32_t n) {
  uint64_t m = (uint64_t)(uint32_t)(rng_next(r) >> 32) * (uint64_t)n;
  uint32_t l = (uint32_t)m;
  if (l < n) {
    uint32_t t = (uint32_t)(-n) % n;
    while (l < t) {
      m = (uint64_t)(uint32_t)(rng_next(r) >> 32) * (uint64_t)n;
      l = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

static inline double rng_u01(wl_rng* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

static inline float draw_value(wl_rng* r, int kind) {
  if (kind == 0) { /* U(-1,1) on the 2^-23 grid */
    int32_t m = (int32_t)(rng_next(r) >> 40);
    return (float)(m - 8388608) * 0x1.0p-23f;
  } else if (kind == 1) { /* U(0,1) on the 2^-24 grid */
    uint32_t m = (uint32_t)(rng_next(r) >> 40);
    return (float)m * 0x1.0p-24f;
  } else { /* N(0,1), Box-Muller */
    double u1 = ((double)(rng_next(r) >> 11) + 1.0) * 0x1.0p-53; /* (0,1] */
    double u2 = rng_u01(r);
    return (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

/* --------------------------------------------------------------- threads -- */

typedef void (*wl_range_fn)(void* ctx, int64_t begin, int64_t end);
typedef struct { wl_range_fn fn; void* ctx; int64_t b, e; } wl_job;

static void* wl_job_main(void* p) {
  wl_job* j = (wl_job*)p;
  j->fn(j->ctx, j->b, j->e);
  return NULL;
}

/* Runs fn over [0, n) split at the given boundaries (bounds[0]=0 .. bounds[t]=n). */
static void wl_parallel_bounds(wl_range_fn fn, void* ctx, const int64_t* bounds, int nt) {
  if (nt <= 1) {
    fn(ctx, bounds[0], bounds[1]);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  wl_job* jobs = (wl_job*)malloc(sizeof(wl_job) * nt);
  for (int t = 0; t < nt; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].b = bounds[t]; jobs[t].e = bounds[t + 1];
    pthread_create(&th[t], NULL, wl_job_main, &jobs[t]);
  }
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

static void wl_parallel(wl_range_fn fn, void* ctx, int64_t n, int nt) {
  if (nt < 1) nt = 1;
  if (n < 4096) nt = 1;
  int64_t bounds[257];
  if (nt > 256) nt = 256;
  for (int t = 0; t <= nt; ++t) bounds[t] = n * t / nt;
  wl_parallel_bounds(fn, ctx, bounds, nt);
}

/* Row ranges balanced by nnz (rp is a CSR offset array). */
static void wl_parallel_rows(wl_range_fn fn, void* ctx, int64_t R, const int32_t* rp, int nt) {
  if (nt < 1) nt = 1;
  if (nt > 256) nt = 256;
  int64_t total = (int64_t)rp[R] + R;
  if (total < 65536) nt = 1;
  int64_t bounds[257];
  bounds[0] = 0;
  int64_t r = 0;
  for (int t = 1; t < nt; ++t) {
    int64_t target = total * t / nt;
    while (r < R && (int64_t)rp[r] + r < target) ++r;
    bounds[t] = r;
  }
  bounds[nt] = R;
  wl_parallel_bounds(fn, ctx, bounds, nt);
}

/* ------------------------------------------------------------- sampling -- */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void sort_i32(int32_t* a, int64_t n) {
  if (n <= 32) {
    for (int64_t i = 1; i < n; ++i) {
      int32_t v = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
      a[j + 1] = v;
    }
  } else {
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
  }
}

typedef struct {
  int32_t* keys; /* open-addressing set, capacity cap (power of two), -1 = empty */
  int64_t cap;
} wl_set;

static void set_reserve(wl_set* s, int64_t n) {
  int64_t need = 16;
  while (need < 2 * n) need <<= 1;
  if (need > s->cap) {
    free(s->keys);
    s->keys = (int32_t*)malloc(sizeof(int32_t) * need);
    for (int64_t i = 0; i < need; ++i) s->keys[i] = -1;
    s->cap = need;
  }
}

/* returns 1 if inserted, 0 if already present */
static inline int set_insert(wl_set* s, int32_t k) {
  uint64_t mask = (uint64_t)s->cap - 1;
  uint64_t h = ((uint64_t)(uint32_t)k * 0x9E3779B97F4A7C15ULL) >> 17;
  for (;;) {
    uint64_t i = h & mask;
    if (s->keys[i] == -1) { s->keys[i] = k; return 1; }
    if (s->keys[i] == k) return 0;
    ++h;
  }
}

static inline void set_erase_all(wl_set* s, const int32_t* ks, int64_t n) {
  uint64_t mask = (uint64_t)s->cap - 1;
  for (int64_t q = 0; q < n; ++q) {
    uint64_t h = ((uint64_t)(uint32_t)ks[q] * 0x9E3779B97F4A7C15ULL) >> 17;
    for (;;) {
      uint64_t i = h & mask;
      if (s->keys[i] == ks[q]) { s->keys[i] = -1; break; }
      ++h;
    }
  }
}

/*
 * L distinct columns from [0, C), sorted ascending, uniformly over L-subsets.
 * 4L >= C: selection sampling (Knuth TAOCP vol. 2, Algorithm S), sorted by
 * construction.  Otherwise Floyd's algorithm (Bentley & Floyd, CACM 1987)
 * followed by a sort.
 */
static void sample_sorted_distinct(wl_rng* r, int32_t C, int32_t L, int32_t* out, wl_set* set) {
  if (L <= 0) return;
  if ((int64_t)L * 4 >= (int64_t)C) {
    int32_t need = L, got = 0;
    for (int32_t t = 0; t < C && got < L; ++t) {
      if (rng_below(r, (uint32_t)(C - t)) < (uint32_t)need) {
        out[got++] = t;
        --need;
      }
    }
    return;
  }
  if (L <= 24) {
    for (int32_t q = 0; q < L; ++q) {
      int32_t j = C - L + q;
      int32_t t = (int32_t)rng_below(r, (uint32_t)j + 1u);
      int dup = 0;
      for (int32_t p = 0; p < q; ++p)
        if (out[p] == t) { dup = 1; break; }
      out[q] = dup ? j : t;
    }
  } else {
    set_reserve(set, L);
    for (int32_t q = 0; q < L; ++q) {
      int32_t j = C - L + q;
      int32_t t = (int32_t)rng_below(r, (uint32_t)j + 1u);
      if (set_insert(set, t)) {
        out[q] = t;
      } else {
        set_insert(set, j);
        out[q] = j;
      }
    }
    set_erase_all(set, out, L);
  }
  sort_i32(out, L);
}

/* ------------------------------------------------------------------ Zipf -- */

#define WL_ZIPF_KMAX 200000
static double* g_zipf_cdf = NULL;
static pthread_once_t g_zipf_once = PTHREAD_ONCE_INIT;

static void zipf_build(void) {
  g_zipf_cdf = (double*)malloc(sizeof(double) * WL_ZIPF_KMAX);
  double acc = 0.0;
  for (int64_t k = 1; k <= WL_ZIPF_KMAX; ++k) {
    acc += 1.0 / ((double)k * (double)k);
    g_zipf_cdf[k - 1] = acc;
  }
}

/* K ~ Zipf(2) on {1..200000}, P(K=k) proportional to k^-2 */
static int32_t zipf2_draw(wl_rng* r) {
  pthread_once(&g_zipf_once, zipf_build);
  double u = rng_u01(r) * g_zipf_cdf[WL_ZIPF_KMAX - 1];
  int32_t lo = 0, hi = WL_ZIPF_KMAX - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (g_zipf_cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo + 1;
}

/* ----------------------------------------------------------- public API -- */

enum { TAG_ROWLEN = 1, TAG_EMPTY = 2, TAG_PLANT = 3, TAG_COLS = 4, TAG_VALS = 5, TAG_VEC = 6,
       TAG_RMAT = 7, TAG_BATCH = 8 };

/* Dense vector of n values of the given kind (0 U(-1,1), 1 U(0,1), 2 N(0,1)). */
typedef struct { int64_t n; int kind; uint64_t seed, tag; float* out; } vec_ctx;
static void vec_range(void* p, int64_t b, int64_t e) {
  vec_ctx* c = (vec_ctx*)p;
  const int64_t BLK = 4096;
  for (int64_t blk = b; blk < e; ++blk) {
    wl_rng r;
    rng_init(&r, c->seed, TAG_VEC * 1000003ULL + c->tag, (uint64_t)blk);
    int64_t i0 = blk * BLK, i1 = i0 + BLK < c->n ? i0 + BLK : c->n;
    for (int64_t i = i0; i < i1; ++i) c->out[i] = draw_value(&r, c->kind);
  }
}
void wl_fill_vector(int64_t n, int kind, uint64_t seed, uint64_t tag, float* out, int nthreads) {
  vec_ctx c = {n, kind, seed, tag, out};
  int64_t blocks = (n + 4095) / 4096;
  wl_parallel(vec_range, &c, blocks, blocks >= 64 ? nthreads : 1);
}

/* Fill columns (sorted, distinct per row) and values for a CSR pattern given rp. */
typedef struct {
  int32_t C; const int32_t* rp; uint64_t seed, tag; int val_kind; int32_t* ci; float* v;
} fill_ctx;
static void fill_range(void* p, int64_t b, int64_t e) {
  fill_ctx* c = (fill_ctx*)p;
  wl_set set = {NULL, 0};
  for (int64_t row = b; row < e; ++row) {
    int32_t L = c->rp[row + 1] - c->rp[row];
    if (L <= 0) continue;
    wl_rng r;
    if (c->ci) {
      rng_init(&r, c->seed, TAG_COLS * 1000003ULL + c->tag, (uint64_t)row);
      sample_sorted_distinct(&r, c->C, L, c->ci + c->rp[row], &set);
    }
    if (c->v) {
      rng_init(&r, c->seed, TAG_VALS * 1000003ULL + c->tag, (uint64_t)row);
      float* vv = c->v + c->rp[row];
      for (int32_t q = 0; q < L; ++q) vv[q] = draw_value(&r, c->val_kind);
    }
  }
  free(set.keys);
}
/* ci may be NULL (keep existing columns); v may be NULL. */
void wl_fill_csr(int32_t R, int32_t C, const int32_t* rp, uint64_t seed, uint64_t tag, int val_kind,
                 int32_t* ci, float* v, int nthreads) {
  fill_ctx c = {C, rp, seed, tag, val_kind, ci, v};
  wl_parallel_rows(fill_range, &c, R, rp, nthreads);
}

/*
 * Power-law row lengths: K_r ~ Zipf(2), row r empty with probability empty_frac,
 * L_r = min(floor(c K_r), lmax, C).  c is found by bisection so that sum L_r is
 * the closest achievable value to target_nnz.  If plant_long is set and fewer
 * than 3 rows exceed 100000, three seeded rows are set to 150000.
 * Returns the total nnz; writes c to *c_out.
 */
int64_t wl_powerlaw_lengths(int32_t R, int32_t C, int64_t target_nnz, int32_t lmax, double empty_frac,
                            int plant_long, uint64_t seed, int32_t* L, double* c_out) {
  int32_t cap = lmax < C ? lmax : C;
  int32_t* K = (int32_t*)malloc(sizeof(int32_t) * (size_t)(R > 0 ? R : 1));
  for (int32_t r = 0; r < R; ++r) {
    wl_rng g;
    rng_init(&g, seed, TAG_ROWLEN, (uint64_t)r);
    int32_t k = zipf2_draw(&g);
    double u = rng_u01(&g);
    K[r] = (u < empty_frac) ? 0 : k;
  }
  double lo = 0.0, hi = 1.0;
  for (;;) {
    int64_t n = 0;
    for (int32_t r = 0; r < R; ++r) {
      double f = floor(hi * (double)K[r]);
      n += f > cap ? cap : (int64_t)f;
    }
    if (n >= target_nnz || hi > 1e12) break;
    hi *= 2.0;
  }
  int64_t n_lo = 0, n_hi = 0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    int64_t n = 0;
    for (int32_t r = 0; r < R; ++r) {
      double f = floor(mid * (double)K[r]);
      n += f > cap ? cap : (int64_t)f;
    }
    if (n >= target_nnz) hi = mid; else lo = mid;
  }
  for (int32_t r = 0; r < R; ++r) {
    double fl = floor(lo * (double)K[r]), fh = floor(hi * (double)K[r]);
    n_lo += fl > cap ? cap : (int64_t)fl;
    n_hi += fh > cap ? cap : (int64_t)fh;
  }
  double c = (target_nnz - n_lo <= n_hi - target_nnz) ? lo : hi;
  int64_t total = 0;
  int32_t n_long = 0;
  for (int32_t r = 0; r < R; ++r) {
    double f = floor(c * (double)K[r]);
    L[r] = f > cap ? cap : (int32_t)f;
    total += L[r];
    if (L[r] > 100000) ++n_long;
  }
  if (plant_long && n_long < 3 && cap >= 150000 && R >= 3) {
    wl_rng g;
    rng_init(&g, seed, TAG_PLANT, 0);
    int planted = 0;
    while (planted < 3 - n_long) {
      int32_t r = (int32_t)rng_below(&g, (uint32_t)R);
      if (L[r] > 100000) continue;
      total += 150000 - L[r];
      L[r] = 150000;
      ++planted;
    }
  }
  if (c_out) *c_out = c;
  free(K);
  return total;
}

/*
 * Row lengths spread by Zipf(2) weights and apportioned to exactly nnz_target
 * (largest remainder, ties to the lower row), then clipped to C.
 * Returns the total after clipping.
 */
typedef struct { int64_t rem; int32_t row; } rem_pair;
static int cmp_rem(const void* a, const void* b) {
  const rem_pair* x = (const rem_pair*)a;
  const rem_pair* y = (const rem_pair*)b;
  if (x->rem != y->rem) return x->rem > y->rem ? -1 : 1;
  return (x->row > y->row) - (x->row < y->row);
}
int64_t wl_apportioned_lengths(int32_t R, int32_t C, int64_t nnz_target, uint64_t seed, uint64_t tag,
                               int32_t* L) {
  if (R <= 0) return 0;
  int64_t* K = (int64_t*)malloc(sizeof(int64_t) * R);
  int64_t S = 0;
  for (int32_t r = 0; r < R; ++r) {
    wl_rng g;
    rng_init(&g, seed, TAG_ROWLEN * 1000003ULL + tag, (uint64_t)r);
    K[r] = zipf2_draw(&g);
    S += K[r];
  }
  rem_pair* rp = (rem_pair*)malloc(sizeof(rem_pair) * R);
  int64_t assigned = 0;
  for (int32_t r = 0; r < R; ++r) {
    /* nnz_target * K[r] < 2^63 for nnz_target < 2^45 */
    int64_t num = nnz_target * K[r];
    L[r] = (int32_t)(num / S);
    rp[r].rem = num % S;
    rp[r].row = r;
    assigned += L[r];
  }
  int64_t left = nnz_target - assigned;
  qsort(rp, (size_t)R, sizeof(rem_pair), cmp_rem);
  for (int64_t q = 0; q < left && q < R; ++q) L[rp[q].row] += 1;
  int64_t total = 0;
  for (int32_t r = 0; r < R; ++r) {
    if (L[r] > C) L[r] = C;
    total += L[r];
  }
  free(rp);
  free(K);
  return total;
}

/* Batch shapes: R_m log-uniform on [rmin, rmax], mean length log-uniform on [mmin, mmax]. */
void wl_batch_dims(int32_t num, double rmin, double rmax, double mmin, double mmax, uint64_t seed,
                   int32_t* R_out, int64_t* nnz_target_out) {
  for (int32_t m = 0; m < num; ++m) {
    wl_rng g;
    rng_init(&g, seed, TAG_BATCH, (uint64_t)m);
    double lr = log(rmin) + rng_u01(&g) * (log(rmax) - log(rmin));
    double lm = log(mmin) + rng_u01(&g) * (log(mmax) - log(mmin));
    int32_t R = (int32_t)llround(exp(lr));
    if (R < 1) R = 1;
    R_out[m] = R;
    nnz_target_out[m] = llround((double)R * exp(lm));
  }
}

/*
 * R-MAT edges (Chakrabarti, Zhan & Faloutsos, SDM 2004): for each of E edges and
 * each of `scale` levels, pick quadrant a/b/c/d.  Edges are bucketed by source,
 * each row's destinations sorted and de-duplicated.  rp has 2^scale + 1 entries,
 * ci room for E entries.  Returns the number of unique edges.
 */
typedef struct { int scale; int64_t E; double a, ab, abc; uint64_t seed; int32_t* src; int32_t* dst; } rmat_ctx;
static void rmat_range(void* p, int64_t b, int64_t e) {
  rmat_ctx* c = (rmat_ctx*)p;
  const int64_t BLK = 65536;
  for (int64_t blk = b; blk < e; ++blk) {
    wl_rng g;
    rng_init(&g, c->seed, TAG_RMAT, (uint64_t)blk);
    int64_t i0 = blk * BLK, i1 = i0 + BLK < c->E ? i0 + BLK : c->E;
    for (int64_t i = i0; i < i1; ++i) {
      uint32_t s = 0, d = 0;
      for (int l = 0; l < c->scale; ++l) {
        double u = rng_u01(&g);
        uint32_t sb = 0, db = 0;
        if (u < c->a) { sb = 0; db = 0; }
        else if (u < c->ab) { sb = 0; db = 1; }
        else if (u < c->abc) { sb = 1; db = 0; }
        else { sb = 1; db = 1; }
        s = (s << 1) | sb;
        d = (d << 1) | db;
      }
      c->src[i] = (int32_t)s;
      c->dst[i] = (int32_t)d;
    }
  }
}
typedef struct { const int32_t* rp_in; int32_t* buf; int32_t* len; } dedup_ctx;
static void dedup_range(void* p, int64_t b, int64_t e) {
  dedup_ctx* c = (dedup_ctx*)p;
  for (int64_t r = b; r < e; ++r) {
    int32_t* seg = c->buf + c->rp_in[r];
    int64_t n = c->rp_in[r + 1] - c->rp_in[r];
    sort_i32(seg, n);
    int64_t w = 0;
    for (int64_t q = 0; q < n; ++q)
      if (w == 0 || seg[w - 1] != seg[q]) seg[w++] = seg[q];
    c->len[r] = (int32_t)w;
  }
}
int64_t wl_rmat(int scale, int64_t E, double a, double b, double c, uint64_t seed, int32_t* rp, int32_t* ci,
                int nthreads) {
  int64_t R = (int64_t)1 << scale;
  int32_t* src = (int32_t*)malloc(sizeof(int32_t) * E);
  int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * E);
  rmat_ctx rc = {scale, E, a, a + b, a + b + c, seed, src, dst};
  int64_t blocks = (E + 65535) / 65536;
  wl_parallel(rmat_range, &rc, blocks, nthreads);
  int32_t* cnt = (int32_t*)calloc((size_t)R + 1, sizeof(int32_t));
  for (int64_t i = 0; i < E; ++i) cnt[src[i] + 1]++;
  for (int64_t r = 0; r < R; ++r) cnt[r + 1] += cnt[r];
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * R);
  memcpy(cur, cnt, sizeof(int32_t) * R);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * E);
  for (int64_t i = 0; i < E; ++i) buf[cur[src[i]]++] = dst[i];
  free(cur);
  free(src);
  free(dst);
  int32_t* len = (int32_t*)malloc(sizeof(int32_t) * R);
  dedup_ctx dc = {cnt, buf, len};
  wl_parallel_rows(dedup_range, &dc, R, cnt, nthreads);
  int64_t w = 0;
  rp[0] = 0;
  for (int64_t r = 0; r < R; ++r) {
    memcpy(ci + w, buf + cnt[r], sizeof(int32_t) * (size_t)len[r]);
    w += len[r];
    rp[r + 1] = (int32_t)w;
  }
  free(len);
  free(buf);
  free(cnt);
  return w;
}

/*
 * 27-point stencil on an n^3 grid, rows in lexicographic order (x fastest),
 * non-periodic.  Columns ascending; diagonal = diag_value, off-diagonals N(0,1)
 * drawn per row.  nnz = (3n-2)^3.
 */
typedef struct { int32_t n; float diag; uint64_t seed; int32_t* rp; int32_t* ci; float* v; } st_ctx;
static void st_rows_range(void* p, int64_t b, int64_t e) {
  st_ctx* c = (st_ctx*)p;
  const int32_t n = c->n;
  for (int64_t row = b; row < e; ++row) {
    int32_t x = (int32_t)(row % n), y = (int32_t)((row / n) % n), z = (int32_t)(row / ((int64_t)n * n));
    int32_t k = c->rp[row];
    wl_rng g;
    rng_init(&g, c->seed, TAG_VALS * 1000003ULL + 27, (uint64_t)row);
    for (int dz = -1; dz <= 1; ++dz) {
      if (z + dz < 0 || z + dz >= n) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        if (y + dy < 0 || y + dy >= n) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          if (x + dx < 0 || x + dx >= n) continue;
          c->ci[k] = (int32_t)((int64_t)(x + dx) + (int64_t)n * ((y + dy) + (int64_t)n * (z + dz)));
          c->v[k] = (dx == 0 && dy == 0 && dz == 0) ? c->diag : draw_value(&g, 2);
          ++k;
        }
      }
    }
  }
}
int64_t wl_stencil27(int32_t n, float diag_value, uint64_t seed, int32_t* rp, int32_t* ci, float* v,
                     int nthreads) {
  int64_t R = (int64_t)n * n * n;
  rp[0] = 0;
  for (int64_t row = 0; row < R; ++row) {
    int32_t x = (int32_t)(row % n), y = (int32_t)((row / n) % n), z = (int32_t)(row / ((int64_t)n * n));
    int32_t cx = (x > 0) + 1 + (x < n - 1), cy = (y > 0) + 1 + (y < n - 1), cz = (z > 0) + 1 + (z < n - 1);
    rp[row + 1] = rp[row] + cx * cy * cz;
  }
  st_ctx c = {n, diag_value, seed, rp, ci, v};
  wl_parallel_rows(st_rows_range, &c, R, rp, nthreads);
  return rp[R];
}
