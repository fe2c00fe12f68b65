/*
 * hgen: seeded synthetic hypergraph generator.
 *
 * Shared input for both the CPU oracle and the CUDA path.  It holds none of
 * the counting method's arithmetic: it only draws hyperedges.
 *
 * Determinism across machines (x86-64 and AArch64) is a design goal: the same
 * parameters must give the byte-identical CSR everywhere.  Therefore
 *   - all randomness is integer (splitmix64 streams),
 *   - vertex popularity is sampled from INTEGER weights held in a Fenwick tree
 *     (exact arithmetic, no drift when weights are withdrawn and restored),
 *   - the few transcendental values (Zipf and power-law weights, log-normal
 *     sizes, log-uniform graph sizes) come from det_log/det_exp below, which
 *     use only IEEE-754 +, -, *, / and exact power-of-two scaling, and the file
 *     must be compiled with -ffp-contract=off (no fused multiply-add).
 *
 * Model (Def. 2.1: a hyperedge is a non-empty vertex set; the paper assumes no
 * two hyperedges are equal, and its datasets were de-duplicated, Sec. 6.1):
 *   - hyperedge sizes k are drawn i.i.d. from one of
 *       uniform on [lo, hi],
 *       truncated power law P(k) ~ k^-gamma on [lo, hi],
 *       log-normal round(exp(mu + sigma z)) clipped to [lo, hi];
 *   - member vertices are drawn one by one without replacement, with
 *     probability proportional to a Zipf weight (rank+1)^-s among vertices
 *     still available;
 *   - optional degree cap: a vertex that reaches `degree_cap` hyperedges is
 *     withdrawn from all later draws;
 *   - optional de-duplication: a hyperedge equal to an earlier one is redrawn
 *     (same size), so |E| stays exact.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct hgen_params {
  int64_t num_vertices;
  int64_t num_edges;
  uint64_t seed;
  int32_t size_dist;      /* 0 uniform, 1 truncated power law, 2 log-normal */
  int32_t size_lo;
  int32_t size_hi;
  int32_t degree_cap;     /* 0 = no cap */
  double size_p1;         /* power-law exponent gamma, or log-normal mu */
  double size_p2;         /* log-normal sigma */
  double zipf_s;          /* vertex popularity exponent */
  int32_t dedup;          /* 1 = redraw duplicate hyperedges */
  int32_t reserved;
} hgen_params;

enum {
  HGEN_OK = 0,
  HGEN_ERR_ARG = -1,
  HGEN_ERR_NOMEM = -2,
  HGEN_ERR_EXHAUSTED = -3,   /* fewer available vertices than a hyperedge needs */
  HGEN_ERR_DEDUP = -4        /* could not find a fresh hyperedge after many redraws */
};

/* ---------------- integer random streams ---------------- */

typedef struct { uint64_t s; } rng_t;

static uint64_t splitmix64(rng_t* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static rng_t rng_stream(uint64_t seed, uint64_t tag) {
  rng_t r;
  r.s = seed * 0xD1342543DE82EF95ull + tag * 0x2545F4914F6CDD1Dull + 0x632BE59BD9B4E019ull;
  (void)splitmix64(&r);
  return r;
}

/* uniform integer in [0, n) by 128-bit multiply-high (n > 0) */
static uint64_t rng_below(rng_t* r, uint64_t n) {
  unsigned __int128 p = (unsigned __int128)splitmix64(r) * (unsigned __int128)n;
  return (uint64_t)(p >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unit(rng_t* r) {
  return (double)(splitmix64(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------- deterministic elementary functions ---------------- */

static const double LN2 = 0.6931471805599453;

static double det_log(double x) {
  /* x = m * 2^e, m in [sqrt(1/2), sqrt(2)); log m = 2 atanh((m-1)/(m+1)) */
  if (!(x > 0.0)) return -INFINITY;
  int e = 0;
  double m = frexp(x, &e);            /* exact: m in [0.5, 1) */
  if (m < 0.70710678118654752) { m *= 2.0; e -= 1; }
  double t = (m - 1.0) / (m + 1.0);
  double t2 = t * t;
  double term = t, sum = 0.0;
  for (int n = 1; n <= 41; n += 2) {   /* |t| <= 0.1716: 21 terms reach far below 1 ulp */
    sum += term / (double)n;
    term *= t2;
  }
  return 2.0 * sum + (double)e * LN2;
}

static double det_exp(double x) {
  /* x = k ln2 + r, |r| <= ln2/2; exp r by its Taylor series; scale by 2^k exactly */
  if (x > 700.0) return INFINITY;
  if (x < -700.0) return 0.0;
  double kd = floor(x / LN2 + 0.5);
  double r = x - kd * LN2;
  double term = 1.0, sum = 1.0;
  for (int n = 1; n <= 24; ++n) {
    term = term * r / (double)n;
    sum += term;
  }
  return ldexp(sum, (int)kd);
}

static double det_pow(double b, double s) { return det_exp(s * det_log(b)); }

/* ---------------- Fenwick tree of integer weights ---------------- */

typedef struct {
  int64_t n;
  uint64_t* t;     /* 1-based */
  int64_t top;     /* highest power of two <= n */
} fenwick;

static int fw_init(fenwick* f, const uint64_t* w, int64_t n) {
  f->n = n;
  f->t = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!f->t) return 0;
  for (int64_t i = 1; i <= n; ++i) {
    f->t[i] += w[i - 1];
    int64_t p = i + (i & -i);
    if (p <= n) f->t[p] += f->t[i];
  }
  f->top = 1;
  while (f->top * 2 <= n) f->top *= 2;
  return 1;
}

static void fw_add(fenwick* f, int64_t idx0, uint64_t delta /* two's complement for negative */) {
  for (int64_t i = idx0 + 1; i <= f->n; i += i & -i) f->t[i] += delta;
}

static uint64_t fw_total(const fenwick* f) {
  uint64_t s = 0;
  for (int64_t i = f->n; i > 0; i -= i & -i) s += f->t[i];
  return s;
}

/* smallest 0-based index whose inclusive prefix sum exceeds target (< total) */
static int64_t fw_find(const fenwick* f, uint64_t target) {
  int64_t pos = 0;
  for (int64_t step = f->top; step > 0; step >>= 1) {
    int64_t nx = pos + step;
    if (nx <= f->n && f->t[nx] <= target) {
      pos = nx;
      target -= f->t[nx];
    }
  }
  return pos;   /* 0-based index = pos */
}

/* ---------------- size distributions ---------------- */

static const double W_SCALE = 1099511627776.0;   /* 2^40 */

typedef struct {
  int32_t lo, hi, kind;
  uint64_t* cum;    /* cumulative integer weights, for the power law */
  uint64_t total;
  double mu, sigma;
} size_sampler;

static int sizes_init(size_sampler* s, const hgen_params* p) {
  memset(s, 0, sizeof(*s));
  s->lo = p->size_lo;
  s->hi = p->size_hi;
  s->kind = p->size_dist;
  if (s->lo < 1 || s->hi < s->lo) return 0;
  if (s->kind == 1) {
    int32_t n = s->hi - s->lo + 1;
    s->cum = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!s->cum) return 0;
    uint64_t acc = 0;
    for (int32_t i = 0; i < n; ++i) {
      double w = det_pow((double)(s->lo + i), -p->size_p1);
      uint64_t wi = (uint64_t)floor(w * W_SCALE + 0.5);
      if (wi == 0) wi = 1;
      acc += wi;
      s->cum[i] = acc;
    }
    s->total = acc;
  } else if (s->kind == 2) {
    s->mu = p->size_p1;
    s->sigma = p->size_p2;
  } else if (s->kind != 0) {
    return 0;
  }
  return 1;
}

static int32_t sizes_draw(size_sampler* s, rng_t* r) {
  if (s->kind == 0) {
    return s->lo + (int32_t)rng_below(r, (uint64_t)(s->hi - s->lo + 1));
  }
  if (s->kind == 1) {
    uint64_t t = rng_below(r, s->total);
    int32_t a = 0, b = s->hi - s->lo;      /* first i with cum[i] > t */
    while (a < b) {
      int32_t m = (a + b) / 2;
      if (s->cum[m] > t) b = m; else a = m + 1;
    }
    return s->lo + a;
  }
  /* log-normal via the Marsaglia polar method (needs only log and sqrt) */
  double u, v, q;
  do {
    u = 2.0 * rng_unit(r) - 1.0;
    v = 2.0 * rng_unit(r) - 1.0;
    q = u * u + v * v;
  } while (q >= 1.0 || q == 0.0);
  double z = u * sqrt(-2.0 * det_log(q) / q);
  double k = floor(det_exp(s->mu + s->sigma * z) + 0.5);
  if (k < (double)s->lo) k = (double)s->lo;
  if (k > (double)s->hi) k = (double)s->hi;
  return (int32_t)k;
}

/* ---------------- duplicate detection ---------------- */

typedef struct {
  int64_t cap;      /* power of two */
  int64_t* slot;    /* hyperedge index or -1 */
} edge_set;

static uint64_t hash_tuple(const int32_t* v, int32_t k) {
  uint64_t h = 0xCBF29CE484222325ull ^ (uint64_t)k;
  for (int32_t i = 0; i < k; ++i) {
    h ^= (uint64_t)(uint32_t)v[i];
    h *= 0x100000001B3ull;
    h ^= h >> 29;
  }
  return h;
}

static int tuple_eq(const int32_t* a, int32_t ka, const int32_t* b, int32_t kb) {
  if (ka != kb) return 0;
  for (int32_t i = 0; i < ka; ++i) if (a[i] != b[i]) return 0;
  return 1;
}

/* returns 1 if inserted, 0 if an equal hyperedge exists */
static int edge_set_insert(edge_set* s, const int64_t* e_ptr, const int32_t* e_idx,
                           int64_t id) {
  const int32_t* v = e_idx + e_ptr[id];
  int32_t k = (int32_t)(e_ptr[id + 1] - e_ptr[id]);
  uint64_t h = hash_tuple(v, k);
  int64_t m = s->cap - 1;
  for (int64_t p = (int64_t)(h & (uint64_t)m);; p = (p + 1) & m) {
    int64_t o = s->slot[p];
    if (o < 0) { s->slot[p] = id; return 1; }
    if (tuple_eq(e_idx + e_ptr[o], (int32_t)(e_ptr[o + 1] - e_ptr[o]), v, k)) return 0;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* ---------------- public entry points ---------------- */

/* Draw the |E| hyperedge sizes (stream 1).  sizes[num_edges]. */
int hgen_sizes(const hgen_params* p, int32_t* sizes) {
  if (!p || !sizes || p->num_edges < 0) return HGEN_ERR_ARG;
  size_sampler ss;
  if (!sizes_init(&ss, p)) return HGEN_ERR_ARG;
  rng_t r = rng_stream(p->seed, 1);
  for (int64_t i = 0; i < p->num_edges; ++i) sizes[i] = sizes_draw(&ss, &r);
  free(ss.cum);
  return HGEN_OK;
}

/*
 * Fill the hyperedge->vertex CSR given the sizes (stream 2).
 * e_ptr[num_edges+1] (int64) and e_idx[sum sizes] (int32) are caller-owned.
 * Rows come out sorted ascending and duplicate-free.
 */
int hgen_fill(const hgen_params* p, const int32_t* sizes, int64_t* e_ptr, int32_t* e_idx) {
  if (!p || !sizes || !e_ptr || !e_idx || p->num_vertices <= 0 || p->num_edges < 0)
    return HGEN_ERR_ARG;
  const int64_t nv = p->num_vertices, ne = p->num_edges;
  int rc = HGEN_OK;
  uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nv);
  int32_t* deg = (int32_t*)calloc((size_t)nv, sizeof(int32_t));
  edge_set es = {0, NULL};
  fenwick fw = {0, NULL, 0};
  if (!w || !deg) { rc = HGEN_ERR_NOMEM; goto done; }
  for (int64_t r = 0; r < nv; ++r) {
    double x = det_pow((double)(r + 1), -p->zipf_s);
    uint64_t wi = (uint64_t)floor(x * W_SCALE + 0.5);
    w[r] = wi ? wi : 1;
  }
  if (!fw_init(&fw, w, nv)) { rc = HGEN_ERR_NOMEM; goto done; }
  int64_t avail = nv;   /* vertices with non-zero weight in the tree */
  if (p->dedup) {
    es.cap = 16;
    while (es.cap < 2 * ne + 16) es.cap *= 2;
    es.slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)es.cap);
    if (!es.slot) { rc = HGEN_ERR_NOMEM; goto done; }
    memset(es.slot, 0xFF, sizeof(int64_t) * (size_t)es.cap);
  }
  rng_t rv = rng_stream(p->seed, 2);
  e_ptr[0] = 0;
  for (int64_t i = 0; i < ne; ++i) {
    const int32_t k = sizes[i];
    if (k < 1) { rc = HGEN_ERR_ARG; goto done; }
    int32_t* row = e_idx + e_ptr[i];
    e_ptr[i + 1] = e_ptr[i] + k;
    int attempt = 0;
    for (;;) {
      if (k > avail) { rc = HGEN_ERR_EXHAUSTED; goto done; }
      uint64_t total = fw_total(&fw);
      for (int32_t j = 0; j < k; ++j) {
        int64_t v = fw_find(&fw, rng_below(&rv, total));
        row[j] = (int32_t)v;
        total -= w[v];
        fw_add(&fw, v, (uint64_t)0 - w[v]);    /* withdraw for the rest of this hyperedge */
      }
      qsort(row, (size_t)k, sizeof(int32_t), cmp_i32);
      int fresh = p->dedup ? edge_set_insert(&es, e_ptr, e_idx, i) : 1;
      if (fresh) break;
      for (int32_t j = 0; j < k; ++j) fw_add(&fw, row[j], w[row[j]]);   /* undo, redraw */
      if (++attempt > 10000) { rc = HGEN_ERR_DEDUP; goto done; }
    }
    for (int32_t j = 0; j < k; ++j) {
      int32_t v = row[j];
      deg[v] += 1;
      if (p->degree_cap > 0 && deg[v] >= p->degree_cap) {
        avail -= 1;                               /* stays withdrawn */
      } else {
        fw_add(&fw, v, w[v]);                     /* back in the pool */
      }
    }
  }
done:
  free(w);
  free(deg);
  free(fw.t);
  free(es.slot);
  return rc;
}

/* round(exp(U(ln lo, ln hi))) from stream `tag` of `seed`: log-uniform integer sizes */
int64_t hgen_loguniform_int(uint64_t seed, uint64_t tag, int64_t lo, int64_t hi) {
  rng_t r = rng_stream(seed, 1000 + tag);
  double a = det_log((double)lo), b = det_log((double)hi);
  double x = det_exp(a + (b - a) * rng_unit(&r));
  int64_t k = (int64_t)floor(x + 0.5);
  if (k < lo) k = lo;
  if (k > hi) k = hi;
  return k;
}

/* exposed for tests of the deterministic elementary functions */
double hgen_det_log(double x) { return det_log(x); }
double hgen_det_exp(double x) { return det_exp(x); }
