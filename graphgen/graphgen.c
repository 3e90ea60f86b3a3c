/*
 * Seeded synthetic graph generators (host C, pthreads).
 *
 * These produce raw edge lists (COO pairs) shaped like the paper's workload
 * classes (Sec. 6.1: power-law social/web graphs, kNN graphs, synthetic
 * graphs). They hold none of the peeling arithmetic and none of the CSR
 * construction: duplicates, both directions and self-loops may appear in the
 * output of the RMAT and kNN generators and are left for the CSR builders
 * (the GPU one and the oracle's) to remove.
 *
 * Randomness is counter-based: every random number is
 *     mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15)
 * where mix64 is the SplitMix64 output function (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) and
 * key = mix64(seed ^ tag) per stream. Because a draw depends only on
 * (seed, stream, counter), parallel loops give the same output for any
 * thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t rng_at(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * GOLDEN);
}
static inline uint64_t stream_key(uint64_t seed, uint64_t tag) {
  return mix64(seed ^ mix64(tag + GOLDEN));
}
/* uniform double in [0, 1) with 53 random bits */
static inline double u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }
/* uniform integer in [0, n) by multiply-high */
static inline uint64_t below(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

/* ------------------------------------------------------------------------- */
/* thread pool helper: run fn(lo, hi, arg) over [0, total) split in chunks   */
typedef void (*range_fn)(int64_t lo, int64_t hi, void* arg);
typedef struct {
  range_fn fn;
  void* arg;
  int64_t total, chunk;
  int64_t next; /* guarded by mu */
  pthread_mutex_t mu;
} par_ctx;

static int gg_threads(void) {
  const char* s = getenv("GRAPHGEN_THREADS");
  if (s && atoi(s) > 0) return atoi(s);
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  if (c < 1) c = 1;
  if (c > 64) c = 64;
  return (int)c;
}

static void* par_worker(void* p) {
  par_ctx* c = (par_ctx*)p;
  for (;;) {
    pthread_mutex_lock(&c->mu);
    int64_t lo = c->next;
    c->next += c->chunk;
    pthread_mutex_unlock(&c->mu);
    if (lo >= c->total) break;
    int64_t hi = lo + c->chunk;
    if (hi > c->total) hi = c->total;
    c->fn(lo, hi, c->arg);
  }
  return NULL;
}

static void parallel_for(int64_t total, int64_t chunk, range_fn fn, void* arg) {
  if (total <= 0) return;
  par_ctx c;
  c.fn = fn;
  c.arg = arg;
  c.total = total;
  c.chunk = chunk < 1 ? 1 : chunk;
  c.next = 0;
  pthread_mutex_init(&c.mu, NULL);
  int nt = gg_threads();
  if ((total + c.chunk - 1) / c.chunk < nt) nt = (int)((total + c.chunk - 1) / c.chunk);
  if (nt <= 1) {
    par_worker(&c);
  } else {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
    for (int i = 0; i < nt; i++) pthread_create(&th[i], NULL, par_worker, &c);
    for (int i = 0; i < nt; i++) pthread_join(th[i], NULL);
    free(th);
  }
  pthread_mutex_destroy(&c.mu);
}

/* ------------------------------------------------------------------------- */
/* open-addressing set of 64-bit keys (key 0 reserved as empty; callers add 1) */
typedef struct {
  uint64_t* slot;
  uint64_t mask;
} u64set;

static int set_init(u64set* s, int64_t expected) {
  uint64_t cap = 16;
  while (cap < (uint64_t)expected * 2 + 16) cap <<= 1;
  s->slot = (uint64_t*)calloc(cap, sizeof(uint64_t));
  s->mask = cap - 1;
  return s->slot ? 0 : -1;
}
static void set_free(u64set* s) { free(s->slot); }
/* returns 1 if inserted, 0 if present */
static int set_insert(u64set* s, uint64_t key) {
  uint64_t k = key + 1, i = mix64(k) & s->mask;
  for (;;) {
    if (s->slot[i] == 0) {
      s->slot[i] = k;
      return 1;
    }
    if (s->slot[i] == k) return 0;
    i = (i + 1) & s->mask;
  }
}

/* ------------------------------------------------------------------------- */
/* Random permutation of [0, n) by Fisher-Yates driven by the counter stream. */
static void random_permutation(int64_t n, uint64_t seed, int32_t* perm) {
  uint64_t key = stream_key(seed, 0x7065726dULL /* "perm" */);
  for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)below(rng_at(key, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

int gg_permutation(int64_t n, uint64_t seed, int32_t* perm) {
  if (n < 0) return -1;
  random_permutation(n, seed, perm);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Erdos-Renyi G(n, m): m distinct unordered pairs {u, v}, u != v, drawn
 * uniformly without replacement by rejection. Pairs are written as drawn
 * (src = first endpoint drawn). Requires m <= n(n-1)/2. */
int gg_er(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
  if (n < 0 || m < 0) return -1;
  if (m == 0) return 0;
  if (n < 2 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -2;
  u64set s;
  if (set_init(&s, m)) return -3;
  uint64_t key = stream_key(seed, 0x6572ULL /* "er" */);
  uint64_t ctr = 0;
  int64_t got = 0;
  while (got < m) {
    uint64_t u = below(rng_at(key, ctr++), (uint64_t)n);
    uint64_t v = below(rng_at(key, ctr++), (uint64_t)n);
    if (u == v) continue;
    uint64_t a = u < v ? u : v, b = u < v ? v : u;
    if (!set_insert(&s, (a << 32) | b)) continue;
    src[got] = (int32_t)u;
    dst[got] = (int32_t)v;
    got++;
  }
  set_free(&s);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* R-MAT (Chakrabarti, Zhan & Faloutsos 2004), Graph500-style, no per-level
 * noise: edge i chooses one quadrant per level from the most significant bit
 * down with probabilities (a, b, c, 1-a-b-c). Vertex ids are then relabelled
 * by a random permutation of [0, 2^scale). Output keeps duplicates and
 * self-loops; count = edges requested. */
typedef struct {
  int scale;
  double a, ab, abc;
  uint64_t key;
  const int32_t* perm;
  int32_t *src, *dst;
} rmat_arg;

static void rmat_range(int64_t lo, int64_t hi, void* p) {
  rmat_arg* r = (rmat_arg*)p;
  for (int64_t i = lo; i < hi; i++) {
    uint64_t u = 0, v = 0;
    uint64_t base = (uint64_t)i * (uint64_t)r->scale;
    for (int l = 0; l < r->scale; l++) {
      double x = u01(rng_at(r->key, base + (uint64_t)l));
      uint64_t bu, bv;
      if (x < r->a) {
        bu = 0; bv = 0;
      } else if (x < r->ab) {
        bu = 0; bv = 1;
      } else if (x < r->abc) {
        bu = 1; bv = 0;
      } else {
        bu = 1; bv = 1;
      }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    r->src[i] = r->perm ? r->perm[u] : (int32_t)u;
    r->dst[i] = r->perm ? r->perm[v] : (int32_t)v;
  }
}

int gg_rmat(int scale, int64_t edges, double a, double b, double c, uint64_t seed,
            uint64_t perm_seed, int permute, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || edges < 0) return -1;
  int64_t n = (int64_t)1 << scale;
  int32_t* perm = NULL;
  if (permute) {
    perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm) return -3;
    random_permutation(n, perm_seed, perm);
  }
  rmat_arg r;
  r.scale = scale;
  r.a = a;
  r.ab = a + b;
  r.abc = a + b + c;
  r.key = stream_key(seed, 0x726d6174ULL /* "rmat" */);
  r.perm = perm;
  r.src = src;
  r.dst = dst;
  parallel_for(edges, 1 << 16, rmat_range, &r);
  free(perm);
  return 0;
}

/* R-MAT restricted to n vertices with exactly m distinct undirected non-loop
 * edges: scale = ceil(log2 n), ids permuted over [0, 2^scale), endpoints >= n
 * rejected, duplicates and loops rejected, drawn until m are kept. Sequential
 * (used per graph of a batch). Requires m well below n(n-1)/2. */
int gg_rmat_n(int64_t n, int64_t m, double a, double b, double c, uint64_t seed,
              int32_t* src, int32_t* dst) {
  if (n < 2 || m < 0) return -1;
  if ((double)m > 0.25 * (double)n * (double)(n - 1)) return -2;
  int scale = 1;
  while (((int64_t)1 << scale) < n) scale++;
  int64_t N = (int64_t)1 << scale;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  if (!perm) return -3;
  random_permutation(N, seed ^ 0x5045524dULL, perm);
  u64set s;
  if (set_init(&s, m)) {
    free(perm);
    return -3;
  }
  uint64_t key = stream_key(seed, 0x726d6174ULL);
  /* quadrant thresholds in 16-bit fixed point: one 64-bit draw serves 4 levels */
  uint32_t ta = (uint32_t)llround(a * 65536.0), tab = (uint32_t)llround((a + b) * 65536.0),
           tabc = (uint32_t)llround((a + b + c) * 65536.0);
  uint64_t ctr = 0;
  int64_t got = 0;
  while (got < m) {
    uint64_t u = 0, v = 0, r = 0;
    for (int l = 0; l < scale; l++) {
      if ((l & 3) == 0) r = rng_at(key, ctr++);
      uint32_t x = (uint32_t)((r >> (16 * (l & 3))) & 0xffffu);
      uint64_t bu = x >= tab, bv = (x >= ta && x < tab) || x >= tabc;
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    uint64_t pu = (uint64_t)perm[u], pv = (uint64_t)perm[v];
    if (pu >= (uint64_t)n || pv >= (uint64_t)n || pu == pv) continue;
    uint64_t lo = pu < pv ? pu : pv, hi = pu < pv ? pv : pu;
    if (!set_insert(&s, (lo << 32) | hi)) continue;
    src[got] = (int32_t)pu;
    dst[got] = (int32_t)pv;
    got++;
  }
  set_free(&s);
  free(perm);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Directed k-nearest-neighbour graph of n points uniform in [0,1)^2.
 * Point i = (u01(r(2i)), u01(r(2i+1))). Distances in double; ties broken by
 * the smaller index. Output: for each i, k pairs (i, j) in order of
 * increasing (distance, j). Exact search on a uniform grid of cells. */
typedef struct {
  int64_t n;
  int k;
  const double *x, *y;
  int64_t G;           /* cells per side */
  double cs;           /* cell size */
  const int64_t* cstart; /* G*G+1 */
  const int32_t* cpts;
  int32_t *src, *dst;
} knn_arg;

static inline int64_t cell_of(double v, int64_t G) {
  int64_t c = (int64_t)(v * (double)G);
  if (c < 0) c = 0;
  if (c >= G) c = G - 1;
  return c;
}

static void knn_range(int64_t lo, int64_t hi, void* p) {
  knn_arg* A = (knn_arg*)p;
  int k = A->k;
  double* bd = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  int32_t* bj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k + 1));
  for (int64_t i = lo; i < hi; i++) {
    double px = A->x[i], py = A->y[i];
    int64_t cx = cell_of(px, A->G), cy = cell_of(py, A->G);
    int cnt = 0;
    for (int64_t R = 0;; R++) {
      for (int64_t gx = cx - R; gx <= cx + R; gx++) {
        if (gx < 0 || gx >= A->G) continue;
        int64_t step = (gx == cx - R || gx == cx + R) ? 1 : 2 * R;
        for (int64_t gy = cy - R; gy <= cy + R; gy += (step ? step : 1)) {
          if (gy < 0 || gy >= A->G) continue;
          int64_t cell = gx * A->G + gy;
          for (int64_t t = A->cstart[cell]; t < A->cstart[cell + 1]; t++) {
            int32_t j = A->cpts[t];
            if (j == i) continue;
            double dx = A->x[j] - px, dy = A->y[j] - py;
            double d = dx * dx + dy * dy;
            /* insertion into the sorted best list of size <= k */
            if (cnt == k && (d > bd[k - 1] || (d == bd[k - 1] && j > bj[k - 1]))) continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && (bd[pos - 1] > d || (bd[pos - 1] == d && bj[pos - 1] > j))) {
              bd[pos] = bd[pos - 1];
              bj[pos] = bj[pos - 1];
              pos--;
            }
            bd[pos] = d;
            bj[pos] = j;
            if (cnt < k) cnt++;
          }
          if (R == 0) break;
        }
      }
      /* every point outside rings 0..R is at distance >= R * cs */
      double bound = (double)R * A->cs;
      if (cnt == k && bd[k - 1] < bound * bound) break;
      if (R > 2 * A->G + 2) break; /* whole domain searched */
    }
    for (int t = 0; t < cnt; t++) {
      A->src[i * k + t] = (int32_t)i;
      A->dst[i * k + t] = bj[t];
    }
    for (int t = cnt; t < k; t++) { /* only when n <= k: pad with self-loops */
      A->src[i * k + t] = (int32_t)i;
      A->dst[i * k + t] = (int32_t)i;
    }
  }
  free(bd);
  free(bj);
}

typedef struct {
  uint64_t key;
  double *x, *y;
} pts_arg;
static void pts_range(int64_t lo, int64_t hi, void* p) {
  pts_arg* a = (pts_arg*)p;
  for (int64_t i = lo; i < hi; i++) {
    a->x[i] = u01(rng_at(a->key, 2 * (uint64_t)i));
    a->y[i] = u01(rng_at(a->key, 2 * (uint64_t)i + 1));
  }
}

int gg_points2d(int64_t n, uint64_t seed, double* x, double* y) {
  pts_arg a;
  a.key = stream_key(seed, 0x6b6e6eULL /* "knn" */);
  a.x = x;
  a.y = y;
  parallel_for(n, 1 << 16, pts_range, &a);
  return 0;
}

int gg_knn2d(int64_t n, int k, uint64_t seed, int32_t* src, int32_t* dst) {
  if (n < 1 || k < 1 || n > 0x7fffffffLL) return -1;
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!x || !y) return -3;
  gg_points2d(n, seed, x, y);
  int64_t G = (int64_t)ceil(sqrt((double)n / 2.0));
  if (G < 1) G = 1;
  int64_t nc = G * G;
  int64_t* cstart = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
  int32_t* cpts = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  if (!cstart || !cpts || !fill) return -3;
  for (int64_t i = 0; i < n; i++) cstart[cell_of(x[i], G) * G + cell_of(y[i], G) + 1]++;
  for (int64_t c = 0; c < nc; c++) cstart[c + 1] += cstart[c];
  memcpy(fill, cstart, sizeof(int64_t) * (size_t)nc);
  for (int64_t i = 0; i < n; i++) cpts[fill[cell_of(x[i], G) * G + cell_of(y[i], G)]++] = (int32_t)i;
  knn_arg A;
  A.n = n;
  A.k = k;
  A.x = x;
  A.y = y;
  A.G = G;
  A.cs = 1.0 / (double)G;
  A.cstart = cstart;
  A.cpts = cpts;
  A.src = src;
  A.dst = dst;
  parallel_for(n, 1 << 12, knn_range, &A);
  free(x);
  free(y);
  free(cstart);
  free(cpts);
  free(fill);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Planted cliques: count cliques with sizes s = floor(exp(U(ln smin, ln smax)))
 * on uniformly random distinct vertex subsets of [0, n). sizes_out[count]
 * receives the sizes; when src is NULL only sizes are computed (so the caller
 * can size the pair buffers: sum s(s-1)/2). Members of clique q are written to
 * members[offset_q ...] if members is not NULL. */
int gg_cliques(int64_t n, int count, int smin, int smax, uint64_t seed, int32_t* sizes_out,
               int32_t* members, int32_t* src, int32_t* dst) {
  if (n < 1 || count < 0 || smin < 2 || smax < smin) return -1;
  uint64_t key = stream_key(seed, 0x636c71ULL /* "clq" */);
  uint64_t ctr = 0;
  double lo = log((double)smin), hi = log((double)smax);
  for (int q = 0; q < count; q++) {
    int s = (int)floor(exp(lo + (hi - lo) * u01(rng_at(key, ctr++))));
    if (s > n) s = (int)n;
    if (s < 2) s = 2;
    sizes_out[q] = s;
  }
  if (!src && !members) return 0;
  int64_t pairs = 0, moff = 0;
  for (int q = 0; q < count; q++) {
    int s = sizes_out[q];
    int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)s);
    u64set set;
    set_init(&set, s);
    uint64_t qkey = stream_key(seed ^ (uint64_t)(q + 1), 0x6d656dULL /* "mem" */);
    uint64_t qc = 0;
    int got = 0;
    while (got < s) {
      uint64_t v = below(rng_at(qkey, qc++), (uint64_t)n);
      if (set_insert(&set, v)) mem[got++] = (int32_t)v;
    }
    set_free(&set);
    if (members) memcpy(members + moff, mem, sizeof(int32_t) * (size_t)s);
    moff += s;
    if (src) {
      for (int i = 0; i < s; i++)
        for (int j = i + 1; j < s; j++) {
          src[pairs] = mem[i];
          dst[pairs] = mem[j];
          pairs++;
        }
    }
    free(mem);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Batch of independent graphs: per graph g, n_g = floor(exp(U(ln nmin, ln nmax))),
 * average degree dbar ~ U(dmin, dmax), m_g = round(n_g * dbar / 2) (capped at a
 * quarter of all pairs), generator ER or R-MAT with probability 1/2 each; the
 * graph uses seed (seed + g). spec_out[4*g + {0,1,2,3}] = n, m, kind (0 ER,
 * 1 RMAT), graph seed. */
int gg_batch_spec(int64_t G, int64_t nmin, int64_t nmax, double dmin, double dmax, uint64_t seed,
                  int64_t* spec_out) {
  if (G < 0 || nmin < 2 || nmax < nmin) return -1;
  for (int64_t g = 0; g < G; g++) {
    uint64_t gs = seed + (uint64_t)g;
    uint64_t key = stream_key(gs, 0x62617463ULL /* "batc" */);
    double ln_lo = log((double)nmin), ln_hi = log((double)nmax);
    int64_t n = (int64_t)floor(exp(ln_lo + (ln_hi - ln_lo) * u01(rng_at(key, 0))));
    if (n < nmin) n = nmin;
    if (n > nmax) n = nmax;
    double dbar = dmin + (dmax - dmin) * u01(rng_at(key, 1));
    int64_t m = (int64_t)llround((double)n * dbar / 2.0);
    double cap = 0.25 * (double)n * (double)(n - 1);
    if ((double)m > cap) m = (int64_t)cap;
    int kind = (int)(rng_at(key, 2) >> 63);
    spec_out[4 * g + 0] = n;
    spec_out[4 * g + 1] = m;
    spec_out[4 * g + 2] = kind;
    spec_out[4 * g + 3] = (int64_t)gs;
  }
  return 0;
}

typedef struct {
  const int64_t* spec;
  const int64_t* eoff; /* edge offset per graph, G+1 */
  double a, b, c;
  int32_t *src, *dst;
  int err;
} batch_arg;

static void batch_range(int64_t lo, int64_t hi, void* p) {
  batch_arg* B = (batch_arg*)p;
  for (int64_t g = lo; g < hi; g++) {
    int64_t n = B->spec[4 * g], m = B->spec[4 * g + 1], kind = B->spec[4 * g + 2];
    uint64_t gs = (uint64_t)B->spec[4 * g + 3];
    int32_t* s = B->src + B->eoff[g];
    int32_t* d = B->dst + B->eoff[g];
    int rc = kind ? gg_rmat_n(n, m, B->a, B->b, B->c, gs, s, d) : gg_er(n, m, gs, s, d);
    if (rc) B->err = rc;
  }
}

/* Generates all graphs of a batch spec; edges of graph g are written at
 * [eoff[g], eoff[g+1]) with graph-local vertex ids. */
int gg_batch_edges(int64_t G, const int64_t* spec, const int64_t* eoff, double a, double b,
                   double c, int32_t* src, int32_t* dst) {
  batch_arg B;
  B.spec = spec;
  B.eoff = eoff;
  B.a = a;
  B.b = b;
  B.c = c;
  B.src = src;
  B.dst = dst;
  B.err = 0;
  parallel_for(G, 1, batch_range, &B);
  return B.err;
}
