/*
 * CPU oracle for exact k-core decomposition.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled and called by the tests,
 * by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * library. It shares no code, header or table with the CUDA path.
 *
 * What it computes (arXiv 2502.08042, Sec. 2 "Notations"): the k-core G_k is
 * the largest subgraph in which every vertex has degree at least k; the
 * coreness of v is the largest k with v in G_k; k_max is the largest coreness.
 * That result is unique, so it is computed here in independent ways:
 *
 *   oc_bz    Batagelj & Zaversnik, "An O(m) Algorithm for Cores Decomposition
 *            of Networks" (2003): the sequential bucket peel the paper uses as
 *            its sequential baseline (Sec. 6, "BZ").
 *   oc_alg1  Algorithm 1 of the paper taken step by step with its sequential
 *            Peel: rounds k = 0, 1, ...; frontier = live vertices with induced
 *            degree equal to k; subrounds decrement every neighbour and collect
 *            those that land on k; after the round keep only vertices with
 *            induced degree above k. It also counts the quantities of
 *            Theorem 1 (sum of active-set sizes, frontier insertions).
 *   oc_kcore_mask  The k'-core alone (App. B): repeated deletion of the
 *            vertices whose remaining degree is below k'.
 *   oc_check A certificate check that needs no decomposition: (i) every v
 *            with value c has at least c neighbours with value >= c (so the
 *            set {value >= c} has minimum degree >= c and lies inside the
 *            c-core), and (iii) a removal order exists, by increasing value,
 *            in which every v has at most value(v) neighbours left when it is
 *            removed (so v is not in the (value(v)+1)-core). Together they
 *            force value == coreness. (ii) every v has at most value(v)
 *            neighbours of larger value, a cheap consequence of (iii).
 *
 * oc_build_csr builds the simple undirected graph of an edge list by its
 * definition: each pair (a, b) with a != b contributes arcs a->b and b->a;
 * arcs are sorted by (source, target) with two stable counting sorts (target
 * first, then source) and equal arcs are kept once. The paper symmetrises
 * directed inputs (Sec. 6.1, "Datasets").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* CSR of the simple undirected graph of an edge list.
 * off[n+1], adj[capacity >= 2*E]. Returns the number of arcs, or < 0 on error
 * (-1 bad argument, -2 vertex id out of range, -3 out of memory). */
int64_t oc_build_csr(int64_t n, int64_t E, const int32_t* src, const int32_t* dst, int64_t* off,
                     int32_t* adj) {
  if (n < 0 || E < 0) return -1;
  int64_t A = 0;
  for (int64_t i = 0; i < E; i++) {
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -2;
    if (src[i] != dst[i]) A += 2;
  }
  int32_t* s1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A ? A : 1));
  int32_t* d1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A ? A : 1));
  int32_t* s2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A ? A : 1));
  int32_t* d2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A ? A : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!s1 || !d1 || !s2 || !d2 || !cnt) {
    free(s1); free(d1); free(s2); free(d2); free(cnt);
    return -3;
  }
  int64_t a = 0;
  for (int64_t i = 0; i < E; i++) {
    if (src[i] == dst[i]) continue;
    s1[a] = src[i]; d1[a] = dst[i]; a++;
    s1[a] = dst[i]; d1[a] = src[i]; a++;
  }
  /* stable counting sort by target: (s1,d1) -> (s2,d2) */
  for (int64_t i = 0; i < A; i++) cnt[d1[i] + 1]++;
  for (int64_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
  for (int64_t i = 0; i < A; i++) {
    int64_t p = cnt[d1[i]]++;
    s2[p] = s1[i]; d2[p] = d1[i];
  }
  /* stable counting sort by source: (s2,d2) -> (s1,d1) */
  memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t i = 0; i < A; i++) cnt[s2[i] + 1]++;
  for (int64_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
  for (int64_t i = 0; i < A; i++) {
    int64_t p = cnt[s2[i]]++;
    s1[p] = s2[i]; d1[p] = d2[i];
  }
  /* keep each arc once; lists come out ascending */
  int64_t m = 0;
  for (int64_t v = 0; v <= n; v++) off[v] = 0;
  for (int64_t i = 0; i < A; i++) {
    if (i > 0 && s1[i] == s1[i - 1] && d1[i] == d1[i - 1]) continue;
    adj[m++] = d1[i];
    off[s1[i] + 1]++;
  }
  for (int64_t v = 0; v < n; v++) off[v + 1] += off[v];
  free(s1); free(d1); free(s2); free(d2); free(cnt);
  return m;
}

/* Checks the CSR is a simple undirected graph: offsets monotone from 0 to m,
 * ids in range, each list strictly ascending (no duplicates), no self-loops,
 * and every arc u->v has its reverse v->u. Returns 0 if so, else a code > 0. */
int oc_check_simple(int64_t n, const int64_t* off, const int32_t* adj) {
  if (n < 0) return 1;
  if (off[0] != 0) return 2;
  for (int64_t v = 0; v < n; v++) {
    if (off[v + 1] < off[v]) return 3;
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      int32_t u = adj[j];
      if (u < 0 || u >= n) return 4;
      if (u == v) return 5;
      if (j > off[v] && adj[j - 1] >= u) return 6;
      /* reverse arc by binary search in u's ascending list */
      int64_t lo = off[u], hi = off[u + 1];
      while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (adj[mid] < (int32_t)v) lo = mid + 1; else hi = mid;
      }
      if (lo >= off[u + 1] || adj[lo] != (int32_t)v) return 7;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Batagelj-Zaversnik bucket peel. Vertices are kept sorted by current degree
 * in vert[] (pos[] is the inverse); bin[d] is where degree d starts. Visiting
 * vertices in that order, a vertex's degree when reached is its coreness;
 * every neighbour with a larger degree moves to the front of its degree block
 * and its degree drops by one. Returns 0, or -3 when out of memory. */
int oc_bz(int64_t n, const int64_t* off, const int32_t* adj, int32_t* core) {
  if (n <= 0) return 0;
  int32_t* deg = core; /* the degree array becomes the coreness array */
  int64_t md = 0;
  for (int64_t v = 0; v < n; v++) {
    deg[v] = (int32_t)(off[v + 1] - off[v]);
    if (deg[v] > md) md = deg[v];
  }
  int64_t* bin = (int64_t*)calloc((size_t)md + 2, sizeof(int64_t));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* vert = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!bin || !pos || !vert) {
    free(bin); free(pos); free(vert);
    return -3;
  }
  for (int64_t v = 0; v < n; v++) bin[deg[v]]++;
  int64_t start = 0;
  for (int64_t d = 0; d <= md; d++) {
    int64_t num = bin[d];
    bin[d] = start;
    start += num;
  }
  for (int64_t v = 0; v < n; v++) {
    pos[v] = bin[deg[v]];
    vert[pos[v]] = (int32_t)v;
    bin[deg[v]]++;
  }
  for (int64_t d = md; d >= 1; d--) bin[d] = bin[d - 1];
  bin[0] = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = vert[i];
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      int32_t u = adj[j];
      if (deg[u] > deg[v]) {
        int32_t du = deg[u];
        int64_t pu = pos[u];
        int64_t pw = bin[du];
        int32_t w = vert[pw];
        if (u != w) {
          pos[u] = pw; vert[pu] = w;
          pos[w] = pu; vert[pw] = u;
        }
        bin[du]++;
        deg[u]--;
      }
    }
  }
  free(bin); free(pos); free(vert);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 with the sequential Peel. stats (may be NULL) receives:
 *   [0] rounds executed (k = 0 .. k_max, empty levels included)
 *   [1] subrounds executed (non-empty frontiers processed)
 *   [2] sum over rounds of the active-set size at the start of the round
 *   [3] frontier insertions (each vertex must be inserted exactly once)
 *   [4] k_max
 *   [5] non-empty rounds
 * Returns 0, or -3 when out of memory. */
int oc_alg1(int64_t n, const int64_t* off, const int32_t* adj, int32_t* core, int64_t* stats) {
  int64_t st[6] = {0, 0, 0, 0, 0, 0};
  if (n <= 0) {
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
  }
  int64_t* dt = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* alive = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* F = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* Fn = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!dt || !alive || !F || !Fn) {
    free(dt); free(alive); free(F); free(Fn);
    return -3;
  }
  int64_t na = n;
  for (int64_t v = 0; v < n; v++) {
    dt[v] = off[v + 1] - off[v];
    alive[v] = (int32_t)v;
  }
  int64_t k = 0;
  while (na > 0) {
    st[0]++;
    st[2] += na;
    /* initial frontier of round k: live vertices with induced degree k */
    int64_t nf = 0;
    for (int64_t i = 0; i < na; i++)
      if (dt[alive[i]] == k) F[nf++] = alive[i];
    if (nf > 0) st[5]++;
    while (nf > 0) {
      st[1]++;
      for (int64_t i = 0; i < nf; i++) {
        core[F[i]] = (int32_t)k;
        st[3]++;
      }
      /* sequential Peel(F, k) */
      int64_t nn = 0;
      for (int64_t i = 0; i < nf; i++) {
        int32_t v = F[i];
        for (int64_t j = off[v]; j < off[v + 1]; j++) {
          int32_t u = adj[j];
          dt[u] = dt[u] - 1;
          if (dt[u] == k) Fn[nn++] = u;
        }
      }
      int32_t* t = F; F = Fn; Fn = t;
      nf = nn;
    }
    /* refine the active set: keep induced degree above k */
    int64_t w = 0;
    int64_t peeled_here = 0;
    for (int64_t i = 0; i < na; i++) {
      if (dt[alive[i]] > k) alive[w++] = alive[i];
      else peeled_here++;
    }
    if (peeled_here > 0) st[4] = k;
    na = w;
    k++;
  }
  if (stats) memcpy(stats, st, sizeof(st));
  free(dt); free(alive); free(F); free(Fn);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Certificate check of a claimed coreness vector (see header). Returns 0 when
 * value == coreness; otherwise 1, 2 or 3 for a failure of (i), (ii) or (iii)
 * (or 4 for a negative value, -3 when out of memory) and stores the first
 * offending vertex in *bad. */
int oc_check(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* val, int64_t* bad) {
  *bad = -1;
  if (n <= 0) return 0;
  int32_t vmax = 0;
  for (int64_t v = 0; v < n; v++) {
    if (val[v] < 0) { *bad = v; return 4; }
    if (val[v] > vmax) vmax = val[v];
  }
  /* (i) and (ii) */
  for (int64_t v = 0; v < n; v++) {
    int64_t ge = 0, gt = 0;
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      int32_t u = adj[j];
      if (val[u] >= val[v]) ge++;
      if (val[u] > val[v]) gt++;
    }
    if (ge < val[v]) { *bad = v; return 1; }
    if (gt > val[v]) { *bad = v; return 2; }
  }
  /* (iii) removal order by increasing value: bucket vertices by value */
  int64_t* bstart = (int64_t*)calloc((size_t)vmax + 2, sizeof(int64_t));
  int32_t* byval = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* left = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  char* gone = (char*)calloc((size_t)n, 1);
  char* queued = (char*)calloc((size_t)n, 1);
  int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!bstart || !byval || !left || !gone || !queued || !q) {
    free(bstart); free(byval); free(left); free(gone); free(queued); free(q);
    return -3;
  }
  for (int64_t v = 0; v < n; v++) bstart[val[v] + 1]++;
  for (int32_t c = 0; c <= vmax; c++) bstart[c + 1] += bstart[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)vmax + 1));
    memcpy(fill, bstart, sizeof(int64_t) * ((size_t)vmax + 1));
    for (int64_t v = 0; v < n; v++) byval[fill[val[v]]++] = (int32_t)v;
    free(fill);
  }
  for (int64_t v = 0; v < n; v++) left[v] = off[v + 1] - off[v];
  int rc = 0;
  for (int32_t c = 0; c <= vmax && rc == 0; c++) {
    int64_t qh = 0, qt = 0;
    for (int64_t i = bstart[c]; i < bstart[c + 1]; i++) {
      int32_t v = byval[i];
      if (left[v] <= c) { q[qt++] = v; queued[v] = 1; }
    }
    while (qh < qt) {
      int32_t v = q[qh++];
      gone[v] = 1;
      for (int64_t j = off[v]; j < off[v + 1]; j++) {
        int32_t u = adj[j];
        if (gone[u]) continue;
        left[u]--;
        if (val[u] == c && !queued[u] && left[u] <= c) { q[qt++] = u; queued[u] = 1; }
      }
    }
    for (int64_t i = bstart[c]; i < bstart[c + 1]; i++)
      if (!gone[byval[i]]) { *bad = byval[i]; rc = 3; break; }
  }
  free(bstart); free(byval); free(left); free(gone); free(queued); free(q);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* The k'-core (App. B, "Maximum k-Core Subgraph"; the k-core definition of
 * Sec. 2): the largest subgraph in which every vertex has degree >= kp,
 * obtained by deleting, as long as one exists, a vertex whose degree among the
 * vertices not yet deleted is below kp. A vertex is queued when its remaining
 * degree first drops below kp (or starts below it) and deleted when taken from
 * the queue; deleting it lowers the remaining degree of its neighbours.
 * mask[v] = 1 when v is in the k'-core, else 0. Returns the k'-core's vertex
 * count, or -1 when out of memory. */
int64_t oc_kcore_mask(int64_t n, const int64_t* off, const int32_t* adj, int32_t kp, int32_t* mask) {
  if (n <= 0) return 0;
  int64_t* left = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!left || !q) {
    free(left);
    free(q);
    return -1;
  }
  int64_t qt = 0;
  for (int64_t v = 0; v < n; v++) {
    left[v] = off[v + 1] - off[v];
    mask[v] = 1;
    if (left[v] < kp) {
      mask[v] = 0; /* queued = deleted once processed */
      q[qt++] = (int32_t)v;
    }
  }
  for (int64_t qh = 0; qh < qt; qh++) {
    int32_t v = q[qh];
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      int32_t u = adj[j];
      if (!mask[u]) continue; /* already deleted or queued */
      if (--left[u] < kp) {
        mask[u] = 0;
        q[qt++] = u;
      }
    }
  }
  free(left);
  free(q);
  return n - qt;
}
