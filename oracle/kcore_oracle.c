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
 *   oc_kcore_sampled  Algorithm 4 with the sampling Peel of Algorithm 5
 *            (Sec. 4.1), round by round, with the recovery check of "Recover
 *            from Errors"; its coins are Philox4x32-10 (oc_philox4x32_10) of
 *            the arc index, so the GPU and this code draw the same coin for the
 *            same arc. Pinned by the generator's published known answers, the
 *            binomial law of the heads on a star, Algorithm 1 when nothing is
 *            sampled, and exactness whenever no miss is reported.
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

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As
 * Easy as 1, 2, 3", SC 2011): ten rounds over a 4-word counter with a 2-word
 * key. A round multiplies counter words 0 and 2 by the two Philox constants,
 * keeps the low halves and xors the high halves with the other two counter
 * words and the key; the key is bumped by the two Weyl constants between
 * rounds. Used for the sampling coins, which are a pure function of the arc
 * (counter = arc index, key = seed). */
void oc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The coin of arc j for a vertex in sample mode with induced degree D: x is
 * the first Philox output word (uniform on 32 bits), and a head means
 * x < floor(2^32 rate) with the sample rate of Sec. 4.1,
 * rate = mu / ((1 - r) D), r = 1/10. In integers: x < floor(10 mu 2^32 / (9 D))
 * holds exactly when 9 D (x + 1) <= 10 mu 2^32, i.e. when
 * D (x + 1) <= floor(10 mu 2^32 / 9). */
static int coin_head(int64_t j, uint64_t seed, int64_t mu, int64_t D) {
  const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  oc_philox4x32_10(ctr, key, o);
  const unsigned __int128 lhs = (unsigned __int128)(9 * (uint64_t)D) * ((uint64_t)o[0] + 1);
  const unsigned __int128 rhs = ((unsigned __int128)(10 * (uint64_t)mu)) << 32;
  return lhs <= rhs;
}

/* Algorithm 4 (the framework with sampling) with the Peel, InitSampler,
 * SetSampler and Error functions of Algorithm 5, sequentially, round by round
 * (k = 0, 1, 2, ... with no round skipped) and subround by subround:
 *   - InitSampler(v, k): sample mode when D r > k and D > threshold, where D
 *     is v's exact induced degree at that moment (r = 1/10, so D > 10 k);
 *     the sample count restarts at 0.
 *   - Round k: the frontier is the live vertices outside sample mode with
 *     induced degree k; then every vertex in sample mode is validated, and
 *     one failing Error(v, k) is recounted by SetSampler (which may add it to
 *     the frontier). Error(v, k) holds when D r > k and
 *     cnt < rate (D - k) / 4, i.e. 18 D cnt < 5 mu (D - k).
 *   - Peel(F, k): the frontier's arcs in frontier order, each arc once; a
 *     neighbour in sample mode takes a head of its coin with probability rate
 *     (the arc's Philox coin), and its mu-th head puts it in the counting bag;
 *     any other neighbour has its induced degree decremented and joins the
 *     next frontier when the decrement returned k + 1. The bag's vertices are
 *     recounted (SetSampler) after the subround.
 *   - SetSampler(v, k, F): the induced degree becomes the number of v's
 *     neighbours whose arcs have not been traversed yet; at or below k, v
 *     joins F; then InitSampler(v, k).
 *   - Recovery (Sec. 4.1, "Recover from Errors"): a recount at round k of a
 *     vertex that had fewer than k untraversed neighbours when round k began
 *     means it missed an earlier round; the run stops and returns 1 (the
 *     caller restarts without sampling).
 * A vertex whose induced degree is 2^29 or more is never sampled (the GPU
 * keeps the sample flag in the induced-degree word).
 * stats (int64[8], may be NULL): [0] vertices sampled by the first
 * InitSampler, [1] SetSampler recounts, [2] counting-bag insertions,
 * [3] failed validations, [4] heads, [5] the round of a detected miss (-1),
 * [6] the vertex of it (-1), [7] rounds.
 * Returns 0 (core[] holds the coreness), 1 (a miss was detected; core[] is
 * incomplete) or -3 (out of memory). */
int oc_kcore_sampled(int64_t n, const int64_t* off, const int32_t* adj, int64_t mu, int64_t threshold,
                     uint64_t seed, int32_t* core, int64_t* stats) {
  int64_t st[8] = {0, 0, 0, 0, 0, -1, -1, 0};
  if (n <= 0) {
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
  }
  if (mu < 1) mu = 1;
  const int64_t kCap = (int64_t)1 << 29;
  int64_t* dt = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);    /* induced degree (D when sampled) */
  int64_t* cnt = (int64_t*)calloc((size_t)n, sizeof(int64_t));    /* heads since InitSampler */
  int64_t* done = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);  /* round its arcs were traversed */
  uint8_t* smode = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* inbag = (uint8_t*)calloc((size_t)n, 1);
  int32_t* alive = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* F = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* Fn = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* bag = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!dt || !cnt || !done || !smode || !inbag || !alive || !F || !Fn || !bag) {
    free(dt); free(cnt); free(done); free(smode); free(inbag); free(alive); free(F); free(Fn); free(bag);
    return -3;
  }
  const int64_t kNever = INT64_MAX;
  int64_t na = n;
  for (int64_t v = 0; v < n; v++) {
    dt[v] = off[v + 1] - off[v];
    done[v] = kNever;
    alive[v] = (int32_t)v;
    core[v] = -1;
  }
  /* InitSampler(v, 0) for every v */
  for (int64_t v = 0; v < n; v++) {
    const int64_t D = dt[v];
    if (D > 0 && D > threshold && D < kCap) {
      smode[v] = 1;
      cnt[v] = 0;
      st[0]++;
    }
  }
  int rc = 0;
  int64_t k = 0;
  while (na > 0 && rc == 0) {
    st[7]++;
    /* frontier of round k: live vertices outside sample mode with induced degree k */
    int64_t nf = 0;
    for (int64_t i = 0; i < na; i++) {
      const int32_t v = alive[i];
      if (!smode[v] && dt[v] == k) F[nf++] = v;
    }
    /* validate every vertex in sample mode; recount those that fail Error(v, k) */
    for (int64_t i = 0; i < na && rc == 0; i++) {
      const int32_t v = alive[i];
      if (!smode[v]) continue;
      const int64_t D = dt[v];
      const int ok = D > 10 * k && 18 * D * cnt[v] < 5 * mu * (D - k);
      if (ok) continue;
      st[3]++;
      /* SetSampler(v, k, F) */
      st[1]++;
      int64_t left = 0, at_start = 0;
      for (int64_t j = off[v]; j < off[v + 1]; j++) {
        const int64_t d = done[adj[j]];
        if (d == kNever) left++;
        if (d >= k) at_start++;
      }
      if (at_start < k) {
        st[5] = k;
        st[6] = v;
        rc = 1;
        break;
      }
      dt[v] = left;
      smode[v] = 0;
      if (left <= k) F[nf++] = v;
      else if (left > 10 * k && left > threshold && left < kCap) {
        smode[v] = 1;
        cnt[v] = 0;
      }
    }
    while (nf > 0 && rc == 0) {
      for (int64_t i = 0; i < nf; i++) core[F[i]] = (int32_t)k;
      /* Peel(F, k) with sampling */
      int64_t nn = 0, nb = 0;
      for (int64_t i = 0; i < nf; i++) {
        const int32_t v = F[i];
        done[v] = k;
        for (int64_t j = off[v]; j < off[v + 1]; j++) {
          const int32_t u = adj[j];
          if (smode[u]) {
            if (coin_head(j, seed, mu, dt[u])) {
              st[4]++;
              if (cnt[u]++ == mu - 1 && !inbag[u]) {
                inbag[u] = 1;
                bag[nb++] = u;
                st[2]++;
              }
            }
          } else {
            const int64_t before = dt[u]--;
            if (before == k + 1) Fn[nn++] = u;
          }
        }
      }
      /* SetSampler(v, k, F') for the counting bag */
      for (int64_t i = 0; i < nb; i++) {
        const int32_t v = bag[i];
        inbag[v] = 0;
        st[1]++;
        int64_t left = 0, at_start = 0;
        for (int64_t j = off[v]; j < off[v + 1]; j++) {
          const int64_t d = done[adj[j]];
          if (d == kNever) left++;
          if (d >= k) at_start++;
        }
        if (at_start < k) {
          st[5] = k;
          st[6] = v;
          rc = 1;
          break;
        }
        dt[v] = left;
        smode[v] = 0;
        if (left <= k) Fn[nn++] = v;
        else if (left > 10 * k && left > threshold && left < kCap) {
          smode[v] = 1;
          cnt[v] = 0;
        }
      }
      int32_t* t = F; F = Fn; Fn = t;
      nf = nn;
    }
    /* keep the live vertices above k (a vertex in sample mode is live) */
    int64_t w = 0;
    for (int64_t i = 0; i < na; i++) {
      const int32_t v = alive[i];
      if (smode[v] || dt[v] > k) alive[w++] = v;
    }
    na = w;
    k++;
  }
  if (stats) memcpy(stats, st, sizeof(st));
  free(dt); free(cnt); free(done); free(smode); free(inbag); free(alive); free(F); free(Fn); free(bag);
  return rc;
}
