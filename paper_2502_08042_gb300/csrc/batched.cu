// Batched k-core peel for sm_103a: thousands of independent graphs, one launch.
//
// Input is a segmented CSR: graph g owns vertices [gv[g], gv[g+1]) of one
// global offsets array, and its adjacency lists hold graph-local ids. Each
// graph is peeled by one CTA with Algorithm 1's round structure and the
// online Peel of Algorithm 3, entirely inside the CTA:
//   * levels: the next level is the minimum induced degree of the live
//     vertices (found while the active list is compacted, so empty levels are
//     never visited); the frontier is the live vertices sitting at that level;
//   * subrounds: the arcs of the current frontier are processed edge-balanced
//     by all threads of the CTA (a block scan of the frontier's degrees, then
//     each thread takes arcs of the concatenated lists); a decrement that
//     returns k+1 lands its vertex on k and appends it to the next subround's
//     frontier; __syncthreads separates subrounds and levels;
//   * the induced degrees live in shared memory when the graph is small enough
//     (shared-memory atomics), otherwise in a per-graph slice of the workspace;
//     when every degree of the graph is below 2^16 they take 16 bits each
//     (twice as many vertices fit in shared memory, half the L2 footprint).
// Persistent CTAs take graphs from a device counter in descending order of
// arcs (longest-processing-time first), so the largest graphs start first.
// Nothing waits on another CTA: the kernel has no spin-waits.
//
// A small batch is bound by its largest graphs, each walked by one CTA while
// the others run out of work. The clustered form (batch_peel_cl) gives every
// graph with more arcs than a threshold (by default the batch's arcs per CTA)
// to a thread-block cluster of C CTAs: the cluster splits each list pass and
// each subround's frontier arcs among its CTAs, keeps the induced degrees in
// L2 and its counters in the first CTA's shared memory (reached through
// distributed shared memory), and closes every phase with the hardware cluster
// barrier. Once a cluster draws a graph below the threshold (the order is by
// arcs, so every later one is too), its CTAs go back to one graph each.
#include <cooperative_groups.h>

#include <climits>

#include "kcore_batched.h"
#include "kcore_device.cuh"

namespace kc {

constexpr int kBatchIlp = 4;
constexpr int kScanItems = 8;  // active-list entries per thread per scan tile

template <int BLOCK>
struct BatchShared {
  int pre[BLOCK];
  long long start[BLOCK];
  int part[BLOCK / 32];
  int red[BLOCK / 32];
  int cnt;
  int g;
  int total;
  int bad;  // this graph failed a bounds check: stop peeling it
  int base;  // clustered peel: this CTA's output position for the current tile
};

// Records a failed bounds check (first one wins: code, graph-local value) and
// flags the status; the access itself is skipped by the caller.
__device__ __forceinline__ void flag_bad(int* status, int code, long long value, int* bad) {
  if (atomicCAS(status, 0, ST_NOT_SIMPLE) == 0) {
    status[1] = code;
    status[2] = (int)(value & 0xffffffffll);
    status[3] = (int)(value >> 32);
  }
  *bad = 1;
}

// Block-wide exclusive scan of one int per thread; returns the exclusive value,
// *total gets the sum. Contains two __syncthreads.
template <int BLOCK>
__device__ __forceinline__ int block_excl_scan(int x, BatchShared<BLOCK>& sh, int* total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int incl = warp_incl_scan(x, lane);
  if (lane == 31) sh.part[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int p = lane < BLOCK / 32 ? sh.part[lane] : 0;
    int pi = warp_incl_scan(p, lane);
    if (lane < BLOCK / 32) sh.part[lane] = pi - p;
    if (lane == BLOCK / 32 - 1) sh.total = pi;
  }
  __syncthreads();
  *total = sh.total;
  return sh.part[warp] + incl - x;
}

template <int BLOCK>
__device__ __forceinline__ int block_min(int x, BatchShared<BLOCK>& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  x = warp_min(x);
  if (lane == 0) sh.red[warp] = x;
  __syncthreads();
  int m = INT_MAX;
  for (int w = 0; w < BLOCK / 32; w++) m = min(m, sh.red[w]);
  __syncthreads();
  return m;
}

// The induced degrees d~ of one graph, in shared memory or in L2 (atomics are
// performed in L2, so a global d~ is never read through L1). Global d~
// accesses carry an evict-last hint and the once-read lists (active list,
// frontiers, adjacency) stream with evict-first loads and stores: with
// hundreds of large graphs in flight their state exceeds L2, and the d~ lines
// are the ones that are hit again.
// Narrow form: two 16-bit values per 32-bit word (vertex v in half v & 1 of
// word v >> 1). A vertex's d~ starts at its degree and falls by one per
// peeled neighbour (each arc is traversed once), so it stays in [0, degree]:
// with every degree below 2^16 a decrement never borrows from the other half.
struct DegStore {
  int* w;
  bool smem, narrow;
  uint64_t pol;
  __device__ __forceinline__ int get(int v) const {
    if (narrow) {
      const int x = smem ? w[v >> 1] : ld_cg_keep(w + (v >> 1), pol);
      return (x >> ((v & 1) * 16)) & 0xffff;
    }
    return smem ? w[v] : ld_cg_keep(w + v, pol);
  }
  // decrements d~[v] by one and returns the value before
  __device__ __forceinline__ int dec(int v) const {
    if (narrow) {
      const int sh = (v & 1) * 16;
      const int old = smem ? atomicSub(w + (v >> 1), 1 << sh) : atom_add_keep(w + (v >> 1), -(1 << sh), pol);
      return (old >> sh) & 0xffff;
    }
    return smem ? atomicSub(w + v, 1) : atom_add_keep(w + v, -1, pol);
  }
  // initial values: one word (narrow: vertices 2i and 2i + 1, degree d1 of
  // the second, 0 past the end)
  __device__ __forceinline__ void put_word(int i, int d0, int d1) const {
    const int x = narrow ? (d0 | (d1 << 16)) : d0;
    if (smem) w[i] = x;
    else st_keep(w + i, x, pol);
  }
};

// One pass over the active list after level k: entries with D > k survive
// into `out` (their minimum goes to *dmin); among them, those at exactly k+1
// are also written to F (the next frontier if level k+1 is not empty).
// Returns the survivors; *nf gets the number written to F.
template <int BLOCK>
__device__ int compact_active(const int* A, int la, int n, int* out, int* F, const DegStore& D, int k,
                              BatchShared<BLOCK>& sh, int* dmin, int* nf) {
  int written = 0, wf = 0, lmin = INT_MAX;
  for (int base = 0; base < la; base += BLOCK * kScanItems) {
    int v[kScanItems];
    unsigned keep = 0, front = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
      int i = base + q * BLOCK + threadIdx.x;
      v[q] = -1;
      if (i < la) {
        int x = __ldcs(A + i);
        v[q] = (unsigned)x < (unsigned)n ? x : -1;  // ids are < n by construction; checked anyway
      }
    }
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
      if (v[q] >= 0) {
        int d = D.get(v[q]);
        if (d > k) {
          keep |= 1u << q;
          lmin = min(lmin, d);
          if (d == k + 1) front |= 1u << q;
        }
      }
    }
    int tot;
    int packed = __popc(keep) | (__popc(front) << 16);
    int pos = block_excl_scan(packed, sh, &tot);
    int pk = written + (pos & 0xffff), pf = wf + (pos >> 16);
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
      if ((keep >> q) & 1u) __stcs(out + pk++, v[q]);
      if ((front >> q) & 1u) __stcs(F + pf++, v[q]);
    }
    written += tot & 0xffff;
    wf += tot >> 16;
  }
  *dmin = block_min(lmin, sh);  // its barriers also publish the writes above
  *nf = wf;
  return written;
}

// Selection of the frontier: entries of A with D[v] == k.
template <int BLOCK>
__device__ int select_frontier(const int* A, int la, int n, int* F, const DegStore& D, int k,
                               BatchShared<BLOCK>& sh) {
  int written = 0;
  for (int base = 0; base < la; base += BLOCK * kScanItems) {
    int v[kScanItems];
    unsigned take = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
      int i = base + q * BLOCK + threadIdx.x;
      v[q] = -1;
      if (i < la) {
        int x = __ldcs(A + i);
        v[q] = (unsigned)x < (unsigned)n ? x : -1;  // ids are < n by construction; checked anyway
      }
    }
#pragma unroll
    for (int q = 0; q < kScanItems; q++)
      if (v[q] >= 0 && D.get(v[q]) == k) take |= 1u << q;
    int tot;
    int pos = block_excl_scan(__popc(take), sh, &tot);
    int p = written + pos;
#pragma unroll
    for (int q = 0; q < kScanItems; q++)
      if ((take >> q) & 1u) __stcs(F + p++, v[q]);
    written += tot;
  }
  __syncthreads();  // the frontier is read by other threads next
  return written;
}

// Peels one graph with the whole CTA (see the file comment).
template <int BLOCK>
__device__ void peel_one_graph(const GraphDesc& gd, int smem_deg_max, int* status, int* sdeg,
                               BatchShared<BLOCK>& sh) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (gd.n <= 0) {
    if (tid == 0) *gd.kmax = 0;
    __syncthreads();
    return;
  }
  const int n = (int)gd.n;
  const long long* O = gd.off;
  const int* adj = gd.adj;
  int* core = gd.core;
  int* A0 = gd.A0;
  int* A1 = gd.A1;
  int* F0 = gd.F0;
  int* F1 = gd.F1;

  // degrees: their minimum (the first level) and maximum (whether 16 bits
  // hold them), then the store, the initial values and the identity active list
  if (tid == 0) sh.bad = 0;
  __syncthreads();
  int lmin = INT_MAX, lmax = 0;
  for (int v = tid; v < n; v += BLOCK) {
    long long o0 = O[v], o1 = O[v + 1];
    if (o0 < 0 || o1 < o0 || o1 > gd.m || o1 - o0 >= n) {
      flag_bad(status, 1, v, &sh.bad);
      o1 = o0;
    }
    const int d = (int)(o1 - o0);
    lmin = min(lmin, d);
    lmax = max(lmax, d);
  }
  int k = block_min(lmin, sh);
  const int dmax = -block_min(-lmax, sh);
  if (sh.bad) {  // malformed offsets: leave this graph (its outputs are undefined)
    if (tid == 0) *gd.kmax = -1;
    __syncthreads();
    return;
  }
  const bool narrow = dmax < 65536;
  const bool in_smem = narrow ? n <= 2 * smem_deg_max : n <= smem_deg_max;
  const DegStore D{in_smem ? sdeg : gd.deg, in_smem, narrow, l2_evict_last_policy()};
  const int nw = narrow ? (n + 1) / 2 : n;
  for (int i = tid; i < nw; i += BLOCK) {
    const int v0 = narrow ? 2 * i : i;
    const int d0 = (int)(O[v0 + 1] - O[v0]);
    const int d1 = narrow && v0 + 1 < n ? (int)(O[v0 + 2] - O[v0 + 1]) : 0;
    D.put_word(i, d0, d1);
  }
  for (int v = tid; v < n; v += BLOCK) __stcs(A0 + v, v);
  __syncthreads();
  int* A = A0;
  int* An = A1;
  int la = n;
  int kmax = 0;
  int nf = select_frontier<BLOCK>(A, la, n, F0, D, k, sh);
  for (;;) {
    int* Fc = F0;
    int* Fn = F1;
    while (nf > 0) {
      for (int i = tid; i < nf; i += BLOCK) {
        int v = __ldcs(Fc + i);
        if ((unsigned)v < (unsigned)n) core[v] = k;
        else flag_bad(status, 6, v, &sh.bad);
      }
      if (tid == 0) sh.cnt = 0;
      __syncthreads();
      for (int c0 = 0; c0 < nf; c0 += BLOCK) {
        const int cnum = min(BLOCK, nf - c0);
        int len = 0;
        long long st = 0;
        if (tid < cnum) {
          int v = __ldcs(Fc + c0 + tid);
          if ((unsigned)v < (unsigned)n) {
            st = O[v];
            long long e = O[v + 1];
            if (st < 0 || e < st || e > gd.m || e - st >= n) flag_bad(status, 2, v, &sh.bad);
            else len = (int)(e - st);
          } else {
            flag_bad(status, 3, v, &sh.bad);
          }
        }
        int total;
        int ex = block_excl_scan(len, sh, &total);
        sh.pre[tid] = ex;
        sh.start[tid] = st;
        __syncthreads();
        for (int j0 = 0; j0 < total; j0 += BLOCK * kBatchIlp) {
          int u[kBatchIlp];
#pragma unroll
          for (int q = 0; q < kBatchIlp; q++) {
            int j = j0 + q * BLOCK + tid;
            u[q] = -1;
            if (j < total) {
              int lo = 0, hi = cnum;
              while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sh.pre[mid] <= j) lo = mid + 1;
                else hi = mid;
              }
              int idx = lo - 1;
              long long arc = sh.start[idx] + (j - sh.pre[idx]);
              if (idx < 0 || arc < 0 || arc >= gd.m) {
                flag_bad(status, 4, arc, &sh.bad);
              } else {
                u[q] = ld_stream_s32(adj + arc);
                if ((unsigned)u[q] >= (unsigned)n) {
                  flag_bad(status, 5, u[q], &sh.bad);
                  u[q] = -1;
                }
              }
            }
          }
#pragma unroll
          for (int q = 0; q < kBatchIlp; q++) {
            bool cross = false;
            // induced degrees in shared memory: read first, decrement the live
            // ones. In global memory each access is an L2 request, so the
            // decrement goes unread: a vertex at or below k is already in a
            // frontier (or peeled), never returns k + 1, and its d~ is only
            // compared with levels above k afterwards.
            if (u[q] >= 0) {
              if (D.smem) cross = D.get(u[q]) > k && D.dec(u[q]) == k + 1;
              else cross = D.dec(u[q]) == k + 1;
            }
            unsigned m = __ballot_sync(kFull, cross);
            if (m) {
              int base = 0;
              if (lane == __ffs(m) - 1) base = atomicAdd(&sh.cnt, __popc(m));
              base = __shfl_sync(kFull, base, __ffs(m) - 1);
              int pos = base + __popc(m & lanemask_lt());
              if (cross) {
                if (pos < n) __stcs(Fn + pos, u[q]);
                else flag_bad(status, 7, pos, &sh.bad);
              }
            }
          }
        }
        __syncthreads();
      }
      nf = sh.cnt;
      if (nf > n) nf = 0;  // cannot happen: every vertex lands on k at most once per level
      __syncthreads();
      int* t = Fc;
      Fc = Fn;
      Fn = t;
    }
    kmax = k;
    // drop the vertices peeled at level k; the minimum induced degree of the
    // rest is the next non-empty level; vertices at k+1 are collected on the
    // way in case that level is the next one
    int dmin;
    la = compact_active<BLOCK>(A, la, n, An, F0, D, k, sh, &dmin, &nf);
    int* t = A;
    A = An;
    An = t;
    if (la == 0) break;
    if (dmin != k + 1) nf = select_frontier<BLOCK>(A, la, n, F0, D, dmin, sh);
    k = dmin;
  }
  if (tid == 0) *gd.kmax = kmax;
  __syncthreads();
}

// ------------------------------------------------------------------ clustered form
namespace cg = cooperative_groups;

// Counters of a cluster, kept in its first CTA. Each phase (the work between
// two cluster barriers) accumulates into slot[phase % 3] -- [0] and [1]
// counts, [2] a minimum, [3] a maximum -- which every CTA reads after the
// barrier that ends the phase; the first CTA clears the slot of the next phase
// at the start of each phase (its last readers passed a barrier since).
struct ClusterCtl {
  int g;    // graph drawn for the cluster
  int bad;  // the graph failed a bounds check
  int slot[3][4];
};

template <int BLOCK, int C>
struct ClusterPeel {
  cg::cluster_group cl;
  ClusterCtl* lc;  // the first CTA's counters
  BatchShared<BLOCK>& sh;
  int* status;
  int r;       // this CTA's rank in the cluster
  int ph = 0;  // phase index (the same in every CTA)

  __device__ ClusterPeel(ClusterCtl* lead, BatchShared<BLOCK>& s, int* st)
      : cl(cg::this_cluster()), lc(lead), sh(s), status(st), r((int)cg::this_cluster().block_rank()) {}

  __device__ int* slot(int p) const { return lc->slot[p % 3]; }
  __device__ void clear(int p) const {
    int* x = slot(p);
    x[0] = 0;
    x[1] = 0;
    x[2] = INT_MAX;
    x[3] = 0;
  }
  __device__ bool first() const { return r == 0 && threadIdx.x == 0; }
  // ends a phase: this CTA's bounds-check failure goes to the cluster flag,
  // then the cluster barrier (release / acquire: the phase's stores, global
  // and distributed shared, are seen by every CTA after it)
  __device__ void next_phase() {
    __syncthreads();  // every thread's flag_bad of this phase is seen by thread 0
    if (threadIdx.x == 0 && sh.bad) atomicOr(&lc->bad, 1);
    cl.sync();
    ph++;
    if (first()) clear(ph + 1);
  }
  // this CTA's part [lo, hi) of a range of len entries
  __device__ long long part_lo(long long len) const { return len * r / C; }
  __device__ long long part_hi(long long len) const { return len * (r + 1) / C; }

  // entries of A with D == k go to F (count in this phase's slot[0])
  __device__ void select(const int* A, int la, int n, int* F, const DegStore& D, int k) {
    const int lo = (int)part_lo(la), hi = (int)part_hi(la);
    for (int base = lo; base < hi; base += BLOCK * kScanItems) {
      int v[kScanItems];
      unsigned take = 0;
#pragma unroll
      for (int q = 0; q < kScanItems; q++) {
        const int i = base + q * BLOCK + threadIdx.x;
        v[q] = -1;
        if (i < hi) {
          const int x = __ldcg(A + i);  // written by other CTAs of the cluster
          v[q] = (unsigned)x < (unsigned)n ? x : -1;
        }
      }
#pragma unroll
      for (int q = 0; q < kScanItems; q++)
        if (v[q] >= 0 && D.get(v[q]) == k) take |= 1u << q;
      int tot;
      const int pos = block_excl_scan(__popc(take), sh, &tot);
      if (threadIdx.x == 0) sh.base = tot ? atomicAdd(&slot(ph)[0], tot) : 0;
      __syncthreads();
      int p = sh.base + pos;
#pragma unroll
      for (int q = 0; q < kScanItems; q++)
        if ((take >> q) & 1u) F[p++] = v[q];
      __syncthreads();  // sh.base is reused by the next tile
    }
  }

  // entries of A with D > k survive into out (count slot[0], minimum slot[2]);
  // those at k + 1 also go to F (count slot[1])
  __device__ void compact(const int* A, int la, int n, int* out, int* F, const DegStore& D, int k) {
    const int lo = (int)part_lo(la), hi = (int)part_hi(la);
    int lmin = INT_MAX;
    for (int base = lo; base < hi; base += BLOCK * kScanItems) {
      int v[kScanItems];
      unsigned keep = 0, front = 0;
#pragma unroll
      for (int q = 0; q < kScanItems; q++) {
        const int i = base + q * BLOCK + threadIdx.x;
        v[q] = -1;
        if (i < hi) {
          const int x = __ldcg(A + i);
          v[q] = (unsigned)x < (unsigned)n ? x : -1;
        }
      }
#pragma unroll
      for (int q = 0; q < kScanItems; q++) {
        if (v[q] >= 0) {
          const int d = D.get(v[q]);
          if (d > k) {
            keep |= 1u << q;
            lmin = min(lmin, d);
            if (d == k + 1) front |= 1u << q;
          }
        }
      }
      int tot;
      const int pos = block_excl_scan(__popc(keep) | (__popc(front) << 16), sh, &tot);
      if (threadIdx.x == 0) {
        const int bk = (tot & 0xffff) ? atomicAdd(&slot(ph)[0], tot & 0xffff) : 0;
        const int bf = (tot >> 16) ? atomicAdd(&slot(ph)[1], tot >> 16) : 0;
        sh.base = bk;
        sh.cnt = bf;
      }
      __syncthreads();
      int pk = sh.base + (pos & 0xffff), pf = sh.cnt + (pos >> 16);
#pragma unroll
      for (int q = 0; q < kScanItems; q++) {
        if ((keep >> q) & 1u) out[pk++] = v[q];
        if ((front >> q) & 1u) F[pf++] = v[q];
      }
      __syncthreads();
    }
    const int m = block_min(lmin, sh);
    if (threadIdx.x == 0 && m != INT_MAX) atomicMin(&slot(ph)[2], m);
  }

  // Peels one graph with the whole cluster (Algorithm 1's levels and
  // subrounds, the online Peel of Algorithm 3, as peel_one_graph does in one CTA).
  __device__ void peel(const GraphDesc& gd) {
    const int tid = threadIdx.x, lane = tid & 31;
    if (first()) {
      lc->bad = 0;
      clear(0);
      clear(1);
      clear(2);
    }
    if (tid == 0) sh.bad = 0;
    ph = 0;
    cl.sync();
    const int n = (int)gd.n;
    const long long* O = gd.off;
    // phase: degrees (least and largest)
    int lmin = INT_MAX, lmax = 0;
    for (long long v = (long long)r * BLOCK + tid; v < n; v += (long long)C * BLOCK) {
      long long o0 = O[v], o1 = O[v + 1];
      if (o0 < 0 || o1 < o0 || o1 > gd.m || o1 - o0 >= n) {
        flag_bad(status, 1, v, &sh.bad);
        o1 = o0;
      }
      lmin = min(lmin, (int)(o1 - o0));
      lmax = max(lmax, (int)(o1 - o0));
    }
    lmin = block_min(lmin, sh);
    lmax = -block_min(-lmax, sh);
    if (tid == 0) {
      atomicMin(&slot(ph)[2], lmin);
      atomicMax(&slot(ph)[3], lmax);
    }
    next_phase();
    int k = slot(ph - 1)[2];
    const int dmax = slot(ph - 1)[3];
    if (lc->bad) {  // malformed offsets: leave this graph (its outputs are undefined)
      if (first()) *gd.kmax = -1;
      return;
    }
    const bool narrow = dmax < 65536;
    const DegStore D{gd.deg, false, narrow, l2_evict_last_policy()};
    // phase: initial induced degrees, the identity active list
    const int nw = narrow ? (n + 1) / 2 : n;
    for (long long i = (long long)r * BLOCK + tid; i < nw; i += (long long)C * BLOCK) {
      const int v0 = narrow ? 2 * (int)i : (int)i;
      const int d0 = (int)(O[v0 + 1] - O[v0]);
      const int d1 = narrow && v0 + 1 < n ? (int)(O[v0 + 2] - O[v0 + 1]) : 0;
      D.put_word((int)i, d0, d1);
    }
    for (long long v = (long long)r * BLOCK + tid; v < n; v += (long long)C * BLOCK) gd.A0[v] = (int)v;
    next_phase();
    int* A = gd.A0;
    int* An = gd.A1;
    int la = n, kmax = 0;
    select(A, la, n, gd.F0, D, k);
    next_phase();
    int nf = slot(ph - 1)[0];
    for (;;) {
      int* Fc = gd.F0;
      int* Fn = gd.F1;
      while (nf > 0) {
        for (long long i = (long long)r * BLOCK + tid; i < nf; i += (long long)C * BLOCK) {
          const int v = __ldcg(Fc + i);
          if ((unsigned)v < (unsigned)n) gd.core[v] = k;
          else flag_bad(status, 6, v, &sh.bad);
        }
        // a large frontier: the CTAs take whole chunks of BLOCK frontier
        // vertices in turn; a small one: every CTA walks every chunk and takes
        // its share of the chunk's arcs
        const bool whole = nf >= 2 * C * BLOCK;
        for (int c0 = whole ? r * BLOCK : 0; c0 < nf; c0 += whole ? C * BLOCK : BLOCK) {
          const int cnum = min(BLOCK, nf - c0);
          int len = 0;
          long long st = 0;
          if (tid < cnum) {
            const int v = __ldcg(Fc + c0 + tid);
            if ((unsigned)v < (unsigned)n) {
              st = O[v];
              const long long e = O[v + 1];
              if (st < 0 || e < st || e > gd.m || e - st >= n) flag_bad(status, 2, v, &sh.bad);
              else len = (int)(e - st);
            } else {
              flag_bad(status, 3, v, &sh.bad);
            }
          }
          int total;
          const int ex = block_excl_scan(len, sh, &total);
          sh.pre[tid] = ex;
          sh.start[tid] = st;
          __syncthreads();
          const int jlo = whole ? 0 : (int)part_lo(total), jhi = whole ? total : (int)part_hi(total);
          for (int j0 = jlo; j0 < jhi; j0 += BLOCK * kBatchIlp) {
            int u[kBatchIlp];
#pragma unroll
            for (int q = 0; q < kBatchIlp; q++) {
              const int j = j0 + q * BLOCK + tid;
              u[q] = -1;
              if (j < jhi) {
                int lo = 0, hi = cnum;
                while (lo < hi) {
                  const int mid = (lo + hi) >> 1;
                  if (sh.pre[mid] <= j) lo = mid + 1;
                  else hi = mid;
                }
                const int idx = lo - 1;
                const long long arc = idx >= 0 ? sh.start[idx] + (j - sh.pre[idx]) : -1;
                if (idx < 0 || arc < 0 || arc >= gd.m) {
                  flag_bad(status, 4, arc, &sh.bad);
                } else {
                  u[q] = ld_stream_s32(gd.adj + arc);
                  if ((unsigned)u[q] >= (unsigned)n) {
                    flag_bad(status, 5, u[q], &sh.bad);
                    u[q] = -1;
                  }
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kBatchIlp; q++) {
              // d~ lives in L2: the decrement goes unread (a vertex at or
              // below k never returns k + 1)
              const bool cross = u[q] >= 0 && D.dec(u[q]) == k + 1;
              const unsigned m = __ballot_sync(kFull, cross);
              if (m) {
                int base = 0;
                if (lane == __ffs(m) - 1) base = atomicAdd(&slot(ph)[0], __popc(m));
                base = __shfl_sync(kFull, base, __ffs(m) - 1);
                const int pos = base + __popc(m & lanemask_lt());
                if (cross) {
                  if (pos < n) Fn[pos] = u[q];
                  else flag_bad(status, 7, pos, &sh.bad);
                }
              }
            }
          }
          __syncthreads();  // sh.pre / sh.start are reused by the next chunk
        }
        next_phase();
        nf = slot(ph - 1)[0];
        if (nf > n) nf = 0;  // cannot happen: every vertex lands on k at most once per level
        if (lc->bad) {
          if (first()) *gd.kmax = -1;
          return;
        }
        int* t = Fc;
        Fc = Fn;
        Fn = t;
      }
      kmax = k;
      compact(A, la, n, An, gd.F0, D, k);
      next_phase();
      la = slot(ph - 1)[0];
      nf = slot(ph - 1)[1];
      const int dmin = slot(ph - 1)[2];
      int* t = A;
      A = An;
      An = t;
      if (la == 0) break;
      if (dmin != k + 1) {
        select(A, la, n, gd.F0, D, dmin);
        next_phase();
        nf = slot(ph - 1)[0];
      }
      k = dmin;
    }
    if (first()) *gd.kmax = kmax;
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, (BLOCK >= 1024 ? 1 : 2048 / BLOCK * 3 / 4)) batch_peel(BatchArgs a) {
  extern __shared__ int sdeg[];
  __shared__ BatchShared<BLOCK> sh;
  for (;;) {
    if (threadIdx.x == 0) sh.g = atomicAdd(a.next_graph, 1);
    __syncthreads();
    long long gi = sh.g;
    __syncthreads();
    if (gi >= a.G) break;
    long long g = a.order ? a.order[gi] : gi;
    if (g < 0 || g >= a.G) {  // the order is a permutation of [0, G); checked anyway
      if (threadIdx.x == 0) flag_bad(a.status, 8, g, &sh.bad);
      continue;
    }
    GraphDesc gd;
    const long long v0 = a.gv[g];
    gd.n = a.gv[g + 1] - v0;
    if (v0 < 0 || gd.n < 0 || v0 + gd.n > a.N) {  // graph outside the vertex range
      if (threadIdx.x == 0) {
        flag_bad(a.status, 9, g, &sh.bad);
        a.kmax[g] = -1;
      }
      continue;
    }
    gd.m = a.m;
    gd.off = a.off + v0;
    gd.adj = a.adj;
    gd.core = a.core + v0;
    gd.kmax = a.kmax + g;
    gd.deg = a.deg + v0;
    gd.A0 = a.A0 + v0;
    gd.A1 = a.A1 + v0;
    gd.F0 = a.F0 + v0;
    gd.F1 = a.F1 + v0;
    peel_one_graph<BLOCK>(gd, a.smem_deg_max, a.status, sdeg, sh);
  }
}

// The batched peel with clusters of C CTAs for the graphs of at least big_arcs
// arcs (see the file comment). A cluster draws graphs together while they are
// big; from the first graph below the threshold on, its CTAs draw one each.
template <int BLOCK, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(BLOCK, (BLOCK >= 1024 ? 1 : 2048 / BLOCK / 2))
    batch_peel_cl(BatchArgs a, long long big_arcs) {
  extern __shared__ int sdeg[];
  __shared__ BatchShared<BLOCK> sh;
  __shared__ ClusterCtl ctl;
  cg::cluster_group cl = cg::this_cluster();
  ClusterCtl* lc = cl.map_shared_rank(&ctl, 0);
  const bool lead = cl.block_rank() == 0;
  bool together = true;
  for (;;) {
    long long gi;
    if (together) {
      if (lead && threadIdx.x == 0) ctl.g = atomicAdd(a.next_graph, 1);
      cl.sync();
      gi = lc->g;
      cl.sync();  // every CTA has read the draw before the next one
    } else {
      if (threadIdx.x == 0) sh.g = atomicAdd(a.next_graph, 1);
      __syncthreads();
      gi = sh.g;
      __syncthreads();
    }
    if (gi >= a.G) break;
    const long long g = a.order ? a.order[gi] : gi;
    if (g < 0 || g >= a.G) {
      if (threadIdx.x == 0) flag_bad(a.status, 8, g, &sh.bad);
      continue;
    }
    GraphDesc gd;
    const long long v0 = a.gv[g];
    gd.n = a.gv[g + 1] - v0;
    if (v0 < 0 || gd.n < 0 || v0 + gd.n > a.N) {
      if (threadIdx.x == 0 && (!together || lead)) {
        flag_bad(a.status, 9, g, &sh.bad);
        a.kmax[g] = -1;
      }
      continue;
    }
    gd.m = a.m;
    gd.off = a.off + v0;
    gd.adj = a.adj;
    gd.core = a.core + v0;
    gd.kmax = a.kmax + g;
    gd.deg = a.deg + v0;
    gd.A0 = a.A0 + v0;
    gd.A1 = a.A1 + v0;
    gd.F0 = a.F0 + v0;
    gd.F1 = a.F1 + v0;
    if (together && gd.n > 0 && gd.n < INT_MAX && gd.off[gd.n] - gd.off[0] >= big_arcs) {
      ClusterPeel<BLOCK, C> cp(lc, sh, a.status);
      cp.peel(gd);
      continue;
    }
    if (together) {
      together = false;  // the first CTA peels this graph, the others draw their own
      if (!lead) continue;
    }
    peel_one_graph<BLOCK>(gd, a.smem_deg_max, a.status, sdeg, sh);
  }
}

// The same peel over graph descriptors held in a device table (graphs in
// separate allocations, as the server holds them). The launch lists the
// table slots to process; CTAs take them from a counter.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, (BLOCK >= 1024 ? 1 : 2048 / BLOCK / 2))
    desc_peel(const GraphDesc* table, SlotList list, int* next, int smem_deg_max, int* status) {
  extern __shared__ int sdeg[];
  __shared__ BatchShared<BLOCK> sh;
  for (;;) {
    if (threadIdx.x == 0) sh.g = atomicAdd(next, 1);
    __syncthreads();
    int gi = sh.g;
    __syncthreads();
    if (gi >= list.count) break;
    GraphDesc gd = table[list.slot[gi]];
    peel_one_graph<BLOCK>(gd, smem_deg_max, status, sdeg, sh);
  }
}

// The descriptor-driven peel with clusters of C CTAs for the graphs of at
// least big_arcs arcs (the launch lists the slots largest first).
template <int BLOCK, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(BLOCK, (BLOCK >= 1024 ? 1 : 2048 / BLOCK / 2))
    desc_peel_cl(const GraphDesc* table, SlotList list, int* next, int smem_deg_max, int* status,
                 long long big_arcs) {
  extern __shared__ int sdeg[];
  __shared__ BatchShared<BLOCK> sh;
  __shared__ ClusterCtl ctl;
  cg::cluster_group cl = cg::this_cluster();
  ClusterCtl* lc = cl.map_shared_rank(&ctl, 0);
  const bool lead = cl.block_rank() == 0;
  bool together = true;
  for (;;) {
    int gi;
    if (together) {
      if (lead && threadIdx.x == 0) ctl.g = atomicAdd(next, 1);
      cl.sync();
      gi = lc->g;
      cl.sync();  // every CTA has read the draw before the next one
    } else {
      if (threadIdx.x == 0) sh.g = atomicAdd(next, 1);
      __syncthreads();
      gi = sh.g;
      __syncthreads();
    }
    if (gi >= list.count) break;
    const GraphDesc gd = table[list.slot[gi]];
    if (together && gd.n > 0 && gd.n < INT_MAX && gd.off[gd.n] - gd.off[0] >= big_arcs) {
      ClusterPeel<BLOCK, C> cp(lc, sh, status);
      cp.peel(gd);
      continue;
    }
    if (together) {
      together = false;  // the first CTA peels this graph, the others draw their own
      if (!lead) continue;
    }
    peel_one_graph<BLOCK>(gd, smem_deg_max, status, sdeg, sh);
  }
}

// Order of graphs: descending number of arcs (ties by index). One CTA sorts
// keys (~arcs << 24 | g) bitonically in shared memory; batches larger than
// kMaxSortGraphs keep their given order.
__global__ void __launch_bounds__(1024) batch_order(const long long* gv, const long long* off,
                                                    long long G, int* order) {
  extern __shared__ unsigned long long key[];
  int P = 1;
  while (P < G) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < G) {
      unsigned long long arcs = (unsigned long long)(off[gv[i + 1]] - off[gv[i]]);
      if (arcs > 0xffffffffffull) arcs = 0xffffffffffull;
      key[i] = ((0xffffffffffull - arcs) << 24) | (unsigned long long)i;
    } else {
      key[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          unsigned long long x = key[i], y = key[j];
          if ((x > y) == up) {
            key[i] = y;
            key[j] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < G; i += blockDim.x) order[i] = (int)(key[i] & 0xffffffull);
}

// ------------------------------------------------------------------ host side
namespace {
template <int BLOCK>
cudaError_t launch_block(const BatchArgs& a, int grid, size_t smem, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(batch_peel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  batch_peel<BLOCK><<<grid, BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}
template <int BLOCK, int C>
cudaError_t launch_cluster(const BatchArgs& a, int grid, size_t smem, long long big_arcs, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(batch_peel_cl<BLOCK, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  grid = grid / C * C;
  if (grid < C) grid = C;
  batch_peel_cl<BLOCK, C><<<grid, BLOCK, smem, stream>>>(a, big_arcs);
  return cudaGetLastError();
}
template <int BLOCK>
int occupancy_block(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(batch_peel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_peel<BLOCK>, BLOCK, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}
}  // namespace

namespace {
template <int C>
cudaError_t desc_launch_cl(const GraphDesc* table, const SlotList& list, int* next, int smem_deg_max, int* status,
                           int grid, size_t smem, long long big_arcs, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(desc_peel_cl<1024, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  grid = std::max(C, grid / C * C);
  desc_peel_cl<1024, C><<<grid, 1024, smem, stream>>>(table, list, next, smem_deg_max, status, big_arcs);
  return cudaGetLastError();
}
}  // namespace

cudaError_t desc_launch(const GraphDesc* table, const SlotList& list, int* next, int smem_deg_max,
                        int* status, int grid, size_t smem, cudaStream_t stream, int cluster, long long big_arcs) {
  switch (cluster) {
    case 2: return desc_launch_cl<2>(table, list, next, smem_deg_max, status, grid, smem, big_arcs, stream);
    case 4: return desc_launch_cl<4>(table, list, next, smem_deg_max, status, grid, smem, big_arcs, stream);
    case 8: return desc_launch_cl<8>(table, list, next, smem_deg_max, status, grid, smem, big_arcs, stream);
  }
  cudaError_t e = cudaFuncSetAttribute(desc_peel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  desc_peel<1024><<<grid, 1024, smem, stream>>>(table, list, next, smem_deg_max, status);
  return cudaGetLastError();
}

size_t desc_static_smem() { return sizeof(BatchShared<1024>); }

__global__ void batch_single_gv_kernel(long long* gv, long long n) {
  gv[0] = 0;
  gv[1] = n;
}

cudaError_t batch_single_gv(long long* gv, long long n, cudaStream_t stream) {
  batch_single_gv_kernel<<<1, 1, 0, stream>>>(gv, n);
  return cudaGetLastError();
}

int batch_occupancy(int block, size_t smem) {
  switch (block) {
    case 256: return occupancy_block<256>(smem);
    case 512: return occupancy_block<512>(smem);
    case 1024: return occupancy_block<1024>(smem);
  }
  return 0;
}

size_t batch_static_smem(int block) {
  switch (block) {
    case 256: return sizeof(BatchShared<256>);
    case 512: return sizeof(BatchShared<512>);
    case 1024: return sizeof(BatchShared<1024>);
  }
  return 0;
}

cudaError_t batch_launch(const BatchArgs& a, int block, int grid, size_t smem, bool sort_graphs,
                         cudaStream_t stream, int cluster, long long big_arcs) {
  if (sort_graphs && a.order) {
    int P = 1;
    while (P < a.G) P <<= 1;
    size_t ss = sizeof(unsigned long long) * (size_t)P;
    cudaError_t e = cudaFuncSetAttribute(batch_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    if (e != cudaSuccess) return e;
    batch_order<<<1, 1024, ss, stream>>>(a.gv, a.off, a.G, (int*)a.order);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (cluster > 1) {
    const int key = block * 16 + cluster;
    switch (key) {
      case 512 * 16 + 2: return launch_cluster<512, 2>(a, grid, smem, big_arcs, stream);
      case 512 * 16 + 4: return launch_cluster<512, 4>(a, grid, smem, big_arcs, stream);
      case 512 * 16 + 8: return launch_cluster<512, 8>(a, grid, smem, big_arcs, stream);
      case 1024 * 16 + 2: return launch_cluster<1024, 2>(a, grid, smem, big_arcs, stream);
      case 1024 * 16 + 4: return launch_cluster<1024, 4>(a, grid, smem, big_arcs, stream);
      case 1024 * 16 + 8: return launch_cluster<1024, 8>(a, grid, smem, big_arcs, stream);
    }
    return cudaErrorInvalidValue;
  }
  switch (block) {
    case 256: return launch_block<256>(a, grid, smem, stream);
    case 512: return launch_block<512>(a, grid, smem, stream);
    case 1024: return launch_block<1024>(a, grid, smem, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace kc
