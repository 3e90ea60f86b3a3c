// Single-graph k-core peel, bulk-synchronous mode: one persistent cooperative
// kernel whose phases are separated by a hand-written, bounded grid barrier.
//
// Algorithm 1's rounds with the online Peel of Algorithm 3, phase by phase:
//   scan   - the active list is compacted to the vertices above the level
//            being tried (k = previous level + 1) while the vertices sitting
//            exactly at k are appended to the work queue as slices of at most
//            `slice` arcs and get coreness k (frontier extraction and active-set
//            refine, fused; Theorem 1 bounds the summed list lengths). The
//            minimum induced degree of the kept vertices rides along: if level
//            k is empty, it is the next non-empty level and a second scan
//            collects its vertices.
//   pass   - one subround over the queue range appended before it: each warp
//            takes its own share of the items, 32 at a time, and processes
//            their arcs edge-balanced. A decrement of a neighbour above k that
//            returns k+1 is the crossing of Algorithm 3: the neighbour gets coreness k and is processed by
//            the same warp in the same pass if its list fits one slice and the
//            warp's local queue has room (the local FIFO of vertical
//            granularity control, Sec. 4.2); otherwise its slices go to the
//            queue for the next pass. The level ends with a pass that appends
//            nothing.
// The queue range of a pass is fixed while it runs, so it is split into
// static per-warp shares (no claim traffic), pushes need no fences and the
// pass ends at the barrier. A queue item is an arc range (first arc,
// length), so processing it needs no offset lookup. Each phase counts its own
// appends, which land after everything appended before the phase, so the next
// range is known to every CTA from the barrier word that ends the phase (it
// carries the appends with the arrivals). Every vertex is appended at
// most once over the whole run, so the queue never wraps. A warp runs at most
// `local_batches` batches from its local queue per chunk it takes and then
// moves the rest to the queue: a large cascade is shared by all warps in the
// next pass instead of being walked by the warp that started it. Heavy
// subrounds may instead count their decrements and apply them in a second
// phase (Algorithm 2's batch update); the offline peel, the level window,
// sampling and warp aggregation are variants compiled apart (see the kernel).
// Every wait is bounded by the handle's time limit (KCORE_ERR_TIMEOUT).
#include <climits>
#include <type_traits>

#include "kcore_device.cuh"
#include "kcore_peel.h"

namespace kc {

namespace {

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / kWarp;
constexpr int kTile = 8;   // active-list entries per thread per scan tile
constexpr int kExpand = 4; // staged frontier vertices per thread per expansion round
constexpr int kIlp = 8;    // arcs per lane in flight
constexpr int kTake = 32;  // queue items per chunk of a warp's share
constexpr int kLenShift = 40;  // item = first arc | length << 40
constexpr unsigned long long kArcMask = (1ull << kLenShift) - 1;
// barrier word: arrivals in bits 0..30, the phase's queue appends in bits
// 31..62 (every append is counted there too, so a pass's range is known from
// the word that ends the wait), bit 63: a status was raised
constexpr int kAppShift = 31;
constexpr unsigned long long kArrMask = (1ull << kAppShift) - 1;
constexpr unsigned long long kAppMask = (1ull << 32) - 1;
constexpr unsigned long long kAbort = 1ull << 63;

// queue items the CTA appended in the current phase (added to its arrival)
__shared__ unsigned long long s_app;
// a thread of this CTA raised a status (ends a tail-mode phase, which has no
// grid barrier to carry the abort bit)
__shared__ int s_abort;

struct Shared {
  int excl[kWarps][kWarp];
  long long a0[kWarps][kWarp];
  union {
    unsigned long long lq[kWarps][kLocalQueueMax];  // passes: the warps' local queues
    int stage[kBlock * kTile];                      // scans (local queues are empty): frontier ids
  };
  int lqn[kWarps];
  int part_i[kWarps];
  int total_i;
  unsigned long long base_a, base_q;
  int red_min[kWarps];
  int red_cnt[kWarps];
  unsigned long long tr_arcs[kWarps], tr_decs[kWarps];  // trace only
  unsigned ncross[kWarps];                               // k'-core query: crossings
  int flag;
  long long trec;            // per-phase trace: records written (CTA 0)
  unsigned long long tarcs;  // per-phase trace: arcs counted at the last record
  // the finished phase's counters, read once per CTA by grid_barrier (every
  // thread loading them would queue thousands of loads on one L2 line)
  struct {
    unsigned long long tail, head, found, alen, rcount, rqtail;
    int minkey, miss;
  } po;
  RoundRec tring[kPhaseRing];  // tail mode: the phases' records, in shared memory
  long long ho[kHandoff];      // a parked CTA: the loop state CTA 0 handed over
  // per-warp counters (lane 0): queue items and local-queue items processed,
  // local batches run (the heartbeat ticks every 64)
  long long w_items[kWarps], w_local[kWarps];
  unsigned w_lb[kWarps];
  // counters and level timeline kept by CTA 0's thread 0 alone (registers
  // held across the level loop make the hot loops spill)
  struct {
    long long levels, empty, scanned, passes, la_scanned, nscan, level_passes;
    unsigned long long level_qb, arcs0, decs0, nfound, t_start, t_scan;
    int kmax, rebuild;
  } ld;
  int sphase;         // tail mode: tail phases run (CTA 0)
  unsigned tail_gen;  // tail episodes begun (thread 0 of every CTA)
};

// Sampling keeps the vertex of each local-queue entry beside it (a spilled
// entry's vertex is traversed a pass later, which its stamp must say) and the
// warps' head counts.
struct SharedS : Shared {
  int lqv[kWarps][kLocalQueueMax];
  unsigned long long heads[kWarps];
};
template <bool kSample>
using ShT = std::conditional_t<kSample, SharedS, Shared>;

// Records the first error and makes every CTA leave at its next barrier (or,
// parked during a tail episode, at once).
__device__ __forceinline__ void raise_status(const PeelArgs& a, int code) {
  atomicCAS(&a.ctl->status, 0, code);
  for (int i = 0; i < 3; i++) atomicOr(&a.ctl->bar_ring[i].v, kAbort);
  atomicOr(&a.ctl->tail_word, kAbort);
  s_abort = 1;
}

__device__ __forceinline__ unsigned long long make_item(long long a0, long long len) {
  return (unsigned long long)a0 | ((unsigned long long)len << kLenShift);
}

// Writes each lane's arc range [e0, e1), cut in `cnt` slices, to the queue
// from slot p on. A lane with a few slices writes its own; the slices of a
// long range (a hub) are written by the whole warp, so one lane never stores
// thousands of items alone. Warp-collective.
__device__ __forceinline__ void write_slices(const PeelArgs& a, long long e0, long long e1, int cnt,
                                             unsigned long long p, int lane) {
  constexpr int kOwn = 4;
  if (cnt <= kOwn)
    for (int i = 0; i < cnt; i++) {
      const long long s0 = e0 + (long long)i * a.slice;
      a.Q[p + i] = make_item(s0, min((long long)a.slice, e1 - s0));
    }
  for (unsigned big = __ballot_sync(kFull, cnt > kOwn); big; big &= big - 1) {
    const int L = __ffs(big) - 1;
    const long long b0 = __shfl_sync(kFull, e0, L), b1 = __shfl_sync(kFull, e1, L);
    const unsigned long long bp = __shfl_sync(kFull, p, L);
    const int bc = __shfl_sync(kFull, cnt, L);
    for (int i = lane; i < bc; i += kWarp) {
      const long long s0 = b0 + (long long)i * a.slice;
      a.Q[bp + i] = make_item(s0, min((long long)a.slice, b1 - s0));
    }
  }
}

// ---- sampling (Sec. 4.1) ------------------------------------------------
// First output word of Philox4x32-10 (Salmon et al., SC 2011) for counter
// (j, 0) and key `seed`: the coin of arc j.
__device__ __forceinline__ unsigned philox_coin(unsigned long long j, unsigned long long seed) {
  unsigned c0 = (unsigned)j, c1 = (unsigned)(j >> 32), c2 = 0u, c3 = 0u;
  unsigned k0 = (unsigned)seed, k1 = (unsigned)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return c0;
}

// Sample rate mu / ((1 - r) D), r = 1/10: a head is a coin x (uniform on
// 32 bits) below floor(2^32 rate), i.e. D (x + 1) <= floor(10 mu 2^32 / 9)
// = a.coin_lim (exact in integers).
__device__ __forceinline__ bool coin_head(unsigned x, int D, unsigned long long lim) {
  return (unsigned long long)D * ((unsigned long long)x + 1ull) <= lim;
}

// Error(v, k) of Algorithm 5 holds (v may stay in sample mode through level
// k): D r > k and cnt < rate (D - k) / 4, i.e. 18 D cnt < 5 mu (D - k).
__device__ __forceinline__ bool sample_safe(int D, int cnt, int k, int mu) {
  return (long long)D > 10ll * k && 18ll * D * cnt < 5ll * mu * ((long long)D - k);
}

// The first level above which sample_safe fails for this (D, cnt): an empty
// level skipped by the scan's minimum must not pass it.
__device__ __forceinline__ int sample_key(int D, int cnt, int mu) {
  const long long k1 = ((long long)D + 9) / 10;
  long long k2 = (long long)D - (18ll * D * cnt) / (5ll * mu);
  if (k2 < 0) k2 = 0;
  return (int)(k1 < k2 ? k1 : k2);
}

// Appends the flagged lanes' vertices to the recount list and their adjacency
// lists, cut in slices of a.rslice arcs, to the recount queue (counts in
// R->rcount and R->rqtail). Warp-collective.
__device__ void append_recount(const PeelArgs& a, RoundRec* R, bool flag, int v, int lane) {
  const unsigned fm = __ballot_sync(kFull, flag);
  if (!fm) return;
  long long e0 = 0, e1 = 0;
  int nsl = 0;
  if (flag) {
    e0 = a.off[v];
    e1 = a.off[v + 1];
    nsl = (int)((e1 - e0 + a.rslice - 1) / a.rslice);
  }
  unsigned long long vb = 0;
  if (lane == 0) vb = atomicAdd(&R->rcount, (unsigned long long)__popc(fm));
  vb = __shfl_sync(kFull, vb, 0);
  const unsigned long long pv = vb + __popc(fm & lanemask_lt());
  if (flag) {
    if (pv < (unsigned long long)a.n) a.rlist[pv] = v;
    else raise_status(a, ST_CAPACITY);
  }
  const int incl = warp_incl_scan(nsl, lane);
  const int tot = __shfl_sync(kFull, incl, 31);
  unsigned long long qb = 0;
  if (lane == 31 && tot) qb = atomicAdd(&R->rqtail, (unsigned long long)tot);
  qb = __shfl_sync(kFull, qb, 31);
  if (qb + (unsigned long long)tot > (unsigned long long)a.rqcap) {
    if (lane == 0 && tot) raise_status(a, ST_CAPACITY);
    return;
  }
  unsigned long long p = qb + (unsigned long long)(incl - nsl);
  for (long long s0 = e0; s0 < e1; s0 += a.rslice, p++) {
    a.RQ[p] = make_item(s0, min((long long)a.rslice, e1 - s0));
    a.RQv[p] = v;
  }
}

// Grid barrier g on word g % 3 (zeroed by CTA 0 during phase g - 1, which
// every CTA finishes polling before CTA 0 can reach phase g + 2): each CTA adds
// one arrival plus its phase's queue appends with a release add; the phase is
// complete when gridDim.x arrivals are counted, and the acquire load that sees
// them makes every CTA's writes of the phase visible and gives the phase's
// appends (sh.po.tail) without another read. Waiters give up after timeout_ns
// without progress (a warp running a long local chain ticks ctl->progress).
// Returns false when a status was raised before the barrier completed, or
// when the wait gave up. With R, thread 0 then also reads R's other counters
// (and the sampling miss flag) into sh.po for the whole CTA.
__device__ bool grid_barrier(const PeelArgs& a, Shared& sh, unsigned long long& gen,
                             const RoundRec* R = nullptr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long* w = &a.ctl->bar_ring[gen % 3].v;
    const unsigned long long add = 1ull + (s_app << kAppShift);
    s_app = 0;
    // the CTA barrier above orders the CTA's writes before this release
    if (!(a.inject_stall && blockIdx.x == 0 && gen == 0))
      asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(w), "l"(add) : "memory");
    uint64_t t0 = 0;
    unsigned long long pg = 0;
    for (unsigned spins = 0;; spins++) {
      const unsigned long long v = ld_acquire_u64(w);
      if (v & kAbort) {
        ok = 0;
        break;
      }
      if ((v & kArrMask) >= gridDim.x) {
        sh.po.tail = (v >> kAppShift) & kAppMask;
        break;
      }
      if ((spins & 31) == 0) {
        const uint64_t now = globaltimer_ns();
        const unsigned long long p2 = ld_relaxed_u64(&a.ctl->progress);
        if (spins == 0 || p2 != pg) {
          pg = p2;
          t0 = now;
        } else if (now - t0 > a.timeout_ns) {
          raise_status(a, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
      __nanosleep(a.poll_sleep_ns);
    }
    sh.flag = ok;
    if (ok && R) {
      sh.po.head = ld_relaxed_u64(&R->head);
      sh.po.found = ld_relaxed_u64(&R->found);
      sh.po.alen = ld_relaxed_u64(&R->alen);
      sh.po.rcount = ld_relaxed_u64(&R->rcount);
      sh.po.rqtail = ld_relaxed_u64(&R->rqtail);
      sh.po.minkey = ld_relaxed_s32(&R->minkey);
      sh.po.miss = ld_relaxed_s32(&a.ctl->s_miss);
    }
  }
  __syncthreads();
  gen++;  // every thread: the barrier count also indexes the phase records
  return sh.flag != 0;
}

struct ScanOut {
  unsigned long long found;
  int dmin;
};

// Block-wide exclusive prefix sum of x; *total receives the block's sum.
// Ends with every thread past the barrier that published the partial sums.
__device__ __forceinline__ int block_excl_scan(Shared& sh, int x, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int incl = warp_incl_scan(x, lane);
  if (lane == 31) sh.part_i[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int y = lane < kWarps ? sh.part_i[lane] : 0;
    const int yi = warp_incl_scan(y, lane);
    if (lane < kWarps) sh.part_i[lane] = yi - y;
    if (lane == kWarps - 1) sh.total_i = yi;
  }
  __syncthreads();
  *total = sh.total_i;
  return sh.part_i[warp] + incl - x;
}

// Scan of active-list entries [lo, hi) by one CTA: entries with d~ > keep_above
// go to Aout (their minimum d~ is returned), entries with d~ == take_at get
// coreness take_at and their slices are appended to the queue after position
// qbase (count in R->tail). With Ain == nullptr the list is 0..n-1 and d~ is
// initialised from the offsets. A tile is read in one step (list entries,
// then their d~: kTile independent loads per thread each), its frontier
// vertices are staged in shared memory and expanded into slices in a second
// step, so the offsets of only those vertices are read.
//
// With sampling (kSample): the first scan runs InitSampler(v, 0) on every
// vertex (and clears its sampling state); a later scan validates every vertex
// in sample mode at level take_at: it is kept, and either contributes the
// first level its validation could fail at to the minimum, or, failing
// Error(v, k), goes to the recount list. Taken vertices get stamp stamp_val.
template <bool kSample = false>
__device__ ScanOut scan_range(const PeelArgs& a, Shared& sh, RoundRec* R, unsigned long long qbase,
                              const int* Ain, int* Aout, long long lo, long long hi, int keep_above,
                              int take_at, bool take_le = false, int take_val = -1, int keep_val = -1,
                              int* Aover = nullptr, int over_from = INT_MAX, int stamp_val = 0) {
  // Aover: kept entries with d~ >= over_from go there instead of Aout (the
  // overflow list of a window rebuild; count in R->head)
  // take_le: take every entry with d~ <= take_at (k'-core query); take_val /
  // keep_val: the value written to core[] for taken / kept entries (-1: the
  // level take_at for taken ones, nothing for kept ones)
  if (take_val < 0) take_val = take_at;
  const int tid = threadIdx.x;
  unsigned long long found = 0;  // staged frontier vertices (block-uniform)
  int direct = 0;                // frontier vertices without arcs (this thread)
  int nsampled = 0;              // first scan with sampling: vertices put in sample mode
  int dmin = INT_MAX;
  for (long long tile = lo; tile < hi; tile += (long long)kBlock * kTile) {
    int v[kTile];
    unsigned keep = 0, take = 0, over = 0, rec = 0;
#pragma unroll
    for (int q = 0; q < kTile; q++) {
      const long long i = tile + (long long)q * kBlock + tid;
      v[q] = i < hi ? (Ain ? ld_once_s32(Ain + i, l2_evict_first_policy()) : (int)i) : -1;
    }
#pragma unroll
    for (int q = 0; q < kTile; q++) {
      const int x = v[q];
      if (x < 0 && tile + (long long)q * kBlock + tid >= hi) continue;
      if ((unsigned)x >= (unsigned)a.n) {
        raise_status(a, ST_NOT_SIMPLE);
        v[q] = -1;
        continue;
      }
      int d;
      if (!Ain) {
        const long long e0 = a.off[x], e1 = a.off[x + 1];
        if (e0 < 0 || e1 < e0 || e1 > a.m || e1 - e0 >= a.n) {
          raise_status(a, ST_NOT_SIMPLE);  // malformed offsets: no arc of x is ever read
          d = -1;
        } else {
          d = (int)(e1 - e0);
        }
        a.deg[x] = d < 0 ? 0 : d;
        if (d < 0) {
          // a malformed vertex is neither kept nor expanded; it takes level 0
          a.core[x] = 0;
          v[q] = -1;
          continue;
        }
        if constexpr (kSample) {
          a.stamp[x] = INT_MAX;
          a.scnt[x] = 0;
          a.racc[x] = 0;
          a.rst[x] = 0;
          if (d > 0 && (long long)d > a.sthreshold) {  // InitSampler(v, 0)
            a.deg[x] = -1 - d;
            nsampled++;
            keep |= 1u << q;
            dmin = min(dmin, sample_key(d, 0, a.mu));
            continue;
          }
        }
      } else {
        d = __ldcg(a.deg + x);
        if constexpr (kSample) {
          if (d < 0) {  // in sample mode: validate at level take_at
            const int D = -1 - d, cnt = __ldcg(a.scnt + x);
            keep |= 1u << q;
            if (sample_safe(D, cnt, take_at, a.mu)) dmin = min(dmin, sample_key(D, cnt, a.mu));
            else rec |= 1u << q;
            continue;
          }
        }
      }
      if (d > keep_above) {
        if (d >= over_from) over |= 1u << q;
        else keep |= 1u << q;
        dmin = min(dmin, d);
        if (keep_val >= 0) a.core[x] = keep_val;
      }
      if (take_le ? d <= take_at : d == take_at) {
        if (!Ain && d == 0) {
          a.core[x] = take_val;  // first scan: no arcs, nothing to expand
          direct++;
        } else {
          take |= 1u << q;
        }
      }
    }
    // block-wide offsets of (kept, taken): kept entries go to Aout after one
    // atomic per tile, taken ones to the shared-memory stage
    int tot;
    const int ex = block_excl_scan(sh, (__popc(take) << 16) | __popc(keep), &tot);
    if (tid == 0) sh.base_a = (tot & 0xffff) ? atomicAdd(&R->alen, (unsigned long long)(tot & 0xffff)) : 0;
    __syncthreads();
    unsigned long long pa = sh.base_a + (ex & 0xffff);
    int ps = ex >> 16;
#pragma unroll
    for (int q = 0; q < kTile; q++) {
      if ((keep >> q) & 1u) st_once_s32(Aout + pa++, v[q], l2_evict_first_policy());
      if ((take >> q) & 1u) sh.stage[ps++] = v[q];
    }
    if (Aover) {
      int otot;
      const int oex = block_excl_scan(sh, __popc(over), &otot);
      if (tid == 0) sh.base_q = otot ? atomicAdd(&R->head, (unsigned long long)otot) : 0;
      __syncthreads();
      unsigned long long po = sh.base_q + oex;
#pragma unroll
      for (int q = 0; q < kTile; q++)
        if ((over >> q) & 1u) Aover[po++] = v[q];
    }
    __syncthreads();
    const int ntaken = tot >> 16;
    found += ntaken;
    // expand the staged frontier vertices into slices, kExpand per thread per round
    for (int base = 0; base < ntaken; base += kBlock * kExpand) {
      long long e0[kExpand], e1[kExpand];
      int nsl = 0;
#pragma unroll
      for (int k = 0; k < kExpand; k++) {
        const int i = base + k * kBlock + tid;
        e0[k] = e1[k] = 0;
        if (i < ntaken) {
          const int x = sh.stage[i];
          e0[k] = __ldcs(a.off + x);
          e1[k] = __ldcs(a.off + x + 1);
          a.core[x] = take_val;
          if constexpr (kSample) a.stamp[x] = stamp_val;
        }
      }
#pragma unroll
      for (int k = 0; k < kExpand; k++) nsl += (int)((e1[k] - e0[k] + a.slice - 1) / a.slice);
      int ntot;
      const int exs = block_excl_scan(sh, nsl, &ntot);
      if (tid == 0) {
        unsigned long long bq = qbase + (ntot ? atomicAdd(&R->tail, (unsigned long long)ntot) : 0);
        s_app += (unsigned long long)ntot;
        if (bq + (unsigned long long)ntot > (unsigned long long)a.qcap) {
          raise_status(a, ST_CAPACITY);
          bq = ~0ull;
        }
        sh.base_q = bq;
      }
      __syncthreads();
      if (sh.base_q != ~0ull) {
        unsigned long long pq = sh.base_q + exs;
#pragma unroll
        for (int k = 0; k < kExpand; k++)
          for (long long s0 = e0[k]; s0 < e1[k]; s0 += a.slice)
            a.Q[pq++] = make_item(s0, min((long long)a.slice, e1[k] - s0));
      }
      __syncthreads();
    }
    if constexpr (kSample) {
      // vertices that failed validation: recount before the level's passes
      const int ln = tid & 31;
#pragma unroll
      for (int q = 0; q < kTile; q++) append_recount(a, R, (rec >> q) & 1u, v[q], ln);
    }
  }
  const int lane = tid & 31, warp = tid >> 5;
  if constexpr (kSample) {
    const int sw = warp_sum(nsampled);
    if (lane == 0 && sw) atomicAdd((unsigned long long*)&a.ctl->s_sampled, (unsigned long long)sw);
  }
  const int mw = warp_min(dmin);
  const int dw = warp_sum(direct);
  if (lane == 0) {
    sh.red_min[warp] = mw;
    sh.red_cnt[warp] = dw;
  }
  __syncthreads();
  ScanOut o{found, INT_MAX};
  if (tid == 0)
    for (int w = 0; w < kWarps; w++) {
      o.dmin = min(o.dmin, sh.red_min[w]);
      o.found += (unsigned long long)sh.red_cnt[w];
    }
  return o;
}

// Context of one pass: where its appends go and its level.
struct PassCtx {
  RoundRec* R;              // R->tail counts this phase's appends
  unsigned long long qbase; // appends start here
  int t;
  int val;                  // written to core[] of a vertex that crosses (t, or 0 in a k'-core query)
  bool precheck;            // long pass: read d~ before decrementing (see process_items)
  int win_hi;               // level window's end (a decrement returning it appends the vertex), or -1
  int* near;                // the active list, appended from near_base on (count in R->found)
  unsigned long long near_base;
  int pass;                 // sampling: index of the running pass (stamps)
};

// Appends `cnt` items per lane (lane-owned arc ranges [e0, e1) cut in
// slices) to the queue.
template <bool kCoop = false>
__device__ __forceinline__ void append_ranges(const PeelArgs& a, const PassCtx& pc, int cnt, long long e0,
                                              long long e1, int lane) {
  const int incl = warp_incl_scan(cnt, lane);
  const int tot = __shfl_sync(kFull, incl, 31);
  if (tot == 0) return;
  unsigned long long base = 0;
  if (lane == 31) {
    base = pc.qbase + atomicAdd(&pc.R->tail, (unsigned long long)tot);
    atomicAdd(&s_app, (unsigned long long)tot);
  }
  base = __shfl_sync(kFull, base, 31);
  if (base + (unsigned long long)tot > (unsigned long long)a.qcap) {
    if (lane == 0) raise_status(a, ST_CAPACITY);
    return;
  }
  unsigned long long p = base + (unsigned long long)(incl - cnt);
  if constexpr (kCoop) {
    write_slices(a, e0, e1, cnt, p, lane);
  } else {
    for (long long s0 = e0; s0 < e1 && cnt > 0; s0 += a.slice) a.Q[p++] = make_item(s0, min((long long)a.slice, e1 - s0));
  }
}

// The vertices u of the lanes with `flag` crossed to the current level (their
// coreness is set): one-slice lists go to the warp's local queue while it has
// room, the rest go to the queue as slices for the next pass.
template <bool kSample = false>
__device__ __forceinline__ void push_crossed(const PeelArgs& a, ShT<kSample>& sh, const PassCtx& pc, bool flag,
                                             int u, int warp, int lane) {
  long long e0 = 0, e1 = 0;
  int nsl = 0;
  if (flag) {
    e0 = __ldcs(a.off + u);
    e1 = __ldcs(a.off + u + 1);
    nsl = (int)((e1 - e0 + a.slice - 1) / a.slice);
    // its first adjacency line is read next, here or by another warp
    if (e1 > e0) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.adj + e0));
  }
  const bool one = flag && nsl == 1;
  const unsigned om = __ballot_sync(kFull, one);
  const int lqn = sh.lqn[warp];
  const int room = max(a.lq_cap - lqn, 0);
  const int rank = __popc(om & lanemask_lt());
  const bool local = one && rank < room;
  if (local) sh.lq[warp][lqn + rank] = make_item(e0, e1 - e0);
  if constexpr (kSample) {
    // a local entry is traversed in this pass, a queued one in the next
    if (local) sh.lqv[warp][lqn + rank] = u;
    if (flag) a.stamp[u] = local ? pc.pass : pc.pass + 1;
  }
  __syncwarp();
  if (lane == 0) sh.lqn[warp] = lqn + min(__popc(om), room);
  __syncwarp();
  append_ranges(a, pc, (flag && !local) ? nsl : 0, e0, e1, lane);
}

// Arcs of the items held by lanes < c, spread evenly over the warp.
// With sampling (kSample), d~ is always read first: a neighbour in sample
// mode (d~ < 0) is not decremented but tosses the arc's coin, and its mu-th
// head puts it in the counting bag (the recount list of the next recount).
template <bool kWin, bool kSample = false, bool kCombine = false>
__device__ void process_items(const PeelArgs& a, ShT<kSample>& sh, const PassCtx& pc, unsigned long long item,
                              int c, int warp, int lane) {
  const int t = pc.t;
  const long long a0 = lane < c ? (long long)(item & kArcMask) : 0;
  const int len = lane < c ? (int)(item >> kLenShift) : 0;
  const int incl = warp_incl_scan(len, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  sh.excl[warp][lane] = incl - len;
  sh.a0[warp][lane] = a0;
  __syncwarp();
  const int* excl = sh.excl[warp];
  int ndec = 0;
  unsigned nheads = 0;
  for (int base = 0; base < total; base += kWarp * kIlp) {
    int u[kIlp];
    int j = base + lane;
    int lo = 0, hi = c;  // last item whose first arc is <= j
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (excl[mid] <= j) lo = mid + 1;
      else hi = mid;
    }
    int idx = lo > 0 ? lo - 1 : 0;
    const int idx0 = idx;
#pragma unroll
    for (int q = 0; q < kIlp; q++, j += kWarp) {
      u[q] = -1;
      if (j < total) {
        while (idx + 1 < c && excl[idx + 1] <= j) idx++;
        const long long arc = sh.a0[warp][idx] + (j - excl[idx]);
        const int x = arc < a.m ? ld_stream_s32(a.adj + arc) : -1;
        if ((unsigned)x < (unsigned)a.n) u[q] = x;
        else raise_status(a, ST_NOT_SIMPLE);
      }
    }
    // Reading d~ first spares the atomics on neighbours at or below the
    // level, at the price of one more dependent access per iteration. It pays
    // in a long pass, where warps have enough work to hide latency and
    // atomic throughput counts (pc.precheck), and only for batches of more
    // than one iteration; otherwise the warp decrements unconditionally. That
    // is safe, as a neighbour at or below k never returns k + 1 and its d~ is
    // not read again.
    int dq[kIlp];
    if (kSample || (pc.precheck && total > kWarp * kIlp)) {
#pragma unroll
      for (int q = 0; q < kIlp; q++) dq[q] = u[q] >= 0 ? __ldcg(a.deg + u[q]) : INT_MIN;
    } else {
#pragma unroll
      for (int q = 0; q < kIlp; q++) dq[q] = u[q] >= 0 ? INT_MAX : INT_MIN;
    }
    unsigned cross = 0, enter = 0, bag = 0;
    if constexpr (kSample) {
      int ix = idx0;
#pragma unroll
      for (int q = 0; q < kIlp; q++)
        if (u[q] >= 0 && dq[q] < 0) {
          // sample mode: one coin of probability mu / ((1 - r) D) per arc,
          // drawn from the arc's index
          const int jq = base + lane + q * kWarp;
          while (ix + 1 < c && excl[ix + 1] <= jq) ix++;
          const long long arc = sh.a0[warp][ix] + (jq - excl[ix]);
          if (coin_head(philox_coin((unsigned long long)arc, a.seed), -1 - dq[q], a.coin_lim)) {
            nheads++;
            if (atomicAdd(a.scnt + u[q], 1) == a.mu - 1) bag |= 1u << q;
          }
        }
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++)
      if (dq[q] > t) {
        if constexpr (kCombine) {
          // warp aggregation: the lanes of this slot that decrement the same
          // vertex send one atomic of their count; the lane whose interval
          // (old - cnt, old] holds k reports the crossing, so it is still
          // decided once per vertex
          const unsigned grp = __match_any_sync(__activemask(), u[q]);
          if (lane == __ffs(grp) - 1) {
            const int cnt = __popc(grp);
            ndec++;
            const int old = atomicSub(a.deg + u[q], cnt);
            if (old > t && old - cnt <= t) cross |= 1u << q;
          }
        } else {
          ndec++;
          const int old = atomicSub(a.deg + u[q], 1);
          if (old == t + 1) cross |= 1u << q;
          if (kWin && old == pc.win_hi) enter |= 1u << q;  // d~ drops into the level window
        }
      }
    if (kWin && __any_sync(kFull, enter != 0)) {
      // append the vertices entering the window to the active list
#pragma unroll
      for (int q = 0; q < kIlp; q++) {
        const bool f = (enter >> q) & 1u;
        const unsigned fm = __ballot_sync(kFull, f);
        if (fm) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(&pc.R->found, (unsigned long long)__popc(fm));
          base = __shfl_sync(kFull, base, 0);
          const unsigned long long p = pc.near_base + base + __popc(fm & lanemask_lt());
          if (f) {
            if (p < (unsigned long long)a.n) pc.near[p] = u[q];
            else raise_status(a, ST_CAPACITY);
          }
        }
      }
    }
    if constexpr (kSample) {
      if (__any_sync(kFull, bag != 0)) {
#pragma unroll
        for (int q = 0; q < kIlp; q++) append_recount(a, pc.R, (bag >> q) & 1u, u[q], lane);
      }
    }
    if (__any_sync(kFull, cross != 0)) {
#pragma unroll
      for (int q = 0; q < kIlp; q++) {
        const bool f = (cross >> q) & 1u;
        if (f) a.core[u[q]] = pc.val;
        if (__any_sync(kFull, f)) push_crossed<kSample>(a, sh, pc, f, u[q], warp, lane);
      }
      if (a.threshold) {
        const int nc = warp_sum(__popc(cross));
        if (lane == 0) sh.ncross[warp] += nc;
      }
    }
  }
  if (a.trace) {
    ndec = warp_sum(ndec);
    if (lane == 0) {
      sh.tr_arcs[warp] += total;
      sh.tr_decs[warp] += ndec;
    }
  }
  if constexpr (kSample) {
    if (__any_sync(kFull, nheads != 0)) {
      nheads = warp_sum(nheads);
      if (lane == 0) sh.heads[warp] += nheads;
    }
  }
  __syncwarp();
}

// Runs up to a.local_batches batches from the warp's local queue (vertices
// that crossed during this pass), then moves what is left to the queue.
template <bool kWin, bool kSample = false, bool kCombine = false>
__device__ void drain_local(const PeelArgs& a, ShT<kSample>& sh, const PassCtx& pc, int warp, int lane) {
  for (int b = 0;; b++) {
    const int lqn = sh.lqn[warp];
    if (lqn == 0) return;
    if (b >= a.local_batches) {
      // spill: one item per queued vertex
      __syncwarp();
      if (lane == 0) sh.lqn[warp] = 0;
      unsigned long long base = 0;
      if (lane == 0) {
        base = pc.qbase + atomicAdd(&pc.R->tail, (unsigned long long)lqn);
        atomicAdd(&s_app, (unsigned long long)lqn);
      }
      base = __shfl_sync(kFull, base, 0);
      if (base + (unsigned long long)lqn > (unsigned long long)a.qcap) {
        if (lane == 0) raise_status(a, ST_CAPACITY);
      } else {
        for (int i = lane; i < lqn; i += kWarp) a.Q[base + i] = sh.lq[warp][i];
      }
      if constexpr (kSample) {
        for (int i = lane; i < lqn; i += kWarp) a.stamp[sh.lqv[warp][i]] = pc.pass + 1;
      }
      __syncwarp();
      return;
    }
    const int c = min(lqn, kWarp);
    const unsigned long long item = lane < c ? sh.lq[warp][lqn - c + lane] : 0;
    __syncwarp();
    if (lane == 0) sh.lqn[warp] = lqn - c;
    __syncwarp();
    process_items<kWin, kSample, kCombine>(a, sh, pc, item, c, warp, lane);
    if (lane == 0) {
      sh.w_local[warp] += c;
      if (((++sh.w_lb[warp]) & 63) == 0) atomicAdd(&a.ctl->progress, 1ull);
    }
  }
}

// One subround: the queue range [qb, qe) is processed once by `nctas` CTAs
// (the grid, or CTA 0 alone in tail mode), this one being number `cta`. Warp
// gw takes its own contiguous share (len / warps items, one more for the
// first len % warps warps) in chunks of up to 32 items, so a pass has no claim
// traffic and ends for a warp as soon as its share and local queue are done.
template <bool kWin, bool kSample = false, bool kCombine = false>
__device__ void run_pass(const PeelArgs& a, ShT<kSample>& sh, const PassCtx& pc, unsigned long long qb,
                         unsigned long long qe, int cta, int nctas) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gw = (unsigned long long)cta * kWarps + warp;
  const unsigned long long nw = (unsigned long long)nctas * kWarps;
  const unsigned long long len = qe - qb, share = len / nw, rem = len % nw;
  const unsigned long long b = qb + gw * share + (gw < rem ? gw : rem);
  const unsigned long long e = b + share + (gw < rem ? 1 : 0);
  for (unsigned long long pos = b; pos < e; pos += kTake) {
    const int c = (int)min((unsigned long long)kTake, e - pos);
    const unsigned long long item = lane < c ? ld_once_u64(a.Q + pos + lane, l2_evict_first_policy()) : 0;
    process_items<kWin, kSample, kCombine>(a, sh, pc, item, c, warp, lane);
    if (lane == 0) sh.w_items[warp] += c;
    drain_local<kWin, kSample, kCombine>(a, sh, pc, warp, lane);
  }
}

// ---- offline subrounds (sync mode 3): Algorithm 2 -------------------------
// A subround is two phases. The histogram phase walks the arcs of the
// frontier items (edge-balanced over each warp, as process_items) and counts,
// per neighbour still above the level, how many frontier arcs reach it; the
// first count of a neighbour appends it to the touched list. The apply phase
// gives each touched vertex to one thread, which subtracts its count from d~
// in one step and, when d~ dropped from above k to k or below, gives it
// coreness k and appends its slices as the next frontier. No decision depends
// on the order of concurrent updates.
template <bool kTouched>
__device__ void hist_items(const PeelArgs& a, Shared& sh, const PassCtx& pc, unsigned long long item, int c,
                           int warp, int lane) {
  const int t = pc.t;
  const long long a0 = lane < c ? (long long)(item & kArcMask) : 0;
  const int len = lane < c ? (int)(item >> kLenShift) : 0;
  const int incl = warp_incl_scan(len, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  sh.excl[warp][lane] = incl - len;
  sh.a0[warp][lane] = a0;
  __syncwarp();
  const int* excl = sh.excl[warp];
  for (int base = 0; base < total; base += kWarp * kIlp) {
    int u[kIlp];
    int j = base + lane;
    int lo = 0, hi = c;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (excl[mid] <= j) lo = mid + 1;
      else hi = mid;
    }
    int idx = lo > 0 ? lo - 1 : 0;
#pragma unroll
    for (int q = 0; q < kIlp; q++, j += kWarp) {
      u[q] = -1;
      if (j < total) {
        while (idx + 1 < c && excl[idx + 1] <= j) idx++;
        const long long arc = sh.a0[warp][idx] + (j - excl[idx]);
        const int x = arc < a.m ? ld_stream_s32(a.adj + arc) : -1;
        if ((unsigned)x < (unsigned)a.n) u[q] = x;
        else raise_status(a, ST_NOT_SIMPLE);
      }
    }
    int dq[kIlp];
#pragma unroll
    for (int q = 0; q < kIlp; q++) dq[q] = u[q] >= 0 ? __ldcg(a.deg + u[q]) : INT_MIN;
    if (!kTouched) {
      // counts only: the apply phase walks the active list, which holds every
      // vertex above k; a reduction without return value is cheaper
#pragma unroll
      for (int q = 0; q < kIlp; q++)
        if (dq[q] > t) asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(a.hcnt + u[q]) : "memory");
      continue;
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++) {
      // d~ does not change during this phase: only neighbours above k count
      const bool first = dq[q] > t && atomicAdd(a.hcnt + u[q], 1) == 0;
      const unsigned fm = __ballot_sync(kFull, first);
      if (fm) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&pc.R->head, (unsigned long long)__popc(fm));
        base = __shfl_sync(kFull, base, 0);
        const unsigned long long p = base + __popc(fm & lanemask_lt());
        if (first) {
          if (p < (unsigned long long)a.n) a.touched[p] = u[q];
          else raise_status(a, ST_CAPACITY);
        }
      }
    }
  }
  __syncwarp();
}

template <bool kTouched>
__device__ void run_hist(const PeelArgs& a, Shared& sh, const PassCtx& pc, unsigned long long qb,
                         unsigned long long qe) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  const unsigned long long len = qe - qb, share = len / nw, rem = len % nw;
  const unsigned long long b = qb + gw * share + (gw < rem ? gw : rem);
  const unsigned long long e = b + share + (gw < rem ? 1 : 0);
  for (unsigned long long pos = b; pos < e; pos += kTake) {
    const int c = (int)min((unsigned long long)kTake, e - pos);
    const unsigned long long item = lane < c ? ld_once_u64(a.Q + pos + lane, l2_evict_first_policy()) : 0;
    hist_items<kTouched>(a, sh, pc, item, c, warp, lane);
    if (lane == 0) sh.w_items[warp] += c;
  }
}

// Apply phase over list[0, nt) (the touched list, or the active list, where
// untouched vertices have count 0): a warp handles 32 vertices at a time.
__device__ void run_apply(const PeelArgs& a, const PassCtx& pc, const int* list, unsigned long long nt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  const int t = pc.t;
  for (unsigned long long base = gw * kWarp; base < nt; base += nw * kWarp) {
    const unsigned long long i = base + lane;
    int u = -1;
    bool cross = false;
    long long e0 = 0, e1 = 0;
    int nsl = 0;
    if (i < nt) {
      u = __ldcg(list + i);
      if ((unsigned)u < (unsigned)a.n) {
        const int f = __ldcg(a.hcnt + u);
        if (f) a.hcnt[u] = 0;
        const int old = __ldcg(a.deg + u);
        a.deg[u] = old - f;
        cross = old > t && old - f <= t;
        if (cross) {
          a.core[u] = pc.val;
          e0 = a.off[u];
          e1 = a.off[u + 1];
          nsl = (int)((e1 - e0 + a.slice - 1) / a.slice);
        }
      } else {
        raise_status(a, ST_CAPACITY);
      }
    }
    append_ranges<true>(a, pc, cross ? nsl : 0, e0, e1, lane);
  }
}

// ---- sampling recounts (SetSampler of Algorithm 5, two phases) ------------
// Counting phase: the recount queue's slices are split into per-warp shares;
// a warp counts the arcs of its slice whose target is not yet traversed
// (stamp >= done_passes: no completed pass traversed it) and those not
// traversed before the level began (stamp >= level_pass), and adds both to
// the slice owner's accumulators.
__device__ void run_recount_count(const PeelArgs& a, unsigned long long nq, long long done_passes,
                                  long long level_pass) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  for (unsigned long long i = gw; i < nq; i += nw) {
    const unsigned long long item = __ldcg(a.RQ + i);
    const int v = __ldcg(a.RQv + i);
    const long long a0 = (long long)(item & kArcMask);
    const int len = (int)(item >> kLenShift);
    int left = 0, at = 0;
    for (int j0 = 0; j0 < len; j0 += kWarp * 4) {
      int st[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int j = j0 + q * kWarp + lane;
        st[q] = INT_MIN;
        if (j < len) {
          const long long arc = a0 + j;
          const int u = arc < a.m ? ld_stream_s32(a.adj + arc) : -1;
          if ((unsigned)u < (unsigned)a.n) st[q] = __ldcg(a.stamp + u);
          else raise_status(a, ST_NOT_SIMPLE);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        left += st[q] >= done_passes ? 1 : 0;
        at += st[q] >= level_pass ? 1 : 0;
      }
    }
    left = warp_sum(left);
    at = warp_sum(at);
    if (lane == 0) {
      if (left) atomicAdd(a.racc + v, left);
      if (at) atomicAdd(a.rst + v, at);
    }
  }
}

// Apply phase: each recounted vertex v (one thread) takes its untraversed
// count as d~. A vertex with fewer than k neighbours untraversed when level k
// began missed an earlier level: the run is marked for a rerun without
// sampling (Sec. 4.1, "Recover from Errors"). Otherwise, at or below k, v
// gets coreness k and joins the next pass (stamp next_pass, slices appended
// after pc.qbase, count in pc.R->found); above it, InitSampler(v, k) puts v
// back in sample mode or leaves its exact d~. Accumulators are cleared. The
// least next key of the vertices kept goes to pc.R->minkey.
__device__ void run_recount_apply(const PeelArgs& a, const PassCtx& pc, unsigned long long nr, int k,
                                  int next_pass) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  int kmin = INT_MAX;
  for (unsigned long long base = gw * kWarp; base < nr; base += nw * kWarp) {
    const unsigned long long i = base + lane;
    bool join = false;
    long long e0 = 0, e1 = 0;
    if (i < nr) {
      const int v = __ldcg(a.rlist + i);
      const int left = __ldcg(a.racc + v), at = __ldcg(a.rst + v);
      a.racc[v] = 0;
      a.rst[v] = 0;
      if (at < k) {
        if (atomicCAS(&a.ctl->s_miss, 0, 1) == 0) {
          a.ctl->s_miss_round = k;
          a.ctl->s_miss_vertex = v;
        }
        a.ctl->s_redo = 1;
      } else if (left <= k) {
        a.core[v] = pc.val;
        a.deg[v] = left;
        a.stamp[v] = next_pass;
        join = true;
        e0 = a.off[v];
        e1 = a.off[v + 1];
      } else if ((long long)left > 10ll * k && (long long)left > a.sthreshold) {
        a.deg[v] = -1 - left;  // InitSampler(v, k): sample mode again
        a.scnt[v] = 0;
        kmin = min(kmin, sample_key(left, 0, a.mu));
      } else {
        a.deg[v] = left;
        kmin = min(kmin, left);
      }
    }
    const unsigned jm = __ballot_sync(kFull, join);
    if (jm && lane == 0) atomicAdd(&pc.R->found, (unsigned long long)__popc(jm));
    const int nsl = join ? (int)((e1 - e0 + a.slice - 1) / a.slice) : 0;
    append_ranges<true>(a, pc, nsl, e0, e1, lane);
  }
  kmin = warp_min(kmin);
  if (lane == 0 && kmin != INT_MAX) atomicMax(&pc.R->minkey, INT_MAX - kmin);
}

// Instantiations: kOffline (Algorithm 2's subrounds), kWindow (the level
// window), kHybrid (batch update of heavy subrounds), kSample (sampling),
// kCombine (warp-aggregated decrements) and kTail (tail mode), each compiled
// apart so the default kernel carries none of the others.
template <bool kOffline, bool kWindow, bool kHybrid, bool kSample, bool kCombine = false, bool kTail = false>
__global__ void __launch_bounds__(kBlock, 2) peel_bsp(PeelArgs a) {
  __shared__ ShT<kSample> sh;
  // a rerun that is not needed ends at once (every CTA reads the same flag)
  if (a.run_if && ld_relaxed_s32(a.run_if) == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool lead = blockIdx.x == 0 && tid == 0;
  if (tid == 0) {
    s_app = 0;
    s_abort = 0;
  }
  if (lane == 0) {
    sh.lqn[warp] = 0;
    sh.tr_arcs[warp] = sh.tr_decs[warp] = 0;
    sh.ncross[warp] = 0;
    sh.w_items[warp] = sh.w_local[warp] = 0;
    sh.w_lb[warp] = 0;
    if constexpr (kSample) sh.heads[warp] = 0;
  }
  // grid barriers taken; grid phase g uses RoundRec g % 3 and barrier word g % 3
  unsigned long long gen = 0;
  // Tail mode (the plain schedule only): a phase whose range is small runs on
  // CTA 0 alone and ends at a CTA barrier; its counters live in the CTA's own
  // ring of records (tail phase s uses sh.tring[s % 3]).
  // (sh.sphase: tail phases run; sh.tail_gen: tail episodes begun, kept by
  // thread 0 of each CTA, the same count in every CTA)
  bool solo = false;
  if (tid == 0) {
    sh.sphase = 0;
    sh.tail_gen = 0;
  }
  auto rec = [&]() -> RoundRec* {
    return solo ? &sh.tring[sh.sphase % kPhaseRing] : a.rounds + (gen % kPhaseRing);
  };
  auto clear_rec = [&](RoundRec* R) {
    R->alen = 0;
    R->found = 0;
    R->minkey = 0;
    R->tail = 0;
    R->head = 0;
    if constexpr (kSample) {
      R->rcount = 0;
      R->rqtail = 0;
    }
  };
  auto reset_next = [&]() {
    // the records of the next phase were last used two phases ago
    if (solo) {
      if (tid == 0) clear_rec(&sh.tring[(sh.sphase + 1) % kPhaseRing]);
      return;
    }
    const int r = (int)((gen + 1) % kPhaseRing);
    if (lead) {
      clear_rec(a.rounds + r);
      a.ctl->bar_ring[r].v = 0;
    }
  };
  auto nscan_of = [&](long long len) {
    long long ns = (len + a.scan_min - 1) / a.scan_min;
    return ns < 1 ? 1ll : (ns > (long long)gridDim.x ? (long long)gridDim.x : ns);
  };
  auto free_list = [&](const int* x, const int* y) -> int* {
    return (x != a.A0 && y != a.A0) ? a.A0 : ((x != a.A1 && y != a.A1) ? a.A1 : a.A2);
  };
  if constexpr (!kSample) {
  // per-phase timeline (trace mode 2): after each barrier CTA 0 records the
  // time, the phase kind (0 scan, 1 pass, 2 count, 3 apply, 4 second scan),
  // the level, the range it worked on, its appends, the frontier found, the
  // arcs read (passes) and whether CTA 0 ran the phase alone (tail mode)
  // (the record count lives in shared memory: a register held across the
  // whole level loop made the hot loop spill)
  if (lead) {
    sh.trec = 0;
    sh.tarcs = 0;
    sh.ld = {};
  }
  // (the phase's appends come from the counters the barrier already read)
  auto prec = [&](int kind, int level, unsigned long long range, unsigned long long found) {
    if (!(lead && a.trace_phases && sh.trec < a.max_rounds)) return;
    unsigned long long* tr = a.trace + (size_t)sh.trec * kTraceFields;
    const unsigned long long arcs = ld_relaxed_u64(&a.ctl->tr_arcs);
    tr[0] = globaltimer_ns();
    tr[1] = (unsigned long long)kind;
    tr[2] = (unsigned long long)level;
    tr[3] = range;
    tr[4] = sh.po.tail;
    tr[5] = found;
    tr[6] = arcs - sh.tarcs;
    tr[7] = solo ? 1 : 0;
    sh.tarcs = arcs;
    sh.trec++;
  };
  // Window of levels [hi_w - W, hi_w) (bucketing, a.window = W > 0): the
  // active list holds only vertices below hi_w; the others wait in the
  // overflow list and enter the active list when a decrement returns exactly
  // hi_w (once per vertex and window). When the next level reaches hi_w, a
  // rebuild scan of the overflow list starts the next window. Three list
  // buffers rotate: active, overflow and the output of the next scan.
  const int W = (kWindow && !kOffline && a.window > 0 && !a.threshold) ? a.window : 0;
  const int* Acur = nullptr;   // active list (nullptr without window: all vertices)
  long long la = W ? 0 : a.n;
  const int* Aover = nullptr;  // overflow list (nullptr with window: all vertices, before the first rebuild)
  long long lover = W ? a.n : 0;
  int hi_w = W ? 0 : INT_MAX;
  long long near_extra = 0;    // entries appended to the active list by the passes since its scan
  int tp = -1;                 // the last level peeled
  int t = 0;                   // the level being peeled
  unsigned long long qend = 0;  // items appended by all completed phases
  unsigned long long qb = 0;    // the current pass's queue range is [qb, qend)
  // Ends a phase: the grid barrier, or in tail mode a CTA barrier after which
  // thread 0 copies the phase's counters from the CTA's own record (and ticks
  // the heartbeat the parked CTAs' bounded wait watches).
  auto sync = [&](RoundRec* R, bool want_rec) -> bool {
    if (!solo) return grid_barrier(a, sh, gen, want_rec ? R : nullptr);
    __syncthreads();
    if (tid == 0) {
      sh.po.tail = R->tail;
      sh.po.head = R->head;
      sh.po.found = R->found;
      sh.po.alen = R->alen;
      sh.po.minkey = R->minkey;
      s_app = 0;
      sh.flag = s_abort == 0;
      sh.sphase++;
      asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(&a.ctl->progress) : "memory");
    }
    __syncthreads();
    return sh.flag != 0;
  };
  // The steps of the level loop; a parked CTA resumes at the step CTA 0 hands it.
  enum : int { kNxScan = 0, kNxPass = 1, kNxEnd = 2, kNxDone = 3 };
  int nx = kNxScan;
  const bool tail_ok = kTail && !kOffline && !W && !a.threshold && (a.tail_items > 0 || a.tail_entries > 0);
  // Starts a tail episode. CTA 0 goes on alone (true); every other CTA parks
  // (false) until CTA 0 hands the loop back.
  auto begin_tail = [&]() -> bool {
    if (tid == 0) sh.tail_gen++;
    if (blockIdx.x != 0) return false;
    solo = true;
    if (tid == 0)
      for (int r = 0; r < kPhaseRing; r++) clear_rec(&sh.tring[r]);
    __syncthreads();
    return true;
  };
  // A parked CTA waits (bounded by the heartbeat) for CTA 0's release of the
  // current episode, then takes the loop state it handed over. False: the
  // kernel ends (the peel finished in tail mode, a status was raised, or the
  // wait gave up).
  auto park = [&]() -> bool {
    if (tid == 0) {
      int okp = 1;
      uint64_t t0 = 0;
      unsigned long long pg = 0;
      for (unsigned spins = 0;; spins++) {
        const unsigned long long v = ld_acquire_u64(&a.ctl->tail_word);
        if (v & kAbort) {
          okp = 0;
          break;
        }
        if (v >= (unsigned long long)sh.tail_gen) break;
        if ((spins & 31) == 0) {
          const uint64_t now = globaltimer_ns();
          const unsigned long long p2 = ld_relaxed_u64(&a.ctl->progress);
          if (spins == 0 || p2 != pg) {
            pg = p2;
            t0 = now;
          } else if (now - t0 > a.timeout_ns) {
            raise_status(a, ST_TIMEOUT);
            okp = 0;
            break;
          }
        }
        __nanosleep(a.park_sleep_ns);
      }
      if (okp)
        for (int i = 0; i < kHandoff; i++) sh.ho[i] = (long long)ld_relaxed_u64(&a.ctl->handoff[i]);
      sh.flag = okp;
    }
    __syncthreads();
    if (!sh.flag) return false;
    nx = (int)sh.ho[0];
    tp = (int)sh.ho[1];
    qend = (unsigned long long)sh.ho[2];
    qb = (unsigned long long)sh.ho[3];
    la = sh.ho[4];
    Acur = sh.ho[5] == 0 ? a.A0 : sh.ho[5] == 1 ? a.A1 : sh.ho[5] == 2 ? a.A2 : nullptr;
    t = (int)sh.ho[6];
    return nx != kNxDone;
  };
  // CTA 0 ends the episode: the loop state (next step `next`) goes to the
  // parked CTAs with one release, and the phases that follow use the grid.
  auto end_tail = [&](int next) {
    __syncthreads();  // orders the CTA's writes of the episode before the release
    if (tid == 0) {
      unsigned long long* h = a.ctl->handoff;
      h[0] = (unsigned long long)next;
      h[1] = (unsigned long long)(long long)tp;
      h[2] = qend;
      h[3] = qb;
      h[4] = (unsigned long long)la;
      h[5] = Acur == a.A0 ? 0 : Acur == a.A1 ? 1 : Acur == a.A2 ? 2 : 3;
      h[6] = (unsigned long long)(long long)t;
      // (test hook: the first release is withheld, so every parked wait runs out)
      if (!(a.inject_stall && sh.tail_gen == 1))
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&a.ctl->tail_word), "l"(1ull) : "memory");
    }
    solo = false;
  };
  for (;;) {
    if (nx == kNxScan) {
      // ---- scan: keep d~ > tp+1, take d~ == tp+1 (a k'-core query: one level,
      // kprime - 1, taking every d~ below kprime and marking the rest 1)
      const int tk = a.threshold ? a.kprime - 1 : tp + 1;
      const bool rebuild = W && tk >= hi_w;
      const long long lin = rebuild ? lover : la + near_extra;
      if (tail_ok) {
        const bool small = lin <= a.tail_entries;
        if (small && !solo) {
          if (!begin_tail()) {
            if (!park()) break;
            continue;
          }
        } else if (!small && solo) {
          end_tail(kNxScan);
        }
      }
      if (lead && a.trace) {
        sh.ld.t_start = globaltimer_ns();
        sh.ld.rebuild = rebuild;
      }
      reset_next();
      RoundRec* R = rec();
      const int* Ain = rebuild ? Aover : Acur;
      int* Aout = free_list(Acur, Aover);
      // a rebuild writes the overflow list to the exhausted active list's buffer
      int* Aov = rebuild ? (Acur ? const_cast<int*>(Acur) : free_list(Aout, Aover)) : nullptr;
      long long nscan = solo ? 1 : nscan_of(lin);
      if (blockIdx.x < nscan) {
        const long long lo = lin * blockIdx.x / nscan, hi = lin * (blockIdx.x + 1) / nscan;
        const ScanOut o = a.threshold ? scan_range(a, sh, R, qend, Ain, Aout, lo, hi, tk, tk, true, 0, 1)
                          : rebuild  ? scan_range(a, sh, R, qend, Ain, Aout, lo, hi, tk, tk, false, -1, -1, Aov,
                                                  tk + W)
                                     : scan_range(a, sh, R, qend, Ain, Aout, lo, hi, tk, tk);
        if (tid == 0) {
          if (o.found) atomicAdd(&R->found, o.found);
          if (o.dmin != INT_MAX) atomicMax(&R->minkey, INT_MAX - o.dmin);
        }
      }
      if (!sync(R, true)) break;
      const unsigned long long found = sh.po.found;
      prec(0, tk, (unsigned long long)lin, found);
      const long long alen = (long long)sh.po.alen;
      const int minkey = sh.po.minkey;
      if (lead) {
        sh.ld.scanned += lin;
        sh.ld.la_scanned = lin;
        sh.ld.nscan = nscan;
        sh.ld.nfound = found;
      }
      qb = qend;
      qend += sh.po.tail;
      Acur = Aout;
      if (rebuild) {
        Aover = Aov;
        lover = (long long)sh.po.head;
        hi_w = tk + W;
      }
      near_extra = 0;
      la = alen;
      t = tk;
      if (!found && !a.threshold) {
        if (alen == 0 && lover == 0) break;  // nothing left
        if (lead) sh.ld.empty++;
        if (W && alen == 0) {
          // nothing left in the window: a rebuild starts the next one at the
          // least d~ of the overflow list (known if this scan was a rebuild)
          tp = rebuild ? INT_MAX - minkey - 1 : hi_w - 1;
          continue;
        }
        // level tk is empty: the least induced degree of the kept vertices is the next level
        t = INT_MAX - minkey;
        if (tail_ok && !solo && la <= a.tail_entries) {
          if (!begin_tail()) {
            if (!park()) break;
            continue;
          }
        }
        reset_next();
        R = rec();
        nscan = solo ? 1 : nscan_of(la);
        if (blockIdx.x < nscan) {
          const long long lo = la * blockIdx.x / nscan, hi = la * (blockIdx.x + 1) / nscan;
          const ScanOut o = scan_range(a, sh, R, qend, Acur, nullptr, lo, hi, INT_MAX, t);
          if (tid == 0 && o.found) atomicAdd(&R->found, o.found);
        }
        if (!sync(R, true)) break;
        prec(4, t, (unsigned long long)la, sh.po.found);
        if (lead) {
          sh.ld.scanned += la;
          sh.ld.nscan = nscan;
          sh.ld.nfound = sh.po.found;
        }
        qend += sh.po.tail;
      }
      tp = t;
      if (lead) {
        sh.ld.kmax = t;
        sh.ld.levels++;
        sh.ld.level_qb = qb;
        sh.ld.level_passes = 0;
        if (a.trace) {
          sh.ld.t_scan = globaltimer_ns();
          sh.ld.arcs0 = ld_relaxed_u64(&a.ctl->tr_arcs);
          sh.ld.decs0 = ld_relaxed_u64(&a.ctl->tr_decs);
        }
      }
      // with no vertex left above the level nothing can be decremented (the
      // offline schedule still counts the level's one subround)
      if (kOffline || la > 0 || lover > 0) {
        nx = kNxPass;
      } else {
        qb = qend;
        nx = kNxEnd;
      }
      continue;
    }
    if (nx == kNxPass) {
      if (kOffline) {
        // Algorithm 1's subrounds exactly: also the last level (nothing left
        // above it) and a frontier without arcs count as one subround each
        if (qend > qb) {
          // histogram phase: counts and the touched list (count in P->head)
          reset_next();
          RoundRec* P = rec();
          const PassCtx hc{P, qend, t, t, false, -1, nullptr, 0};
          run_hist<true>(a, sh, hc, qb, qend);
          if (!sync(P, true)) break;
          const unsigned long long nt = sh.po.head;
          // apply phase: crossings append the next frontier (count in P2->tail)
          reset_next();
          RoundRec* P2 = rec();
          const PassCtx pc{P2, qend, t, t, false, -1, nullptr, 0};
          run_apply(a, pc, a.touched, nt);
          if (!sync(P2, false)) break;
          if (lead) {
            sh.ld.passes++;
            sh.ld.level_passes++;
          }
          qb = qend;
          qend += sh.po.tail;
          continue;
        }
        if (lead && sh.ld.level_passes == 0 && sh.ld.nfound > 0) {
          sh.ld.passes++;
          sh.ld.level_passes++;
        }
        nx = kNxEnd;
        continue;
      }
      if (qend <= qb) {
        nx = kNxEnd;
        continue;
      }
      if (tail_ok) {
        const bool small = qend - qb <= (unsigned long long)a.tail_items;
        if (small && !solo) {
          if (!begin_tail()) {
            if (!park()) break;
            continue;
          }
        } else if (!small && solo) {
          end_tail(kNxPass);
        }
      }
      if (kHybrid && !W && !solo && 4 * (qend - qb) >= (unsigned long long)gridDim.x * kWarps &&
          (qend - qb) >= (unsigned long long)la) {
        // a heavy subround over a short active list: count the decrements
        // per neighbour with reductions, then apply them walking the active
        // list (Algorithm 2's batch update, the crossing decided once per
        // vertex by its owner). Reductions need no return trip and run at
        // about 1.5x the rate of returning atomics on this GPU; the apply
        // walk costs one pass over the active list and a second barrier.
        // Measured on R-MAT 24 / R-MAT 22 / kNN: -2.7% / -0.5% / -1.4%.
        reset_next();
        RoundRec* P = rec();
        const PassCtx hc{P, qend, t, t, false, -1, nullptr, 0};
        run_hist<false>(a, sh, hc, qb, qend);
        if (!sync(P, false)) break;
        prec(2, t, qend - qb, 0);
        reset_next();
        RoundRec* P2 = rec();
        const PassCtx pc{P2, qend, t, t, false, -1, nullptr, 0};
        run_apply(a, pc, Acur, (unsigned long long)la);
        if (!sync(P2, false)) break;
        prec(3, t, (unsigned long long)la, 0);
        if (lead) {
          sh.ld.passes++;
          sh.ld.level_passes++;
        }
        qb = qend;
        qend += sh.po.tail;
        continue;
      }
      reset_next();
      RoundRec* P = rec();
      const int nctas = solo ? 1 : (int)gridDim.x;
      // a pass whose per-warp share is at least a.precheck_items items is
      // throughput-bound (measured: kNN's largest level 1,700 items per
      // warp; R-MAT passes a few)
      const bool pre = (qend - qb) >= (unsigned long long)a.precheck_items * nctas * kWarps;
      const PassCtx pc{P, qend, t, a.threshold ? 0 : t, pre, W ? hi_w : -1, const_cast<int*>(Acur),
                       (unsigned long long)(la + near_extra)};
      run_pass<kWindow, false, kCombine>(a, sh, pc, qb, qend, solo ? 0 : (int)blockIdx.x, nctas);
      if (a.threshold && lane == 0 && sh.ncross[warp]) {
        atomicAdd(&a.ctl->crossed, (unsigned long long)sh.ncross[warp]);
        sh.ncross[warp] = 0;
      }
      if (a.trace) {
        // one pair of atomics per CTA (per warp, 9,728 same-address atomics
        // would add several microseconds to every traced pass)
        __syncthreads();
        if (tid == 0) {
          unsigned long long ta = 0, td = 0;
          for (int w = 0; w < kWarps; w++) {
            ta += sh.tr_arcs[w];
            td += sh.tr_decs[w];
            sh.tr_arcs[w] = sh.tr_decs[w] = 0;
          }
          if (ta) atomicAdd(&a.ctl->tr_arcs, ta);
          if (td) atomicAdd(&a.ctl->tr_decs, td);
        }
      }
      if (!sync(P, W != 0)) break;
      if (lead) {
        sh.ld.passes++;
        sh.ld.level_passes++;
      }
      prec(1, t, qend - qb, 0);
      qb = qend;
      qend += sh.po.tail;
      if (W) near_extra += (long long)sh.po.found;
      continue;
    }
    // ---- nx == kNxEnd: the level is finished
    if (lead && a.trace && !a.trace_phases && sh.ld.levels - 1 < a.max_rounds) {
      unsigned long long* tr = a.trace + (size_t)(sh.ld.levels - 1) * kTraceFields;
      tr[0] = sh.ld.t_start;
      tr[1] = sh.ld.t_scan;
      tr[2] = globaltimer_ns();
      tr[3] = (unsigned long long)t;
      tr[4] = (unsigned long long)sh.ld.la_scanned;
      tr[5] = sh.ld.nfound;
      tr[6] = qend - sh.ld.level_qb;
      tr[7] = (unsigned long long)sh.ld.nscan;
      tr[8] = ld_relaxed_u64(&a.ctl->tr_arcs) - sh.ld.arcs0;
      tr[9] = ld_relaxed_u64(&a.ctl->tr_decs) - sh.ld.decs0;
      tr[10] = sh.ld.rebuild ? 1 : 0;
      tr[13] = (unsigned long long)sh.ld.level_passes;
    }
    if (a.threshold) {
      // the k'-core: the vertices kept by the scan that no decrement removed
      if (lead && a.size_out) *a.size_out = la - (long long)ld_relaxed_u64(&a.ctl->crossed);
      break;
    }
    if (la == 0 && lover == 0 && near_extra == 0) break;
    nx = kNxScan;
  }
  // the parked CTAs leave with the loop
  if (solo) end_tail(kNxDone);
  if (lead) {
    if (a.kmax_out) *a.kmax_out = sh.ld.kmax;
    a.ctl->rounds = sh.ld.levels + sh.ld.empty;
    a.ctl->empty_rounds = sh.ld.empty;
    a.ctl->scanned = sh.ld.scanned;
    a.ctl->kmax = sh.ld.kmax;
    a.ctl->passes = sh.ld.passes;
    a.ctl->barriers = (long long)gen;
    a.ctl->tail_phases = sh.sphase;
    a.ctl->tail_episodes = (long long)sh.tail_gen;
  }
  } else {
    // ---- Algorithm 4 with the sampling Peel of Algorithm 5. A level is a
    // scan at k = previous level + 1 that also validates the vertices in
    // sample mode (those failing Error(v, k) are recounted before the first
    // pass), then passes as above in which a neighbour in sample mode tosses
    // a coin instead of being decremented; after a pass that filled counting
    // bags, those vertices are recounted. A recount is two phases (count,
    // apply), each closed by the grid barrier. A level that finds no vertex
    // moves to the least next key of the kept vertices: their least d~, or
    // for a vertex in sample mode the first level its validation could fail
    // at. A recount that finds a missed level ends the run (the result is
    // then recomputed without sampling).
    const int* Acur = nullptr;  // active list (nullptr: all vertices)
    long long la = a.n;
    int tp = -1, kmax = 0;
    long long levels = 0, empty = 0, scanned = 0, passes = 0;
    unsigned long long qend = 0;  // items appended by all completed phases
    for (;;) {
      const int tk = tp + 1;
      reset_next();
      RoundRec* R = rec();
      int* Aout = free_list(Acur, nullptr);
      const long long lin = la;
      const long long nscan = nscan_of(lin);
      if (blockIdx.x < nscan) {
        const long long lo = lin * blockIdx.x / nscan, hi = lin * (blockIdx.x + 1) / nscan;
        const ScanOut o = scan_range<true>(a, sh, R, qend, Acur, Aout, lo, hi, tk, tk, false, -1, -1, nullptr,
                                           INT_MAX, (int)passes);
        if (tid == 0) {
          if (o.found) atomicAdd(&R->found, o.found);
          if (o.dmin != INT_MAX) atomicMax(&R->minkey, INT_MAX - o.dmin);
        }
      }
      if (!grid_barrier(a, sh, gen, R)) break;
      scanned += lin;
      unsigned long long nfound = sh.po.found;
      la = (long long)sh.po.alen;
      const int mk = sh.po.minkey;
      int kmin = mk ? INT_MAX - mk : INT_MAX;
      unsigned long long qb = qend;
      qend += sh.po.tail;
      const unsigned long long nr = sh.po.rcount, nrq = sh.po.rqtail;
      Acur = Aout;
      if (lead && nr) a.ctl->s_failed += (long long)nr;
      const long long level_pass = passes;
      bool ok = true, miss = false;
      auto recount = [&](unsigned long long nrv, unsigned long long nrqv) {
        // an append past either bound raised a status, which ended the phase's
        // barrier, so the counts are within them here
        nrv = min(nrv, (unsigned long long)a.n);
        nrqv = min(nrqv, (unsigned long long)a.rqcap);
        reset_next();
        run_recount_count(a, nrqv, passes, level_pass);
        if (!(ok = grid_barrier(a, sh, gen))) return;
        reset_next();
        RoundRec* P = rec();
        const PassCtx pc{P, qend, tk, tk, false, -1, nullptr, 0, (int)passes};
        run_recount_apply(a, pc, nrv, tk, (int)passes);
        if (!(ok = grid_barrier(a, sh, gen, P))) return;
        nfound += sh.po.found;
        qend += sh.po.tail;
        const int mk2 = sh.po.minkey;
        if (mk2) kmin = min(kmin, INT_MAX - mk2);
        if (lead) a.ctl->s_recounts += (long long)nrv;
        miss = sh.po.miss != 0;
      };
      if (nr) recount(nr, nrq);
      if (!ok || miss) break;
      if (nfound == 0) {
        if (la == 0) break;  // nothing left
        empty++;
        tp = kmin == INT_MAX ? tk : kmin - 1;
        continue;
      }
      kmax = tk;
      tp = tk;
      levels++;
      while (qend > qb) {
        reset_next();
        RoundRec* P = rec();
        const PassCtx pc{P, qend, tk, tk, true, -1, nullptr, 0, (int)passes};
        run_pass<false, true>(a, sh, pc, qb, qend, (int)blockIdx.x, (int)gridDim.x);
        if (!(ok = grid_barrier(a, sh, gen, P))) break;
        passes++;
        qb = qend;
        qend += sh.po.tail;
        const unsigned long long br = sh.po.rcount, bq = sh.po.rqtail;
        if (br) {
          if (lead) a.ctl->s_bag += (long long)br;
          recount(br, bq);
          if (!ok || miss) break;
        }
      }
      if (!ok || miss || la == 0) break;
    }
    if (lane == 0 && sh.heads[warp]) atomicAdd((unsigned long long*)&a.ctl->s_heads, sh.heads[warp]);
    if (lead) {
      if (a.kmax_out) *a.kmax_out = kmax;
      a.ctl->rounds = levels + empty;
      a.ctl->empty_rounds = empty;
      a.ctl->scanned = scanned;
      a.ctl->kmax = kmax;
      a.ctl->passes = passes;
      a.ctl->barriers = (long long)gen;
    }
  }
  if (lane == 0) {
    if (sh.w_items[warp]) atomicAdd(&a.ctl->items, (unsigned long long)sh.w_items[warp]);
    if (sh.w_local[warp]) atomicAdd(&a.ctl->local_items, (unsigned long long)sh.w_local[warp]);
  }
}

// Measures the grid barrier alone: `iters` barriers back to back with no work
// between them, on the same words and with the same waits as the peel; CTA 0
// writes the elapsed device time (ns) to *out.
__global__ void __launch_bounds__(kBlock, 2) barrier_probe(PeelArgs a, int iters, unsigned long long* out) {
  __shared__ Shared sh;
  if (threadIdx.x == 0) {
    s_app = 0;
    s_abort = 0;
  }
  unsigned long long gen = 0;
  __syncthreads();
  const uint64_t t0 = globaltimer_ns();
  for (int i = 0; i < iters; i++) {
    // the word of the next barrier was last polled two barriers ago
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->bar_ring[(gen + 1) % kPhaseRing].v = 0;
    if (!grid_barrier(a, sh, gen)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = globaltimer_ns() - t0;
}

}  // namespace

cudaError_t bsp_barrier_probe(const PeelArgs& args, int grid, int iters, unsigned long long* out_ns,
                              cudaStream_t stream) {
  PeelArgs a = args;
  void* params[] = {&a, &iters, &out_ns};
  return cudaLaunchCooperativeKernel((const void*)barrier_probe, dim3(grid), dim3(kBlock), params, 0, stream);
}

int bsp_max_ctas_per_sm() {
  const void* fns[] = {(const void*)peel_bsp<false, false, false, false>,
                       (const void*)peel_bsp<true, false, false, false>,
                       (const void*)peel_bsp<false, true, false, false>,
                       (const void*)peel_bsp<false, false, true, false>,
                       (const void*)peel_bsp<false, false, false, true>,
                       (const void*)peel_bsp<false, false, true, false, true>,
                       (const void*)peel_bsp<false, false, false, false, true>,
                       (const void*)peel_bsp<false, false, true, false, false, true>,
                       (const void*)peel_bsp<false, false, false, false, false, true>,
                       (const void*)peel_bsp<false, false, true, false, true, true>,
                       (const void*)peel_bsp<false, false, false, false, true, true>};
  int best = 1 << 30;
  for (const void* f : fns) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, 0) != cudaSuccess) return 0;
    best = nb < best ? nb : best;
  }
  return best;
}

int bsp_block_size() { return kBlock; }

cudaError_t bsp_launch(const PeelArgs& args, int grid, cudaStream_t stream) {
  PeelArgs a = args;
  void* params[] = {&a};
  // tail mode has instantiations of its own (the plain schedule, with or
  // without batch update and warp aggregation)
  const bool tail = !a.sample && !a.offline && a.window == 0 && !a.threshold &&
                    (a.tail_items > 0 || a.tail_entries > 0);
  const void* fn =
      a.sample    ? (const void*)peel_bsp<false, false, false, true>
      : a.offline ? (const void*)peel_bsp<true, false, false, false>
      : tail      ? (a.combine ? (a.hybrid ? (const void*)peel_bsp<false, false, true, false, true, true>
                                           : (const void*)peel_bsp<false, false, false, false, true, true>)
                               : (a.hybrid ? (const void*)peel_bsp<false, false, true, false, false, true>
                                           : (const void*)peel_bsp<false, false, false, false, false, true>))
      : a.combine && a.window == 0
          ? (a.hybrid ? (const void*)peel_bsp<false, false, true, false, true>
                      : (const void*)peel_bsp<false, false, false, false, true>)
      : a.window > 0 ? (const void*)peel_bsp<false, true, false, false>
      : a.hybrid     ? (const void*)peel_bsp<false, false, true, false>
                     : (const void*)peel_bsp<false, false, false, false>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), params, 0, stream);
}

}  // namespace kc
