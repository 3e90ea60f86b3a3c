// Single-graph k-core peel for sm_103a: one persistent cooperative kernel.
//
// What it computes: Algorithm 1 (rounds over the level k: the frontier is the
// live vertices whose induced degree equals k; after the round only vertices
// above k stay active) with the online Peel of Algorithm 3 (atomic decrement
// of a neighbour's induced degree; the decrement that returns k+1 is the one
// that lands it on k and puts it into the same level's work).
//
// How it is organised on the GPU (no per-subround barrier):
//  * Rounds end by a device-wide counter per round,
//    cnt = (scan tokens << 40) + (work items pushed - work items finished).
//    Each CTA that scans part of the active list adds one token after its
//    scan; the update that brings cnt to (scanning CTAs << 40) finishes the
//    round, and that thread broadcasts the round's results. Subrounds never
//    synchronise: work flows through a global queue (each vertex enters it
//    once over the run, as in Theorem 1's proof) and through per-warp local
//    queues in shared memory (the role of the local FIFO of vertical
//    granularity control, Sec. 4.2: a vertex that drops to k is processed by
//    the same worker without waiting for a new subround).
//  * The queue is append-only; round r owns the segment that starts where
//    round r-1's ended. A warp takes tickets with one fetch-and-add on the
//    round's head counter and then watches only its own slots; items carry
//    the round number's low 4 bits, so a slot written by the next round is
//    never taken for this one.
//  * A vertex enters the work as one "whole" item, without reading its
//    offsets; the warp that takes it splits an adjacency list longer than
//    `slice` arcs into slices and queues all but the first, so a hub's arcs
//    spread over many warps.
//  * Empty levels are skipped: the scan after level k speculates on k+1; if no
//    vertex sits at k+1 the round is empty and the scan's minimum over the
//    surviving induced degrees is the next level (the framework's "k <- k+1"
//    with empty levels skipped, which changes no coreness).
//  * The scan of a level overlaps its processing (a frontier vertex found by
//    one CTA is peeled while other CTAs still scan). A vertex can then be
//    found both by the scan and by a decrement that lands it on k, so its one
//    owner is chosen by atomicCAS(core[v], -1, k).
//  * Inside a warp the arcs of up to 32 items are processed edge-balanced:
//    lanes take consecutive arcs of the concatenated lists, 16 arcs per lane
//    in flight, so loads of the adjacency, of d~ and the decrements overlap.
//  * A warp keeps at most `lq_cap` vertices that dropped to k in its local
//    queue (the rest go to the global queue), so no warp hoards a burst.
//  * Every wait is bounded by a wall-clock limit (globaltimer); on expiry the
//    kernel records KCORE_ERR_TIMEOUT and returns.
#include <climits>

#include "kcore_device.cuh"
#include "kcore_peel.h"

namespace kc {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / kWarp;
constexpr int kTileItems = 8;  // active-list entries per thread per scan tile
constexpr int kIlp = 16;       // arcs per lane in flight per iteration
constexpr unsigned long long kEmpty = ~0ull;
// Work item: bits 0-31 vertex, 32-58 slice index, 59 "whole vertex, not yet
// split", 60-63 round tag. kEmpty is never a valid item (vertex ids < 2^31).
constexpr unsigned long long kWhole = 1ull << 59;

__device__ __forceinline__ unsigned long long item_tag(int r) {
  return (unsigned long long)(r & 0xf) << 60;
}
__device__ __forceinline__ unsigned long long make_slice_item(int v, long long slice, int r) {
  return (unsigned long long)(unsigned)v | ((unsigned long long)slice << 32) | item_tag(r);
}
__device__ __forceinline__ unsigned long long make_whole_item(int v, int r) {
  return (unsigned long long)(unsigned)v | kWhole | item_tag(r);
}

struct PeelShared {
  int excl[kWarps][kWarp];
  long long a0[kWarps][kWarp];
  unsigned long long lq[kWarps][kLocalQueueMax];
  int lqn[kWarps];
  unsigned long long scan_part[kWarps];
  unsigned long long tile_base_a;
  unsigned long long tile_base_q;
  int tile_qok;
  int red_min[kWarps];
  unsigned long long red_found[kWarps];
  int rflag;  // 0 running, 1 round finished, 2 abort
};

struct RoundCtx {
  RoundRec* R;
  int r;
  int t;                          // level of this round
  unsigned long long base;        // first queue slot of this round's segment
  unsigned long long all_tokens;  // scanning CTAs << 40
};

__device__ __forceinline__ void set_status(PeelCtl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

// Adds a token or releases finished items; if this update finishes the round,
// publish the round's results on every broadcast line.
__device__ __forceinline__ void finish_update(const PeelArgs& a, const RoundCtx& rc,
                                              unsigned long long delta) {
  unsigned long long old = atomicAdd(&rc.R->cnt, delta);
  if (a.trace && (delta >> 40) && ((old + delta) >> 40) == (rc.all_tokens >> 40))
    a.trace[(size_t)rc.r * kTraceFields + 1] = globaltimer_ns();
  if (old + delta == rc.all_tokens) {
    __threadfence();
    unsigned long long found = ld_relaxed_u64(&rc.R->found);
    unsigned long long alen = ld_relaxed_u64(&rc.R->alen);
    unsigned long long tail = ld_relaxed_u64(&rc.R->tail);
    int minkey = ld_relaxed_s32(&rc.R->minkey);
    for (int i = 0; i < kDoneLines; i++) {
      a.ctl->done[i].found = found;
      a.ctl->done[i].alen = alen;
      a.ctl->done[i].tail = tail;
      a.ctl->done[i].minkey = minkey;
    }
    __threadfence();
    for (int i = 0; i < kDoneLines; i++) atomicExch(&a.ctl->done[i].round, rc.r + 1);
    if (a.trace) {
      unsigned long long* tr = a.trace + (size_t)rc.r * kTraceFields;
      tr[2] = globaltimer_ns();
      tr[3] = (unsigned long long)rc.t;
      tr[5] = found;
      tr[6] = tail;
    }
  }
}

// Appends `cnt` items per lane (warp-aggregated) to the round's queue
// segment; item i of a lane is make(i). The round counter is raised before any
// of the items can be seen.
template <typename MakeItem>
__device__ __forceinline__ void push_global(const PeelArgs& a, const RoundCtx& rc, long long cnt,
                                            int lane, MakeItem make) {
  long long incl = warp_incl_scan(cnt, lane);
  long long tot = __shfl_sync(kFull, incl, 31);
  if (tot == 0) return;
  unsigned long long pos0 = 0;
  if (lane == 31) {
    atomicAdd(&rc.R->cnt, (unsigned long long)tot);
    pos0 = atomicAdd(&rc.R->tail, (unsigned long long)tot);
    __threadfence();
  }
  pos0 = __shfl_sync(kFull, pos0, 31);
  if (rc.base + pos0 + (unsigned long long)tot > (unsigned long long)a.qcap) {
    if (lane == 0) set_status(a.ctl, ST_CAPACITY);
    return;
  }
  unsigned long long pos = rc.base + pos0 + (unsigned long long)(incl - cnt);
  for (long long i = 0; i < cnt; i++) a.Q[pos + i] = make(i);
}

// Pushes the vertices u of the lanes with `flag` set as whole items: into this
// warp's local queue while it holds fewer than lq_cap, the rest to the round's
// global queue segment.
__device__ __forceinline__ void push_vertices(const PeelArgs& a, PeelShared& sh,
                                              const RoundCtx& rc, bool flag, int u, int warp,
                                              int lane) {
  unsigned fm = __ballot_sync(kFull, flag);
  if (!fm) return;
  int lqn = sh.lqn[warp];
  int room = max(a.lq_cap - lqn, 0);
  int rank = __popc(fm & lanemask_lt());
  bool to_local = flag && rank < room;
  if (to_local) sh.lq[warp][lqn + rank] = (unsigned long long)(unsigned)u | kWhole;
  int nloc = min(__popc(fm), room);
  __syncwarp();
  if (lane == 0) sh.lqn[warp] = lqn + nloc;
  __syncwarp();
  if (__popc(fm) <= room) return;
  bool to_glob = flag && !to_local;
  push_global(a, rc, to_glob ? 1 : 0, lane, [&](long long) { return make_whole_item(u, rc.r); });
}

// Processes up to 32 work items (one per lane < c). A whole-vertex item whose
// list is longer than one slice first queues its other slices. Then every arc
// v->u of the items' slices decrements d~[u] when u is still above level t;
// the decrement returning t+1 lands u on t, claims it for level t and pushes it.
__device__ __forceinline__ void process_batch_body(const PeelArgs& a, PeelShared& sh,
                                                   const RoundCtx& rc, unsigned long long item,
                                                   int c, int warp, int lane) {
  const int t = rc.t;
  long long a0 = 0, nsplit = 0;
  int len = 0, v = 0;
  if (lane < c) {
    v = (int)(unsigned)(item & 0xffffffffull);
    long long sl = (long long)((item >> 32) & 0x7ffffffull);
    long long o0 = a.off[v], o1 = a.off[v + 1];
    if (item & kWhole) {
      long long nsl = (o1 - o0 + a.slice - 1) / a.slice;
      nsplit = nsl > 1 ? nsl - 1 : 0;
      sl = 0;
    }
    a0 = o0 + sl * a.slice;
    long long e = min(o1, a0 + (long long)a.slice);
    len = (int)max(e - a0, 0ll);
  }
  // queue the remaining slices of long lists first (other warps take them)
  if (__any_sync(kFull, nsplit > 0))
    push_global(a, rc, nsplit, lane, [&](long long i) { return make_slice_item(v, i + 1, rc.r); });
  int incl = warp_incl_scan(len, lane);
  int total = __shfl_sync(kFull, incl, 31);
  sh.excl[warp][lane] = incl - len;
  sh.a0[warp][lane] = a0;
  __syncwarp();
  const int* excl = sh.excl[warp];
  if (a.trace && lane == 0) atomicAdd(a.trace + (size_t)rc.r * kTraceFields + 8, (unsigned long long)total);
  for (int base = 0; base < total; base += kWarp * kIlp) {
    int u[kIlp];
    // item of the first arc of this lane, then step forward (arcs increase with q)
    int j = base + lane;
    int idx = 0;
    {
      int lo = 0, hi = c;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (excl[mid] <= j) lo = mid + 1;
        else hi = mid;
      }
      idx = lo > 0 ? lo - 1 : 0;
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++, j += kWarp) {
      u[q] = -1;
      if (j < total) {
        while (idx + 1 < c && excl[idx + 1] <= j) idx++;
        u[q] = ld_stream_s32(a.adj + sh.a0[warp][idx] + (j - excl[idx]));
      }
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++) {
      if (u[q] >= 0 && (unsigned long long)(unsigned)u[q] >= (unsigned long long)a.n) {
        set_status(a.ctl, ST_NOT_SIMPLE);  // neighbour id out of range: skip it
        u[q] = -1;
      }
    }
    int dq[kIlp];
#pragma unroll
    for (int q = 0; q < kIlp; q++) dq[q] = u[q] >= 0 ? __ldcg(a.deg + u[q]) : INT_MIN;
    unsigned cross = 0;
    int ndec = 0;
#pragma unroll
    for (int q = 0; q < kIlp; q++) {
      if (dq[q] > t) {
        ndec++;
        if (atomicSub(a.deg + u[q], 1) == t + 1) cross |= 1u << q;
      }
    }
    if (a.trace) {
      int wd = warp_sum(ndec);
      if (lane == 0 && wd) atomicAdd(a.trace + (size_t)rc.r * kTraceFields + 9, (unsigned long long)wd);
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++)
      if ((cross >> q) & 1u)
        if (atomicCAS(a.core + u[q], -1, t) != -1) cross &= ~(1u << q);
    if (__any_sync(kFull, cross != 0)) {
#pragma unroll
      for (int q = 0; q < kIlp; q++) push_vertices(a, sh, rc, (cross >> q) & 1u, u[q], warp, lane);
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void process_batch(const PeelArgs& a, PeelShared& sh,
                                              const RoundCtx& rc, unsigned long long item, int c,
                                              int warp, int lane) {
  if (!a.trace) {
    process_batch_body(a, sh, rc, item, c, warp, lane);
    return;
  }
  uint64_t t0 = globaltimer_ns();
  process_batch_body(a, sh, rc, item, c, warp, lane);
  if (lane == 0) {
    unsigned long long* tr = a.trace + (size_t)rc.r * kTraceFields;
    atomicAdd(tr + 12, (unsigned long long)(globaltimer_ns() - t0));
    atomicAdd(tr + 13, 1ull);
  }
}

// Scan of one round: active-list entries [lo, hi) of this CTA. Round 0 reads
// the degrees from the offsets (and initialises d~ and core); later rounds
// read d~. Entries above t survive into the next active list, entries equal
// to t are claimed for level t and pushed, entries below t were peeled earlier
// and are dropped.
__device__ void scan_share(const PeelArgs& a, PeelShared& sh, const RoundCtx& rc,
                           const int* Ain, int* Aout, long long lo, long long hi,
                           unsigned long long* found_out, int* min_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = rc.r, t = rc.t;
  unsigned long long found = 0;
  int dmin = INT_MAX;
  for (long long tile = lo; tile < hi; tile += (long long)kBlock * kTileItems) {
    int v[kTileItems], d[kTileItems];
    unsigned char st[kTileItems];  // 0 none, 1 survivor, 2 claimed frontier vertex
    int cs = 0;
    long long ps = 0;
#pragma unroll
    for (int q = 0; q < kTileItems; q++) {
      long long i = tile + (long long)q * kBlock + tid;
      st[q] = 0;
      v[q] = -1;
      d[q] = 0;
      if (i < hi) {
        v[q] = Ain ? Ain[i] : (int)i;
        if (r == 0) {
          long long o0 = a.off[v[q]], o1 = a.off[v[q] + 1];
          if (o0 < 0 || o1 < o0 || o1 > a.m || o1 - o0 >= a.n) {
            set_status(a.ctl, ST_NOT_SIMPLE);  // malformed offsets: stop before any arc is read
            o1 = o0 = 0;
          }
          d[q] = (int)(o1 - o0);
          a.deg[v[q]] = d[q];
          a.core[v[q]] = d[q] == t ? t : -1;
          if (d[q] == t) found++;  // degree-0 vertices at level 0: nothing to push
          else st[q] = 1;
        } else {
          d[q] = ld_relaxed_s32(a.deg + v[q]);
          if (d[q] > t) {
            st[q] = 1;
          } else if (d[q] == t) {
            if (atomicCAS(a.core + v[q], -1, t) == -1) {
              st[q] = 2;
              found++;
            }
          }
        }
      }
      if (st[q] == 1) {
        cs++;
        dmin = min(dmin, d[q]);
      }
      if (st[q] == 2) ps++;
    }
    // block exclusive scan of (ps << 32 | cs)
    unsigned long long packed = ((unsigned long long)ps << 32) | (unsigned)cs;
    unsigned long long incl = warp_incl_scan(packed, lane);
    if (lane == 31) sh.scan_part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long x = lane < kWarps ? sh.scan_part[lane] : 0;
      unsigned long long xi = warp_incl_scan(x, lane);
      if (lane < kWarps) sh.scan_part[lane] = xi - x;
      if (lane == kWarps - 1) {
        unsigned long long tot_c = xi & 0xffffffffull, tot_p = xi >> 32;
        sh.tile_base_a = tot_c ? atomicAdd(&rc.R->alen, tot_c) : 0;
        sh.tile_qok = 1;
        sh.tile_base_q = 0;
        if (tot_p) {
          atomicAdd(&rc.R->cnt, tot_p);
          sh.tile_base_q = rc.base + atomicAdd(&rc.R->tail, tot_p);
          __threadfence();
          if (sh.tile_base_q + tot_p > (unsigned long long)a.qcap) {
            set_status(a.ctl, ST_CAPACITY);
            sh.tile_qok = 0;
          }
        }
      }
    }
    __syncthreads();
    unsigned long long ex = sh.scan_part[warp] + incl - packed;
    unsigned long long pa = sh.tile_base_a + (ex & 0xffffffffull);
    unsigned long long pq = sh.tile_base_q + (ex >> 32);
    bool qok = sh.tile_qok != 0;
#pragma unroll
    for (int q = 0; q < kTileItems; q++) {
      if (st[q] == 1) Aout[pa++] = v[q];
      if (st[q] == 2 && qok) a.Q[pq++] = make_whole_item(v[q], r);
    }
    __syncthreads();
  }
  unsigned long long fw = warp_sum(found);
  int mw = warp_min(dmin);
  if (lane == 0) {
    sh.red_found[warp] = fw;
    sh.red_min[warp] = mw;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long f = 0;
    int mn = INT_MAX;
    for (int w = 0; w < kWarps; w++) {
      f += sh.red_found[w];
      mn = min(mn, sh.red_min[w]);
    }
    *found_out = f;
    *min_out = mn;
  }
}

// Work loop of one warp for one round. Returns 1 when the round has finished,
// 2 on abort (time limit or error status).
__device__ int process_round(const PeelArgs& a, PeelShared& sh, const RoundCtx& rc,
                             unsigned long long& my_items, unsigned long long& my_local,
                             unsigned& local_batches) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long tag = item_tag(rc.r);
  const DoneLine* dl = &a.ctl->done[blockIdx.x % kDoneLines];
  int held = 0;
  bool have = false;
  unsigned long long tk = 0, tk_end = 0;
  uint64_t idle_t0 = 0;
  unsigned long long last_cnt = ~0ull, last_pg = ~0ull;
  unsigned polls = 0;
  for (;;) {
    int lqn = sh.lqn[warp];
    __syncwarp();
    if (lqn > 0) {
      int take = min(lqn, kWarp);
      unsigned long long item = lane < take ? sh.lq[warp][lqn - take + lane] : 0;
      __syncwarp();
      if (lane == 0) sh.lqn[warp] = lqn - take;
      __syncwarp();
      process_batch(a, sh, rc, item, take, warp, lane);
      if (lane == 0) {
        my_local += take;
        // heartbeat: a long chain kept inside one warp still shows progress
        if (((++local_batches) & 63) == 0) atomicAdd(&a.ctl->progress, 1ull);
      }
      continue;
    }
    if (held) {
      __threadfence();
      __syncwarp();
      if (lane == 0) finish_update(a, rc, (unsigned long long)(-(long long)held));
      held = 0;
    }
    if (!have) {
      unsigned long long h = 0, take = 1;
      if (lane == 0) {
        unsigned long long tl = ld_relaxed_u64(&rc.R->tail), hd = ld_relaxed_u64(&rc.R->head);
        unsigned long long av = tl > hd ? tl - hd : 0;
        take = av / (unsigned long long)a.take_div;
        if (take < 1) take = 1;
        if (take > (unsigned long long)a.max_take) take = a.max_take;
        h = atomicAdd(&rc.R->head, take);
      }
      tk = __shfl_sync(kFull, h, 0);
      tk_end = tk + __shfl_sync(kFull, take, 0);
      have = true;
    }
    // items present at the front of this warp's tickets
    unsigned long long item = 0;
    bool rdy = false;
    unsigned long long want = tk_end - tk < 32 ? tk_end - tk : 32;
    if ((unsigned long long)lane < want) {
      unsigned long long slot = rc.base + tk + lane;
      if (slot < (unsigned long long)a.qcap) {
        item = ld_relaxed_u64(a.Q + slot);
        rdy = item != kEmpty && (item & (0xfull << 60)) == tag;
      }
    }
    unsigned rm = __ballot_sync(kFull, rdy);
    int c = rm == kFull ? 32 : __ffs(~rm) - 1;
    if (c > 0) {
      process_batch(a, sh, rc, item, c, warp, lane);
      held += c;
      tk += c;
      if (tk == tk_end) have = false;
      if (lane == 0) my_items += c;
      idle_t0 = 0;
      continue;
    }
    // idle: one poller per CTA (warp 0) watches the round's broadcast line
    int flag = *(volatile int*)&sh.rflag;
    if (flag) return flag;
    if (warp == 0) {
      int f = 0;
      if (lane == 0) {
        if (ld_acquire_s32(&dl->round) > rc.r) {
          f = 1;
        } else if (((++polls) & 31) == 0) {
          if (ld_relaxed_s32(&a.ctl->status) != 0) {
            f = 2;
          } else {
            uint64_t now = globaltimer_ns();
            unsigned long long cn = ld_relaxed_u64(&rc.R->cnt);
            unsigned long long pg = ld_relaxed_u64(&a.ctl->progress);
            if (idle_t0 == 0 || cn != last_cnt || pg != last_pg) {
              idle_t0 = now;
              last_cnt = cn;
              last_pg = pg;
            } else if (now - idle_t0 > a.timeout_ns) {
              set_status(a.ctl, ST_TIMEOUT);
              f = 2;
            }
          }
        }
        if (f) *(volatile int*)&sh.rflag = f;
      }
      f = __shfl_sync(kFull, f, 0);
      if (f) return f;
      __nanosleep(a.poll_sleep_ns);
    } else {
      __nanosleep(a.idle_sleep_ns);
    }
  }
}

__global__ void __launch_bounds__(kBlock, 4) peel_persistent(PeelArgs a) {
  __shared__ PeelShared sh;
  __shared__ unsigned long long s_found;
  __shared__ int s_min;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (lane == 0) sh.lqn[warp] = 0;
  unsigned long long my_items = 0, my_local = 0;
  unsigned local_batches = 0;

  int t = 0, r = 0, kmax = 0;
  unsigned long long base = 0;
  long long len = a.n;
  long long rounds = 0, empty_rounds = 0, scanned = 0;
  for (;;) {
    if (r >= a.max_rounds) {
      if (tid == 0) set_status(a.ctl, ST_CAPACITY);
      break;
    }
    long long nscan = (len + a.scan_min - 1) / a.scan_min;
    if (nscan < 1) nscan = 1;
    if (nscan > gridDim.x) nscan = gridDim.x;
    RoundCtx rc{a.rounds + r, r, t, base, (unsigned long long)nscan << 40};
    const int* Ain = r == 0 ? nullptr : ((r - 1) & 1 ? a.A1 : a.A0);
    int* Aout = (r & 1) ? a.A1 : a.A0;
    if (tid == 0) sh.rflag = 0;
    uint64_t my_start = 0;
    if (a.trace && tid == 0) {
      my_start = globaltimer_ns();
      if (blockIdx.x == 0) {
        a.trace[(size_t)r * kTraceFields + 0] = my_start;
        a.trace[(size_t)r * kTraceFields + 4] = (unsigned long long)len;
        a.trace[(size_t)r * kTraceFields + 7] = (unsigned long long)nscan;
      }
    }
    __syncthreads();
    scanned += len;

    // ---- scan (frontier extraction + active-set refinement)
    if (blockIdx.x < nscan) {
      long long lo = len * (long long)blockIdx.x / nscan;
      long long hi = len * (long long)(blockIdx.x + 1) / nscan;
      scan_share(a, sh, rc, Ain, Aout, lo, hi, &s_found, &s_min);
      __threadfence();
      __syncthreads();
      if (a.trace && tid == 0)
        atomicMax(a.trace + (size_t)r * kTraceFields + 10, (unsigned long long)(globaltimer_ns() - my_start));
      if (tid == 0) {
        if (s_found) atomicAdd(&rc.R->found, s_found);
        if (s_min != INT_MAX) atomicMax(&rc.R->minkey, INT_MAX - s_min);
        __threadfence();
        // Test hook (host-set option): CTA 0 withholds its round-1 token, so
        // the round can never finish and every waiting warp must hit its limit.
        if (!(a.inject_stall && blockIdx.x == 0 && r == 1)) finish_update(a, rc, 1ull << 40);
      }
    }

    if (a.trace && tid == 0 && blockIdx.x != 0) {
      unsigned long long s0 = ld_relaxed_u64(a.trace + (size_t)r * kTraceFields + 0);
      if (s0 && my_start > s0) atomicMax(a.trace + (size_t)r * kTraceFields + 11, (unsigned long long)(my_start - s0));
    }
    // ---- processing until the round's counter says everything is done
    int res = process_round(a, sh, rc, my_items, my_local, local_batches);
    if (res == 2) *(volatile int*)&sh.rflag = 2;
    __syncthreads();
    if (sh.rflag == 2) break;

    // ---- round end: next level from the broadcast results
    const DoneLine* dl = &a.ctl->done[blockIdx.x % kDoneLines];
    unsigned long long found = ld_relaxed_u64(&dl->found);
    unsigned long long alen = ld_relaxed_u64(&dl->alen);
    unsigned long long tail = ld_relaxed_u64(&dl->tail);
    int minkey = ld_relaxed_s32(&dl->minkey);
    rounds++;
    if (found) kmax = t;
    else empty_rounds++;
    if (alen == 0) break;
    t = found ? t + 1 : INT_MAX - minkey;
    base += tail;
    len = (long long)alen;
    r++;
  }
  // ---- results and counters
  if (lane == 0) {
    if (my_items) atomicAdd(&a.ctl->items, my_items);
    if (my_local) atomicAdd(&a.ctl->local_items, my_local);
  }
  if (blockIdx.x == 0 && tid == 0) {
    *a.kmax_out = a.n > 0 ? kmax : 0;
    a.ctl->rounds = rounds;
    a.ctl->empty_rounds = empty_rounds;
    a.ctl->scanned = scanned;
    a.ctl->kmax = kmax;
  }
}

}  // namespace kc

// ---------------------------------------------------------------- host side
namespace kc {

int peel_max_ctas_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, peel_persistent, kBlock, 0) != cudaSuccess)
    return 0;
  return nb;
}

int peel_block_size() { return kBlock; }

cudaError_t peel_launch(const PeelArgs& args, int grid, cudaStream_t stream) {
  PeelArgs a = args;
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)peel_persistent, dim3(grid), dim3(kBlock), params,
                                     0, stream);
}

}  // namespace kc
