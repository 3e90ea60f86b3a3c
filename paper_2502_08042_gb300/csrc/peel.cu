// Single-graph k-core peel for sm_103a: one persistent cooperative kernel.
//
// What it computes: Algorithm 1 (the round structure: frontier = live vertices
// whose induced degree equals the level k, then refine the active set to the
// vertices above k) with the online Peel of Algorithm 3 (atomic decrement of a
// neighbour's induced degree; the decrement that returns k+1 is the one that
// lands it on k and puts it into the same level's work).
//
// How it is organised on the GPU (no per-subround barrier):
//  * Levels ("rounds") are separated by a device-wide termination counter per
//    round, cnt = (scan tokens << 40) + (work items pushed - items finished).
//    Every CTA adds one token after scanning its share of the active list; the
//    round is over when cnt == grid << 40. Subrounds never synchronise: work
//    items flow through one append-only global queue (each vertex enters it
//    once over the whole run, as in Theorem 1's proof) and through per-warp
//    local queues in shared memory (the role vertical granularity control,
//    Sec. 4.2, gives its local FIFO: a vertex that drops to k is processed by
//    the same worker without waiting for a new subround).
//  * Empty levels are skipped: the scan of the level after k speculates on
//    k+1; if no vertex sits at k+1 the scan's minimum over the surviving
//    induced degrees is the next level (the min search of the framework's
//    "k <- k+1" made exact).
//  * The scan of level k+1 overlaps the processing of level k+1 (a frontier
//    vertex found by one CTA is peeled while other CTAs still scan). A vertex
//    can then be found both by the scan and by a crossing decrement, so the
//    single owner is chosen by atomicCAS(core[v], -1, k).
//  * Long adjacency lists are split into slices of `slice` arcs, so the arcs
//    of a hub vertex are spread over many warps; inside a warp, the arcs of up
//    to 32 items are processed edge-balanced (each lane takes consecutive arc
//    indices of the concatenated lists).
//  * Every wait is bounded by a wall-clock limit (globaltimer); on expiry the
//    kernel records KCORE_ERR_TIMEOUT and returns.
#include <climits>

#include "kcore_device.cuh"
#include "kcore_peel.h"

namespace kc {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / kWarp;
constexpr int kTileItems = 4;  // active-list entries per thread per scan tile
constexpr int kIlp = 4;        // arcs per lane in flight per iteration
constexpr unsigned long long kEmpty = ~0ull;

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
};

__device__ __forceinline__ void set_status(PeelCtl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

// Pushes the vertices u of the lanes with `flag` set: one-slice vertices go to
// this warp's local queue while it has room; the rest are appended to the
// global queue as slices (round counter raised before the items appear).
__device__ __forceinline__ void push_vertices(const PeelArgs& a, PeelShared& sh, RoundRec* R,
                                              bool flag, int u, int warp, int lane) {
  unsigned any = __ballot_sync(kFull, flag);
  if (!any) return;
  long long nsl = 0;
  if (flag) {
    long long o0 = a.off[u], o1 = a.off[u + 1];
    nsl = (o1 - o0 + a.slice - 1) / a.slice;
  }
  bool local_ok = flag && nsl == 1;
  unsigned lm = __ballot_sync(kFull, local_ok);
  int lqn = sh.lqn[warp];
  int room = a.lq_cap - lqn;
  int rank = __popc(lm & lanemask_lt());
  bool to_local = local_ok && rank < room;
  if (to_local) sh.lq[warp][lqn + rank] = (unsigned long long)(unsigned)u;
  int nloc = min(__popc(lm), max(room, 0));
  __syncwarp();
  if (lane == 0) sh.lqn[warp] = lqn + nloc;
  __syncwarp();
  bool to_glob = flag && !to_local;
  long long gsl = to_glob ? nsl : 0;
  long long gincl = warp_incl_scan(gsl, lane);
  long long gtot = __shfl_sync(kFull, gincl, 31);
  if (gtot == 0) return;
  unsigned long long base = 0;
  if (lane == 31) {
    atomicAdd(&R->cnt, (unsigned long long)gtot);
    base = atomicAdd(&a.ctl->qtail, (unsigned long long)gtot);
    __threadfence();
  }
  base = __shfl_sync(kFull, base, 31);
  if (base + (unsigned long long)gtot > (unsigned long long)a.qcap) {
    if (lane == 0) set_status(a.ctl, ST_CAPACITY);
    return;
  }
  if (to_glob) {
    unsigned long long pos = base + (unsigned long long)(gincl - gsl);
    for (long long s = 0; s < nsl; s++)
      a.Q[pos + s] = ((unsigned long long)s << 32) | (unsigned)u;
  }
}

// Processes up to 32 work items (one per lane < c): every arc v->u of the
// items' slices decrements d~[u] when u is still above level t; the decrement
// returning t+1 claims u for level t and pushes it.
__device__ __forceinline__ void process_batch(const PeelArgs& a, PeelShared& sh, RoundRec* R,
                                              unsigned long long item, int c, int t, int warp,
                                              int lane) {
  long long a0 = 0;
  int len = 0;
  if (lane < c) {
    int v = (int)(unsigned)(item & 0xffffffffull);
    long long sl = (long long)(item >> 32);
    long long o0 = a.off[v], o1 = a.off[v + 1];
    a0 = o0 + sl * a.slice;
    long long e = min(o1, a0 + (long long)a.slice);
    len = (int)(e - a0);
  }
  int incl = warp_incl_scan(len, lane);
  int total = __shfl_sync(kFull, incl, 31);
  sh.excl[warp][lane] = incl - len;
  sh.a0[warp][lane] = a0;
  __syncwarp();
  const int* excl = sh.excl[warp];
  for (int base = 0; base < total; base += kWarp * kIlp) {
    int u[kIlp];
    bool cross[kIlp];
#pragma unroll
    for (int q = 0; q < kIlp; q++) {
      int j = base + q * kWarp + lane;
      u[q] = -1;
      if (j < total) {
        int lo = 0, hi = c;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (excl[mid] <= j) lo = mid + 1;
          else hi = mid;
        }
        int idx = lo - 1;
        u[q] = ld_stream_s32(a.adj + sh.a0[warp][idx] + (j - excl[idx]));
        if ((unsigned long long)(unsigned)u[q] >= (unsigned long long)a.n) {
          set_status(a.ctl, ST_NOT_SIMPLE);  // neighbour id out of range: skip it
          u[q] = -1;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++) {
      cross[q] = false;
      if (u[q] >= 0) {
        int d = __ldcg(a.deg + u[q]);
        if (d > t) cross[q] = atomicSub(a.deg + u[q], 1) == t + 1;
      }
    }
#pragma unroll
    for (int q = 0; q < kIlp; q++)
      if (cross[q]) cross[q] = atomicCAS(a.core + u[q], -1, t) == -1;
#pragma unroll
    for (int q = 0; q < kIlp; q++) push_vertices(a, sh, R, cross[q], u[q], warp, lane);
  }
  __syncwarp();
}

// Waits (bounded) until a reserved queue slot has been written.
__device__ __forceinline__ bool wait_item(const PeelArgs& a, unsigned long long* slot,
                                          unsigned long long* out) {
  unsigned long long v = ld_relaxed_u64(slot);
  if (v != kEmpty) {
    *out = v;
    return true;
  }
  uint64_t t0 = globaltimer_ns();
  for (;;) {
    __nanosleep(32);
    v = ld_relaxed_u64(slot);
    if (v != kEmpty) {
      *out = v;
      return true;
    }
    if (globaltimer_ns() - t0 > a.timeout_ns) {
      set_status(a.ctl, ST_TIMEOUT);
      return false;
    }
    if (ld_relaxed_s32(&a.ctl->status) != 0) return false;
  }
}

// Scan of round r at target level t: active-list entries [lo, hi) of this CTA.
// Round 0 reads the degrees from the offsets (and initialises d~ and core);
// later rounds read d~. Entries above t survive into the next active list,
// entries equal to t are claimed for level t and pushed, entries below t were
// peeled earlier and are dropped.
__device__ void scan_share(const PeelArgs& a, PeelShared& sh, RoundRec* R, int r, int t,
                           const int* Ain, int* Aout, long long lo, long long hi,
                           unsigned long long* found_out, int* min_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long found = 0;
  int dmin = INT_MAX;
  for (long long tile = lo; tile < hi; tile += (long long)kBlock * kTileItems) {
    int v[kTileItems], d[kTileItems];
    unsigned char st[kTileItems];  // 0 none, 1 survivor, 2 claimed frontier
    long long nsl[kTileItems];
    int cs = 0;
    long long ps = 0;
#pragma unroll
    for (int q = 0; q < kTileItems; q++) {
      long long i = tile + (long long)q * kBlock + tid;
      st[q] = 0;
      nsl[q] = 0;
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
              long long o0 = a.off[v[q]], o1 = a.off[v[q] + 1];
              nsl[q] = (o1 - o0 + a.slice - 1) / a.slice;
            }
          }
        }
      }
      if (st[q] == 1) {
        cs++;
        dmin = min(dmin, d[q]);
      }
      ps += nsl[q];
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
        sh.tile_base_a = tot_c ? atomicAdd(&R->alen, tot_c) : 0;
        sh.tile_qok = 1;
        if (tot_p) {
          atomicAdd(&R->cnt, tot_p);
          sh.tile_base_q = atomicAdd(&a.ctl->qtail, tot_p);
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
      if (st[q] == 2 && qok) {
        for (long long s = 0; s < nsl[q]; s++)
          a.Q[pq + s] = ((unsigned long long)s << 32) | (unsigned)v[q];
        pq += nsl[q];
      }
    }
    __syncthreads();
  }
  // block reductions of found and min
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

__global__ void __launch_bounds__(kBlock) peel_persistent(PeelArgs a) {
  __shared__ PeelShared sh;
  __shared__ unsigned long long s_found;
  __shared__ int s_min;
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long all_tokens = (unsigned long long)gridDim.x << 40;
  if (lane == 0) sh.lqn[warp] = 0;
  unsigned long long my_items = 0, my_local = 0;
  unsigned local_batches = 0;

  int t = 0, r = 0, kmax = 0;
  long long rounds = 0, empty_rounds = 0, scanned = 0;
  for (;;) {
    if (r >= a.max_rounds) {
      if (tid == 0) set_status(a.ctl, ST_CAPACITY);
      break;
    }
    RoundRec* R = a.rounds + r;
    long long len = r == 0 ? a.n : (long long)ld_acquire_u64(&a.rounds[r - 1].alen);
    const int* Ain = r == 0 ? nullptr : ((r - 1) & 1 ? a.A1 : a.A0);
    int* Aout = (r & 1) ? a.A1 : a.A0;
    long long lo = len * (long long)blockIdx.x / gridDim.x;
    long long hi = len * (long long)(blockIdx.x + 1) / gridDim.x;
    scanned += len;

    // ---- scan (frontier extraction + active-set refinement)
    scan_share(a, sh, R, r, t, Ain, Aout, lo, hi, &s_found, &s_min);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      if (s_found) atomicAdd(&R->found, s_found);
      if (s_min != INT_MAX) atomicMax(&R->minkey, INT_MAX - s_min);
      __threadfence();
      // Test hook (host-set option): CTA 0 withholds its round-1 token, so the
      // round can never end and every waiting warp must hit its time limit.
      if (!(a.inject_stall && blockIdx.x == 0 && r == 1)) atomicAdd(&R->cnt, 1ull << 40);
    }

    // ---- processing until the round's counter says everything is done
    int held = 0;
    uint64_t idle_t0 = 0;
    unsigned long long last_cnt = 0, last_progress = 0;
    int backoff = 32;
    bool abort = false;
    for (;;) {
      int lqn = sh.lqn[warp];
      __syncwarp();
      if (lqn > 0) {
        int take = min(lqn, kWarp);
        unsigned long long item = lane < take ? sh.lq[warp][lqn - take + lane] : 0;
        __syncwarp();
        if (lane == 0) sh.lqn[warp] = lqn - take;
        __syncwarp();
        process_batch(a, sh, R, item, take, t, warp, lane);
        my_local += take;
        // heartbeat: a long chain kept inside one warp still shows progress
        if (lane == 0 && ((++local_batches) & 63) == 0) atomicAdd(&a.ctl->progress, 1ull);
        continue;
      }
      if (held) {
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(&R->cnt, (unsigned long long)(-(long long)held));
        held = 0;
      }
      unsigned long long base = 0;
      int got = 0;
      if (lane == 0) {
        for (;;) {
          unsigned long long tail = ld_relaxed_u64(&a.ctl->qtail);
          unsigned long long head = ld_relaxed_u64(&a.ctl->qhead);
          if (head >= tail) break;
          unsigned long long avail = tail - head;
          unsigned long long take = avail / (unsigned long long)a.take_div;
          if (take < 1) take = 1;
          if (take > (unsigned long long)a.max_take) take = a.max_take;
          if (atomicCAS(&a.ctl->qhead, head, head + take) == head) {
            base = head;
            got = (int)take;
            break;
          }
        }
      }
      got = __shfl_sync(kFull, got, 0);
      base = __shfl_sync(kFull, base, 0);
      if (got > 0) {
        held = got;
        my_items += got;
        idle_t0 = 0;
        backoff = 32;
        for (int o = 0; o < got; o += kWarp) {
          int c = min(kWarp, got - o);
          unsigned long long item = 0;
          bool ok = true;
          if (lane < c) ok = wait_item(a, a.Q + base + o + lane, &item);
          if (!__all_sync(kFull, ok)) {
            abort = true;
            break;
          }
          process_batch(a, sh, R, item, c, t, warp, lane);
        }
        if (abort) break;
        continue;
      }
      // idle: round over?
      int done = 0;
      if (lane == 0) {
        unsigned long long c = ld_acquire_u64(&R->cnt);
        if (c == all_tokens) {
          done = 1;
        } else if (ld_relaxed_s32(&a.ctl->status) != 0) {
          done = 2;
        } else {
          uint64_t now = globaltimer_ns();
          unsigned long long pg = ld_relaxed_u64(&a.ctl->progress);
          if (idle_t0 == 0 || c != last_cnt || pg != last_progress) {
            idle_t0 = now;
            last_cnt = c;
            last_progress = pg;
          } else if (now - idle_t0 > a.timeout_ns) {
            set_status(a.ctl, ST_TIMEOUT);
            done = 2;
          }
        }
      }
      done = __shfl_sync(kFull, done, 0);
      if (done == 1) break;
      if (done == 2) {
        abort = true;
        break;
      }
      __nanosleep(backoff);
      backoff = min(backoff * 2, a.max_backoff_ns);
    }
    if (tid == 0) s_flag = 0;
    __syncthreads();
    if (abort) s_flag = 1;
    __syncthreads();
    if (s_flag) break;
    if (ld_relaxed_s32(&a.ctl->status) != 0) break;

    // ---- round end: next level
    unsigned long long found = ld_acquire_u64(&R->found);
    unsigned long long alen = ld_acquire_u64(&R->alen);
    int minkey = ld_acquire_s32(&R->minkey);
    rounds++;
    if (found) kmax = t;
    else empty_rounds++;
    if (alen == 0) break;
    t = found ? t + 1 : INT_MAX - minkey;
    r++;
  }
  // ---- results and counters
  unsigned long long wi = warp_sum(my_items), wl = warp_sum(my_local);
  if (lane == 0) {
    if (wi) atomicAdd(&a.ctl->items, wi);
    if (wl) atomicAdd(&a.ctl->local_items, wl);
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
