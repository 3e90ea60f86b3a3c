// CSR build on sm_103a: edge list -> simple undirected CSR.
//
// The paper symmetrises directed inputs (Sec. 6.1, "Datasets"); the peel needs
// a simple graph. Steps, all on the device:
//   1. keys: each pair (a, b) with a != b gives the arcs a->b and b->a as
//      integers (a << B) | b with B = bits of n-1; self-loops and ids out of
//      range become a sentinel that sorts last (ids out of range also set an
//      error status). The keys are not stored: the first radix pass (which
//      need not be stable) makes them from the edge arrays as it reads them.
//   2. stable LSD radix sort of the keys over their 2B significant bits, 8-bit
//      digits. Each CTA owns a contiguous chunk; a pass is an upsweep (digit
//      histogram per CTA), a scan of each digit's row of the 256 x CTAs
//      histogram (one CTA per digit), and a downsweep that ranks each
//      2,048-key tile in shared memory and writes runs of equal digits
//      contiguously, while the next tile arrives by asynchronous copy
//      (cp.async). A key's rank within its warp and digit comes from one pass:
//      the lanes holding a digit elect a leader (warp match), which adds their
//      number to the warp's counter for that digit and hands the old value on.
//   3. unique + emit: keys equal to their predecessor are dropped; the rest
//      are written in order as adj[] (low B bits), and the first arc of each
//      source vertex fixes offsets[] (vertices without arcs take the next
//      vertex's offset). Keys are read striped (a warp reads 32 consecutive
//      keys), the predecessor comes from the next lower lane, and the
//      positions from warp ballots, so no key passes through shared memory.
// A single graph takes a shorter route through steps 1-3: each pair (a, b)
// with a != b gives ONE key (min << B) | max; sorting these E keys by both
// fields gives every vertex's upper neighbours in order (A), and a stable
// sort of A by its low B bits (the larger endpoint) gives every vertex's
// lower neighbours in order (B). A vertex's list is its lower neighbours
// followed by its upper ones, both ascending, so emission writes the CSR from
// A and B directly: 2B + B digit passes over E keys instead of 2B over 2E.
// Repeats stay in A as adjacent equal keys and are dropped on emission; the
// first pass of B's sort drops them (and the sentinels), and the rest of B's
// buffer holds sentinels written beforehand, which every stable pass keeps
// behind the real keys.
//
// Lists come out ascending and duplicate-free, the canonical form of the CPU
// builder, so the two are comparable bit for bit.
#include <climits>

#include "kcore_csr.h"
#include "kcore_device.cuh"

namespace kc {

constexpr int kCsrBlock = 256;
constexpr int kKeysPerThread = 8;
constexpr int kTile = kCsrBlock * kKeysPerThread;  // 2048
constexpr unsigned long long kSentinel = ~0ull;

// Keys (source << Bd) | target. Single graph: ids in [0, n), source = id.
// Batch (gv != nullptr): edge i belongs to the graph g with eoff[g] <= i <
// eoff[g+1]; its ids are graph-local in [0, gv[g+1] - gv[g]); the source part
// is the global id gv[g] + local, the target part stays local.
struct EdgeList {
  const int* src;
  const int* dst;
  long long n;
  int Bd;
  const long long* gv;
  const long long* eoff;
  long long G;
  int* status;
};

// a batch: the last graph g in [glo, ghi) with eoff[g] <= i
__device__ __forceinline__ long long graph_of(const EdgeList& es, long long i, long long glo, long long ghi) {
  long long lo = glo, hi = ghi;
  while (hi - lo > 1) {
    const long long mid = (lo + hi) >> 1;
    if (es.eoff[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// a batch: the graphs [*glo, *ghi) that hold edges [e0, e1) (a CTA's chunk;
// one binary search each for its first and last edge, by thread 0, shared
// through *glo / *ghi in shared memory; the caller synchronises)
__device__ __forceinline__ void chunk_graphs(const EdgeList& es, long long e0, long long e1, long long* glo,
                                             long long* ghi) {
  if (threadIdx.x == 0) {
    *glo = es.gv && e0 < e1 ? graph_of(es, e0, 0, es.G) : 0;
    *ghi = es.gv && e0 < e1 ? graph_of(es, e1 - 1, *glo, es.G) + 1 : es.G;
  }
}

// the arcs of edge i = (a, b): keys 2i (a -> b) and 2i + 1 (b -> a); a batch's
// edge i lies in one of the graphs [glo, ghi)
__device__ __forceinline__ void edge_keys(const EdgeList& es, long long i, int a, int b, unsigned long long& k0,
                                          unsigned long long& k1, long long glo = 0, long long ghi = 0) {
  long long base = 0, lim = es.n;
  if (es.gv) {
    const long long g = ghi - glo == 1 ? glo : graph_of(es, i, glo, ghi > glo ? ghi : es.G);
    base = es.gv[g];
    lim = es.gv[g + 1] - base;
  }
  k0 = k1 = kSentinel;
  if ((unsigned long long)(unsigned)a >= (unsigned long long)lim ||
      (unsigned long long)(unsigned)b >= (unsigned long long)lim) {
    atomicCAS(es.status, 0, 1);
  } else if (a != b) {
    k0 = ((unsigned long long)(base + a) << es.Bd) | (unsigned long long)b;
    k1 = ((unsigned long long)(base + b) << es.Bd) | (unsigned long long)a;
  }
}

// a single graph's edge i = (a, b) as one key (min << B) | max
__device__ __forceinline__ unsigned long long edge_canon(const EdgeList& es, int a, int b) {
  if ((unsigned long long)(unsigned)a >= (unsigned long long)es.n ||
      (unsigned long long)(unsigned)b >= (unsigned long long)es.n) {
    atomicCAS(es.status, 0, 1);
    return kSentinel;
  }
  if (a == b) return kSentinel;
  const unsigned lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
  return ((unsigned long long)lo << es.Bd) | (unsigned long long)hi;
}

// Where a pass's keys come from: a key array, the edge list as two arcs per
// edge (the first pass of the general build), the edge list as one key per
// edge (the first pass of a single graph's build), or a sorted key array
// without its sentinels and without keys equal to their predecessor (the
// first pass of B's sort).
enum KeySrc : int { kKeys = 0, kArcs = 1, kCanon = 2, kKeysDrop = 3 };

// digit of a pass: bits [shift, shift + 8) of the key, masked by dmask (the
// last pass over a field narrower than a multiple of 8 bits keeps only its bits)
__device__ __forceinline__ int digit_of(unsigned long long k, int shift, int dmask) {
  return (int)((k >> shift) & (unsigned long long)dmask);
}

// Per-CTA digit histogram of its chunk: hist[d * G + g]. kArcs: the keys are
// made from the edge list, two per edge (chunks hold whole edges: chunk and lo
// are even); kCanon: one per edge.
template <int kSrc>
__global__ void __launch_bounds__(kCsrBlock) rs_upsweep(const unsigned long long* keys, EdgeList es,
                                                        long long N, long long chunk, int shift, int dmask,
                                                        unsigned* hist) {
  __shared__ unsigned cnt[kCsrBlock / 32][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (kCsrBlock / 32) * 256; i += kCsrBlock) (&cnt[0][0])[i] = 0;
  __syncthreads();
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  if constexpr (kSrc == kCanon) {
    constexpr int kU = 4;
    for (long long e0 = lo + tid; e0 < hi; e0 += kU * kCsrBlock) {
      int a[kU], b[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const long long e = e0 + u * kCsrBlock;
        a[u] = e < hi ? __ldcs(es.src + e) : 0;
        b[u] = e < hi ? __ldcs(es.dst + e) : 0;
      }
#pragma unroll
      for (int u = 0; u < kU; u++)
        if (e0 + u * kCsrBlock < hi) atomicAdd(&cnt[warp][digit_of(edge_canon(es, a[u], b[u]), shift, dmask)], 1u);
    }
  } else if constexpr (kSrc == kArcs) {
    __shared__ long long cg_lo, cg_hi;
    chunk_graphs(es, lo / 2, hi > lo ? hi / 2 : lo / 2, &cg_lo, &cg_hi);
    __syncthreads();
    const long long glo = cg_lo, ghi = cg_hi;
    constexpr int kU = 4;  // edges per thread per step, loaded before any count
    for (long long e0 = lo / 2 + tid; e0 < hi / 2; e0 += kU * kCsrBlock) {
      int a[kU], b[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const long long e = e0 + u * kCsrBlock;
        a[u] = e < hi / 2 ? __ldcs(es.src + e) : 0;
        b[u] = e < hi / 2 ? __ldcs(es.dst + e) : 0;
      }
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const long long e = e0 + u * kCsrBlock;
        if (e < hi / 2) {
          unsigned long long k0, k1;
          edge_keys(es, e, a[u], b[u], k0, k1, glo, ghi);
          atomicAdd(&cnt[warp][digit_of(k0, shift, dmask)], 1u);
          atomicAdd(&cnt[warp][digit_of(k1, shift, dmask)], 1u);
        }
      }
    }
  } else if constexpr (kSrc == kKeysDrop) {
    for (long long i = lo + tid; i < hi; i += kCsrBlock) {
      const unsigned long long x = keys[i], p = i > 0 ? keys[i - 1] : kSentinel;
      if (x != kSentinel && x != p) atomicAdd(&cnt[warp][digit_of(x, shift, dmask)], 1u);
    }
  } else {
    for (long long i = lo + tid; i < hi; i += kCsrBlock) atomicAdd(&cnt[warp][digit_of(keys[i], shift, dmask)], 1u);
  }
  __syncthreads();
  unsigned s = 0;
  for (int w = 0; w < kCsrBlock / 32; w++) s += cnt[w][tid];
  hist[(long long)tid * gridDim.x + blockIdx.x] = s;
}

// Exclusive scans of uint32 rows into uint64: CTA r (1024 threads) scans
// in[r * len, (r + 1) * len) into out[] at the same place and, if totals is
// given, writes the row's sum to totals[r].
__global__ void __launch_bounds__(1024) scan_u32_to_u64(const unsigned* in, unsigned long long* out,
                                                        long long len, unsigned long long* totals) {
  __shared__ unsigned long long part[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  in += (long long)blockIdx.x * len;
  out += (long long)blockIdx.x * len;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < len; base += 1024) {
    long long i = base + tid;
    unsigned long long x = i < len ? in[i] : 0;
    unsigned long long incl = warp_incl_scan(x, lane);
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long p = part[lane];
      unsigned long long pi = warp_incl_scan(p, lane);
      part[lane] = pi - p;
    }
    __syncthreads();
    unsigned long long c = carry;
    if (i < len) out[i] = c + part[warp] + incl - x;
    __syncthreads();
    if (tid == 1023) carry = c + part[warp] + incl;
    __syncthreads();
  }
  if (totals && tid == 0) totals[blockIdx.x] = carry;
}

// Stable scatter of one radix pass. Each CTA walks its chunk tile by tile, in
// order. offs[d * G + g] counts the keys of digit d in the chunks before g,
// rowtot[d] all keys of digit d; so the CTA's first key of digit d goes after
// every key of a smaller digit and the digit-d keys of earlier chunks.
// kArcs / kCanon: the first pass, whose keys are made from the edge list (a
// tile is 1,024 edges / 2,048 edges; the order within a tile does not matter
// in the first pass).
// Pos: the type of an output position (32 bits when there are at most 2^32
// keys: positions are then computed modulo 2^32).
static_assert(kCsrBlock == 256, "one thread per 8-bit digit");
template <int kSrc, typename Pos>
__global__ void __launch_bounds__(kCsrBlock, 5) rs_downsweep(const unsigned long long* in, EdgeList es,
                                                          unsigned long long* out, long long N,
                                                          long long chunk, int shift, int dmask,
                                                          const unsigned long long* offs,
                                                          const unsigned long long* rowtot) {
  __shared__ unsigned long long buf[kTile];
  __shared__ __align__(16) unsigned long long stage[kTile];  // the next tile, copied asynchronously
  __shared__ unsigned wcnt[kCsrBlock / 32][256];  // keys per (warp, digit), then their tile offsets
  __shared__ Pos dstb[256];  // output position of the tile's first key of digit d, minus its tile offset
  __shared__ unsigned long long part64[kCsrBlock / 32];
  __shared__ unsigned part[kCsrBlock / 32];
  __shared__ unsigned tile_keys;  // keys of the tile that are written (all but kKeysDrop's dropped ones)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const unsigned lt = lanemask_lt();
  // run: where this CTA's next key of digit tid goes
  unsigned long long run;
  {
    const unsigned long long rt = rowtot[tid];
    const unsigned long long incl = warp_incl_scan(rt, lane);
    if (lane == 31) part64[warp] = incl;
    for (int i = tid; i < (kCsrBlock / 32) * 256; i += kCsrBlock) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    unsigned long long before = 0;
    for (int w = 0; w < warp; w++) before += part64[w];
    run = before + incl - rt + offs[(long long)tid * G + blockIdx.x];
  }
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  __shared__ long long cg_lo, cg_hi;  // kArcs, a batch: the graphs of this chunk's edges
  if constexpr (kSrc == kArcs) {
    chunk_graphs(es, lo / 2, hi > lo ? hi / 2 : lo / 2, &cg_lo, &cg_hi);
    __syncthreads();
  }
  // 16-byte asynchronous copies of a tile's keys into `stage` (pairs of keys;
  // a last odd key is copied with its neighbour, which lies inside the
  // key buffer and is not used). kArcs / kCanon: the tile's sources and
  // targets go to the stage's two halves (4 KB each for kArcs, 8 KB for
  // kCanon), by 16-byte copies when both arrays are 16-byte aligned and the
  // tile is whole, else by 4-byte copies (nothing past the last edge is read).
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(stage);
  const bool al16 =
      ((reinterpret_cast<unsigned long long>(es.src) | reinterpret_cast<unsigned long long>(es.dst)) & 15) == 0;
  auto prefetch = [&](long long t0) {
    const long long tn = min((long long)kTile, hi - t0);
    if constexpr (kSrc == kArcs || kSrc == kCanon) {
      constexpr int kE = kSrc == kArcs ? kTile / 2 : kTile;  // edges per tile
      constexpr unsigned kHalf = 4u * kE;                     // bytes of one array's share
      const long long e0 = kSrc == kArcs ? t0 / 2 : t0, ne = kSrc == kArcs ? tn / 2 : tn;
      if (al16 && ne == kE) {
        for (int c = tid; 4 * c < kE; c += kCsrBlock) {
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * c), "l"(es.src + e0 + 4 * c)
                       : "memory");
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + kHalf + 16u * c),
                       "l"(es.dst + e0 + 4 * c)
                       : "memory");
        }
      } else {
        for (int c = tid; c < ne; c += kCsrBlock) {
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sbase + 4u * c), "l"(es.src + e0 + c)
                       : "memory");
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sbase + kHalf + 4u * c), "l"(es.dst + e0 + c)
                       : "memory");
        }
      }
    } else {
      for (int c = tid; 2 * c < tn; c += kCsrBlock)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * c), "l"(in + t0 + 2 * c)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (lo < hi) prefetch(lo);
  for (long long ts = lo; ts < hi; ts += kTile) {
    const long long tn = min((long long)kTile, hi - ts);
    unsigned long long k[kKeysPerThread];
    unsigned rk[kKeysPerThread / 2];  // ranks below 2,048: two per word
    // key it of this thread is key j_of(it) of the tile (kArcs: arc it & 1 of
    // the tile's edge el_of(it); kCanon: edge j_of(it)); 256 is the digit of no key
    auto j_of = [&](int it) { return warp * (kKeysPerThread * 32) + it * 32 + lane; };
    auto el_of = [&](int it) { return warp * (kKeysPerThread * 16) + (it >> 1) * 32 + lane; };
    unsigned dropped = 0;  // kKeysDrop: bit it set for a dropped key
    auto valid = [&](int it) {
      return kSrc == kArcs ? el_of(it) < tn / 2 : (j_of(it) < tn && !((dropped >> it) & 1u));
    };
    auto dg_of = [&](int it) { return valid(it) ? digit_of(k[it], shift, dmask) : 256; };
    const unsigned long long pre = kSrc == kKeysDrop && tid == 0 && ts > 0 ? in[ts - 1] : kSentinel;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if constexpr (kSrc == kCanon) {
      const int* sa = reinterpret_cast<const int*>(stage);
#pragma unroll
      for (int it = 0; it < kKeysPerThread; it++)
        k[it] = valid(it) ? edge_canon(es, sa[j_of(it)], sa[kTile + j_of(it)]) : 0;
    } else if constexpr (kSrc == kArcs) {
      const int* sa = reinterpret_cast<const int*>(stage);
#pragma unroll
      for (int it = 0; it < kKeysPerThread; it += 2) {
        k[it] = k[it + 1] = 0;
        if (valid(it))
          edge_keys(es, ts / 2 + el_of(it), sa[el_of(it)], sa[1024 + el_of(it)], k[it], k[it + 1], cg_lo, cg_hi);
      }
    } else {
#pragma unroll
      for (int it = 0; it < kKeysPerThread; it++) k[it] = j_of(it) < tn ? stage[j_of(it)] : 0;
      if constexpr (kSrc == kKeysDrop) {
#pragma unroll
        for (int it = 0; it < kKeysPerThread; it++) {
          const int j = j_of(it);
          const unsigned long long p = j > 0 ? stage[j - 1] : pre;
          if (j < tn && (k[it] == kSentinel || k[it] == p)) dropped |= 1u << it;
        }
      }
    }
    __syncthreads();  // the stage is read: copy the next tile into it
    if (ts + kTile < hi) prefetch(ts + kTile);
    // rank within (warp, digit) in key order: iterations in order, lanes in
    // order within an iteration
#pragma unroll
    for (int it = 0; it < kKeysPerThread; it++) {
      const int dg = dg_of(it);
      const unsigned peers = __match_any_sync(kFull, dg);
      const int leader = __ffs(peers) - 1;
      unsigned old = 0;
      if (lane == leader && dg < 256) old = atomicAdd(&wcnt[warp][dg], (unsigned)__popc(peers));
      old = __shfl_sync(kFull, old, leader);
      const unsigned r = old + __popc(peers & lt);
      if (it & 1) rk[it >> 1] |= r << 16;
      else rk[it >> 1] = r;
    }
    __syncthreads();
    // per digit (thread d): tile count, exclusive offsets over digits, then
    // over warps
    unsigned tc = 0;
    for (int w = 0; w < kCsrBlock / 32; w++) tc += wcnt[w][tid];
    unsigned incl = warp_incl_scan(tc, lane);
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned p = lane < kCsrBlock / 32 ? part[lane] : 0;
      unsigned pi = warp_incl_scan(p, lane);
      if (lane < kCsrBlock / 32) part[lane] = pi - p;
    }
    __syncthreads();
    const unsigned lo_d = part[warp] + incl - tc;
    unsigned acc = lo_d;
    for (int w = 0; w < kCsrBlock / 32; w++) {
      unsigned c = wcnt[w][tid];
      wcnt[w][tid] = acc;
      acc += c;
    }
    dstb[tid] = (Pos)(run - lo_d);  // modulo 2^64 (2^32): adding a tile offset of digit tid lands at or after run
    run += tc;
    if (tid == 255) tile_keys = lo_d + tc;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kKeysPerThread; it++) {
      const int dg = dg_of(it);
      if (dg < 256) buf[wcnt[warp][dg] + ((rk[it >> 1] >> (16 * (it & 1))) & 0xffffu)] = k[it];
    }
    __syncthreads();
    for (int w = 0; w < kCsrBlock / 32; w++) wcnt[w][tid] = 0;  // for the next tile
    const int tk = (int)tile_keys;
    for (int j = tid; j < tk; j += kCsrBlock) {
      const unsigned long long key = buf[j];
      out[(unsigned long long)(Pos)(dstb[digit_of(key, shift, dmask)] + (Pos)j)] = key;
    }
  }
}

// A tile is kRows rows of kCsrBlock consecutive keys; a thread takes one key
// per row (a warp 32 consecutive keys). A key's neighbours come from
// the next lower and higher lanes; at a warp's edges from the keys the
// neighbouring warps publish in shared memory, and at the tile's edges from
// the keys just before and after it (read by threads 0 and kCsrBlock - 1).
template <int kRows>
struct TileEdges {
  unsigned long long first[kRows][kCsrBlock / 32];
  unsigned long long last[kRows][kCsrBlock / 32];
};

template <int kRows>
__device__ __forceinline__ void publish_edges(TileEdges<kRows>& e, const unsigned long long* x, int lane, int warp) {
#pragma unroll
  for (int q = 0; q < kRows; q++) {
    if (lane == 0) e.first[q][warp] = x[q];
    if (lane == 31) e.last[q][warp] = x[q];
  }
}

// predecessor of this thread's key in row q (pre: the key before the tile, held by thread 0)
template <int kRows>
__device__ __forceinline__ unsigned long long pred_key(const TileEdges<kRows>& e, unsigned long long xq, int q, int lane,
                                                       int warp, unsigned long long pre) {
  const unsigned long long up = __shfl_up_sync(kFull, xq, 1);
  if (lane > 0) return up;
  if (warp > 0) return e.last[q][warp - 1];
  return q > 0 ? e.last[q - 1][kCsrBlock / 32 - 1] : pre;
}

// successor (post: the key after the tile, held by thread kCsrBlock - 1)
template <int kRows>
__device__ __forceinline__ unsigned long long succ_key(const TileEdges<kRows>& e, unsigned long long xq, int q, int lane,
                                                       int warp, unsigned long long post) {
  const unsigned long long dn = __shfl_down_sync(kFull, xq, 1);
  if (lane < 31) return dn;
  if (warp < kCsrBlock / 32 - 1) return e.first[q][warp + 1];
  return q < kRows - 1 ? e.first[q + 1][0] : post;
}

// Unique keys of each CTA chunk (a key differing from its predecessor).
__global__ void __launch_bounds__(kCsrBlock, 5) csr_count_unique(const unsigned long long* k, long long N,
                                                              long long chunk, unsigned* cnt) {
  constexpr int kRows = kKeysPerThread;
  __shared__ TileEdges<kRows> edges;
  __shared__ unsigned part[kCsrBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  unsigned c = 0;
  for (long long ts = lo; ts < hi; ts += kTile) {
    unsigned long long x[kRows];
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      x[q] = i < hi ? __ldcs(k + i) : kSentinel;
    }
    const unsigned long long pre = tid == 0 && ts > 0 ? __ldcg(k + ts - 1) : kSentinel;
    publish_edges(edges, x, lane, warp);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      const unsigned long long p = pred_key(edges, x[q], q, lane, warp, pre);
      if (i < hi && x[q] != kSentinel && (i == 0 || p != x[q])) c++;
    }
    __syncthreads();  // the edges are read: the next tile may publish its own
  }
  c = warp_sum(c);
  if (lane == 0) part[warp] = c;
  __syncthreads();
  if (tid == 0) {
    unsigned s = 0;
    for (int w = 0; w < kCsrBlock / 32; w++) s += part[w];
    cnt[blockIdx.x] = s;
  }
}

// Ordered emission of the unique keys. A unique key's position ("before":
// unique keys ahead of it) is the chunk's base, plus the unique keys of
// earlier rows and of earlier warps in its row (one warp scans the tile's rows
// x warps counts), plus those of lower lanes (a ballot). A key's group is its
// high field (the source, or the smaller endpoint).
//   kEmitAll: adj[pos] = low B bits; the first arc of each source fixes
//     offsets[] for that source and every source without arcs just below it;
//     the last arc fills the offsets of the sources above it.
//   kEmitUpper (sequence A): vertex u's upper neighbours go after its lower
//     ones: adj[pos + starts[u + 1]] = larger endpoint, and offsets[x] = A's
//     unique keys with smaller endpoint below x (csr_finish_offsets adds
//     starts[x]); m = twice A's unique keys.
enum EmitMode : int { kEmitAll = 0, kEmitUpper = 2 };
template <int kMode>
__global__ void __launch_bounds__(kCsrBlock, 5) csr_emit(const unsigned long long* __restrict__ k, long long N,
                                                      long long chunk, int B, long long n,
                                                      const unsigned long long* __restrict__ base,
                                                      int* __restrict__ adj, long long* __restrict__ off,
                                                      long long* __restrict__ m_out,
                                                      unsigned long long* __restrict__ starts,
                                                      long long* __restrict__ tail) {
  constexpr int kW = kCsrBlock / 32;
  constexpr int kRows = 4;  // a tile of kRows * kCsrBlock keys (chunks are whole tiles of either size)
  constexpr int kT = kRows * kCsrBlock;
  static_assert(kRows * kW == 32 && kTile % kT == 0, "the tile's counts are scanned by one warp, one per lane");
  __shared__ TileEdges<kRows> edges;
  __shared__ unsigned cnt[kRows * kW];  // unique keys per (row, warp), then their offsets in the tile
  __shared__ unsigned tile_total;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long mask = (1ull << B) - 1;
  const unsigned lt = lanemask_lt();
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  unsigned long long running = base[blockIdx.x];
  for (long long ts = lo; ts < hi; ts += kT) {
    unsigned long long x[kRows];
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      x[q] = i < hi ? __ldcs(k + i) : kSentinel;
    }
    const unsigned long long pre = tid == 0 && ts > 0 ? __ldcg(k + ts - 1) : kSentinel;
    // chunks are whole tiles, so a key past the tile's end lies in the next chunk or past N
    const unsigned long long post = tid == kCsrBlock - 1 && ts + kT < N ? __ldcg(k + ts + kT) : kSentinel;
    publish_edges(edges, x, lane, warp);
    __syncthreads();
    unsigned bal[kRows];
    int ps[kRows];  // source of the predecessor (-1: none)
    unsigned closing = 0;    // bit q: the key of row q is the last valid key
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      const unsigned long long p = pred_key(edges, x[q], q, lane, warp, pre);
      const unsigned long long sk = succ_key(edges, x[q], q, lane, warp, post);  // every lane: a shuffle
      const unsigned long long nx = i + 1 < N ? sk : kSentinel;
      const bool valid = i < hi && x[q] != kSentinel;
      ps[q] = (i == 0 || p == kSentinel) ? -1 : (int)(p >> B);
      if (valid && nx == kSentinel) closing |= 1u << q;
      bal[q] = __ballot_sync(kFull, valid && (i == 0 || p != x[q]));
      if (lane == q) mine = __popc(bal[q]);
    }
    if (lane < kRows) cnt[lane * kW + warp] = mine;
    __syncthreads();
    if (warp == 0) {
      const unsigned c0 = cnt[lane];
      const unsigned incl = warp_incl_scan(c0, lane);
      cnt[lane] = incl - c0;
      if (lane == 31) tile_total = incl;
    }
    // the lookups of each unique key, all issued before any store
    unsigned long long look0[kRows];
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      look0[q] = 0;
      if ((bal[q] >> lane) & 1u) {
        if constexpr (kMode == kEmitUpper) {
          const long long u = (long long)(x[q] >> B);
          look0[q] = starts[u + 1];  // the lower neighbours of u come first
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRows; q++) {
      const bool u = (bal[q] >> lane) & 1u;
      const unsigned long long before = running + cnt[q * kW + warp] + __popc(bal[q] & lt);
      const long long hi_f = (long long)(x[q] >> B), lo_f = (long long)(x[q] & mask);
      const long long s = hi_f;  // the key's group
      if (u) {
        if constexpr (kMode == kEmitAll) {
          adj[before] = (int)lo_f;
          for (long long v = (long long)ps[q] + 1; v <= s; v++) off[v] = (long long)before;
        } else {
          adj[before + look0[q]] = (int)lo_f;
          for (long long v = (long long)ps[q] + 1; v <= s; v++) off[v] = (long long)before;
        }
      }
      // the last valid key (unique or a repeat) closes the groups above its own
      if ((closing >> q) & 1u) {
        const long long m_val = (long long)before + (u ? 1 : 0);
        if constexpr (kMode == kEmitAll) {
          for (long long v = s + 1; v <= n; v++) off[v] = m_val;
          *m_out = m_val;
        } else {
          // the groups above the last one are finished by csr_finish_offsets
          tail[0] = s;
          tail[1] = m_val;
          *m_out = 2 * m_val;
        }
      }
    }
    running += tile_total;
  }
}

// Sequence B: its E' = tail[1] keys, unique and ordered by (larger, smaller)
// endpoint, then sentinels. starts[x] = keys of B whose larger endpoint is
// below x, for x in [0, n] (cleared beforehand: the groups up to the first key's
// need no store; the last key records its group in tail[0] and E' in tail[1]).
__global__ void csr_lower_starts(const unsigned long long* __restrict__ Bq, long long E, int B, long long n,
                                 unsigned long long* __restrict__ starts, long long* __restrict__ tail) {
  constexpr int kU = 4;  // keys per thread per step, all loaded first
  const unsigned long long mask = (1ull << B) - 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < E; i0 += kU * stride) {
    unsigned long long x[kU], xp[kU], xn[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const long long i = i0 + u * stride;
      x[u] = i < E ? __ldcs(Bq + i) : kSentinel;
      xp[u] = i < E && i > 0 ? __ldg(Bq + i - 1) : kSentinel;
      xn[u] = i + 1 < E ? __ldg(Bq + i + 1) : kSentinel;
    }
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const long long i = i0 + u * stride;
      if (x[u] == kSentinel) continue;
      const long long g = (long long)(x[u] & mask);
      if (i > 0) {
        const long long gp = (long long)(xp[u] & mask);  // a key: sentinels only follow the keys
        for (long long v = gp + 1; v <= g; v++) starts[v] = (unsigned long long)i;
      }
      if (xn[u] == kSentinel) {
        tail[0] = g;
        tail[1] = i + 1;
      }
    }
  }
}

// starts[v] = E' for the groups above the last key's group s = tail[0], in parallel.
__global__ void csr_fill_starts(const long long* __restrict__ tail, long long n,
                                unsigned long long* __restrict__ starts) {
  const long long s = tail[0], m_val = tail[1];
  for (long long v = s + 1 + blockIdx.x * (long long)blockDim.x + threadIdx.x; v <= n;
       v += (long long)gridDim.x * blockDim.x)
    starts[v] = (unsigned long long)m_val;
}

// The lower neighbours: B's key i (u, v) is v's (i - starts[v])-th lower
// neighbour, and v's list opens with them.
__global__ void csr_lower_emit(const unsigned long long* __restrict__ Bq, long long E, int B,
                               const long long* __restrict__ off, const unsigned long long* __restrict__ starts,
                               int* __restrict__ adj) {
  constexpr int kU = 4;  // keys per thread per step, all loaded first, then all their lookups
  const unsigned long long mask = (1ull << B) - 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < E; i0 += kU * stride) {
    unsigned long long x[kU], at[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const long long i = i0 + u * stride;
      x[u] = i < E ? __ldcs(Bq + i) : kSentinel;
    }
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const long long v = (long long)(x[u] & mask);
      at[u] = x[u] != kSentinel ? (unsigned long long)__ldg(off + v) - __ldg(starts + v) : 0;
    }
#pragma unroll
    for (int u = 0; u < kU; u++)
      if (x[u] != kSentinel) adj[at[u] + (unsigned long long)(i0 + u * stride)] = (int)(x[u] >> B);
  }
}

// offsets[v] = (A's unique keys with smaller endpoint below v) + starts[v]:
// csr_emit<kEmitUpper> wrote the first term for v up to the last valid key's
// group tail[0]; above it the term is tail[1], A's unique keys in all.
__global__ void csr_finish_offsets(const long long* __restrict__ tail, long long n, long long* __restrict__ off,
                                   const unsigned long long* __restrict__ starts) {
  const long long s = tail[0], m_val = tail[1];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v <= n; v += (long long)gridDim.x * blockDim.x)
    off[v] = (v > s ? m_val : off[v]) + (long long)starts[v];
}

// ------------------------------------------------------------------ host side
static int bits_for(long long n) {
  int B = 1;
  while ((1ll << B) < n) B++;
  return B;
}

CsrLayout csr_layout(long long n, long long E, int sms, long long max_graph_n) {
  CsrLayout L{};
  long long N = 2 * E;
  // five CTAs per SM, each sorting 2,048-key tiles with the next tile copied
  // into shared memory while the current one is ranked (43 KB of shared
  // memory, which admits five; registers held to five CTAs' worth by the
  // kernels' launch bounds): resident warps and loads in flight count. Measured on R-MAT 24 (ms per build): 2 CTAs x
  // 4,096-key tiles 56.8, 4 x 4,096 37.7, 6 x 2,048 35.6, 7 x 2,048 38.2,
  // 8 x 1,536 37.3; with the asynchronous copy 5 x 2,048 31.0, 4 x 2,048 31.8
  long long G = (long long)sms * 5;
  long long tiles = (N + kTile - 1) / kTile;
  if (tiles < G) G = tiles < 1 ? 1 : tiles;
  L.grid = (int)G;
  auto chunk_of = [&](long long keys) {
    long long c = (keys + G - 1) / G;
    c = (c + kTile - 1) / kTile * kTile;
    return c < kTile ? (long long)kTile : c;
  };
  L.chunk = chunk_of(N);
  L.chunk1 = chunk_of(E);
  L.N = N;
  L.Bs = bits_for(n);
  // batched: one spare code so that no valid (local) target has all bits set
  // and a valid key can never equal the sentinel in the sorted bits
  L.B = max_graph_n > 0 ? bits_for(max_graph_n + 1) : L.Bs;
  size_t off = 0;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  L.status = off;
  off = al(off + 256);
  // two spare keys per buffer: a single graph's build keeps two sequences of
  // E keys per buffer, the second from an even index, and a 16-byte copy may
  // read the key after a sequence's last
  L.keys0 = off;
  off = al(off + 8 * (size_t)(N + 2));
  L.keys1 = off;
  off = al(off + 8 * (size_t)(N + 2));
  L.hist = off;
  off = al(off + 4 * 256 * (size_t)G);
  L.offs = off;
  off = al(off + 8 * 256 * (size_t)G);
  L.rowtot = off;
  off = al(off + 8 * 256);
  L.starts = off;  // a single graph's build: starts of the lower-neighbour lists
  off = al(off + (max_graph_n > 0 ? 8 : 8 * (size_t)(n + 1)));
  L.total = off;
  return L;
}

cudaError_t csr_build_launch(const CsrLayout& L, char* ws, long long n, long long E, const int* src,
                             const int* dst, const long long* gv, const long long* eoff, long long ngraphs,
                             long long* off_out, int* adj_out, long long* m_out, cudaStream_t stream) {
  cudaError_t e;
  int* status = (int*)(ws + L.status);
  unsigned long long* k0 = (unsigned long long*)(ws + L.keys0);
  unsigned long long* k1 = (unsigned long long*)(ws + L.keys1);
  unsigned* hist = (unsigned*)(ws + L.hist);
  unsigned long long* offs = (unsigned long long*)(ws + L.offs);
  unsigned long long* rowtot = (unsigned long long*)(ws + L.rowtot);
  if ((e = cudaMemsetAsync(status, 0, 256, stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(off_out, 0, 8 * (size_t)(n + 1), stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(m_out, 0, 8, stream)) != cudaSuccess) return e;
  if (E == 0) return cudaSuccess;
  const int G = L.grid;
  const EdgeList es{src, dst, n, L.B, gv, eoff, ngraphs, status};
  // one radix pass: upsweep, row scans, downsweep (32-bit positions when the
  // keys number at most 2^32)
  auto pass = [&](int src_kind, const unsigned long long* in, unsigned long long* out, long long N, long long chunk,
                  int shift, int dmask) {
#define KC_UP(S) rs_upsweep<S><<<G, kCsrBlock, 0, stream>>>(in, es, N, chunk, shift, dmask, hist)
    switch (src_kind) {
      case kKeys: KC_UP(kKeys); break;
      case kArcs: KC_UP(kArcs); break;
      case kCanon: KC_UP(kCanon); break;
      default: KC_UP(kKeysDrop); break;
    }
#undef KC_UP
    scan_u32_to_u64<<<256, 1024, 0, stream>>>(hist, offs, G, rowtot);
    const bool narrow = N <= (1ll << 32);
#define KC_DOWN(S, P) rs_downsweep<S, P><<<G, kCsrBlock, 0, stream>>>(in, es, out, N, chunk, shift, dmask, offs, rowtot)
    switch (src_kind) {
      case kKeys: narrow ? KC_DOWN(kKeys, unsigned) : KC_DOWN(kKeys, unsigned long long); break;
      case kArcs: narrow ? KC_DOWN(kArcs, unsigned) : KC_DOWN(kArcs, unsigned long long); break;
      case kCanon: narrow ? KC_DOWN(kCanon, unsigned) : KC_DOWN(kCanon, unsigned long long); break;
      default: narrow ? KC_DOWN(kKeysDrop, unsigned) : KC_DOWN(kKeysDrop, unsigned long long); break;
    }
#undef KC_DOWN
  };
  if (!gv) {
    // a single graph: A = the E edge keys sorted by (min, max); B = A stably
    // sorted by max. A ping-pongs between the first halves of the two key
    // buffers, B between their second halves (from an even index: 16-byte
    // copies stay aligned)
    const long long off2 = (E + 1) / 2 * 2;
    unsigned long long *a0 = k0, *a1 = k1, *b0 = k0 + off2, *b1 = k1 + off2;
    const int passes_a = (2 * L.B + 7) / 8;
    for (int p = 0; p < passes_a; p++) {
      pass(p == 0 ? kCanon : kKeys, a0, a1, E, L.chunk1, 8 * p, 0xff);
      std::swap(a0, a1);
    }
    const unsigned long long* A = a0;
    // B: A without sentinels and repeats, stably by the larger endpoint; the
    // first pass writes E' <= E keys over a buffer of sentinels
    if ((e = cudaMemsetAsync(b1, 0xff, 8 * (size_t)E, stream)) != cudaSuccess) return e;
    const int passes_b = (L.B + 7) / 8;
    for (int p = 0; p < passes_b; p++) {
      const int bits = std::min(8, L.B - 8 * p);
      pass(p == 0 ? kKeysDrop : kKeys, p == 0 ? A : b0, b1, E, L.chunk1, 8 * p, (1 << bits) - 1);
      std::swap(b0, b1);
    }
    const unsigned long long* Bq = b0;
    unsigned long long* starts = (unsigned long long*)(ws + L.starts);
    // B's last key's group and E' (0, 0 when no key is valid: the fills then
    // write what the cleared arrays hold)
    long long* tail = (long long*)(ws + L.status + 64);
    const int fill_grid = (int)std::min<long long>((n + kCsrBlock) / kCsrBlock, 4 * (long long)G);
    const int key_grid = (int)std::min<long long>((E + 4 * kCsrBlock - 1) / (4 * kCsrBlock), 8 * (long long)G);
    if ((e = cudaMemsetAsync(starts, 0, 8 * (size_t)(n + 1), stream)) != cudaSuccess) return e;
    csr_lower_starts<<<key_grid, kCsrBlock, 0, stream>>>(Bq, E, L.B, n, starts, tail);
    csr_fill_starts<<<fill_grid, kCsrBlock, 0, stream>>>(tail, n, starts);
    csr_count_unique<<<G, kCsrBlock, 0, stream>>>(A, E, L.chunk1, hist);
    scan_u32_to_u64<<<1, 1024, 0, stream>>>(hist, offs, G, nullptr);
    csr_emit<kEmitUpper><<<G, kCsrBlock, 0, stream>>>(A, E, L.chunk1, L.B, n, offs, adj_out, off_out, m_out,
                                                     starts, tail);
    csr_finish_offsets<<<fill_grid, kCsrBlock, 0, stream>>>(tail, n, off_out, starts);
    csr_lower_emit<<<key_grid, kCsrBlock, 0, stream>>>(Bq, E, L.B, off_out, starts, adj_out);
    return cudaGetLastError();
  }
  // a batch: two arcs per edge, sorted by (global source, local target)
  const long long N = L.N;
  const int passes = (L.Bs + L.B + 7) / 8;
  for (int p = 0; p < passes; p++) {
    pass(p == 0 ? kArcs : kKeys, k0, k1, N, L.chunk, 8 * p, 0xff);
    std::swap(k0, k1);
  }
  csr_count_unique<<<G, kCsrBlock, 0, stream>>>(k0, N, L.chunk, hist);
  scan_u32_to_u64<<<1, 1024, 0, stream>>>(hist, offs, G, nullptr);
  csr_emit<kEmitAll><<<G, kCsrBlock, 0, stream>>>(k0, N, L.chunk, L.B, n, offs, adj_out, off_out, m_out, nullptr,
                                                  nullptr);
  return cudaGetLastError();
}

}  // namespace kc
