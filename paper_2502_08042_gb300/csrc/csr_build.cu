// CSR build on sm_103a: edge list -> simple undirected CSR.
//
// The paper symmetrises directed inputs (Sec. 6.1, "Datasets"); the peel needs
// a simple graph. Steps, all on the device:
//   1. keys: each pair (a, b) with a != b gives the arcs a->b and b->a as
//      integers (a << B) | b with B = bits of n-1; self-loops and ids out of
//      range become a sentinel that sorts last (ids out of range also set an
//      error status).
//   2. stable LSD radix sort of the keys over their 2B significant bits, 8-bit
//      digits. Each CTA owns a contiguous chunk; a pass is an upsweep (digit
//      histogram per CTA), a scan of the 256 x CTAs histogram, and a downsweep
//      that ranks each 2,048-key tile in shared memory (warp match for the
//      within-iteration rank) and writes runs of equal digits contiguously,
//      while the next tile arrives by asynchronous copy (cp.async).
//   3. unique + emit: keys equal to their predecessor are dropped; the rest
//      are written in order as adj[] (low B bits), and the first arc of each
//      source vertex fixes offsets[] (vertices without arcs take the next
//      vertex's offset).
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
__global__ void csr_make_keys(const int* src, const int* dst, long long E, long long n, int Bd,
                              const long long* gv, const long long* eoff, long long G,
                              unsigned long long* keys, int* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < E;
       i += (long long)gridDim.x * blockDim.x) {
    int a = src[i], b = dst[i];
    long long base = 0, lim = n;
    if (gv) {
      long long lo = 0, hi = G;  // last g with eoff[g] <= i
      while (hi - lo > 1) {
        long long mid = (lo + hi) >> 1;
        if (eoff[mid] <= i) lo = mid;
        else hi = mid;
      }
      base = gv[lo];
      lim = gv[lo + 1] - base;
    }
    unsigned long long k0 = kSentinel, k1 = kSentinel;
    if ((unsigned long long)(unsigned)a >= (unsigned long long)lim ||
        (unsigned long long)(unsigned)b >= (unsigned long long)lim) {
      atomicCAS(status, 0, 1);
    } else if (a != b) {
      k0 = ((unsigned long long)(base + a) << Bd) | (unsigned long long)b;
      k1 = ((unsigned long long)(base + b) << Bd) | (unsigned long long)a;
    }
    keys[2 * i] = k0;
    keys[2 * i + 1] = k1;
  }
}

__device__ __forceinline__ int digit_of(unsigned long long k, int shift) {
  return (int)((k >> shift) & 0xffull);
}

// Per-CTA digit histogram of its chunk: hist[d * G + g].
__global__ void __launch_bounds__(kCsrBlock) rs_upsweep(const unsigned long long* keys, long long N,
                                                        long long chunk, int shift,
                                                        unsigned* hist) {
  __shared__ unsigned cnt[kCsrBlock / 32][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (kCsrBlock / 32) * 256; i += kCsrBlock) (&cnt[0][0])[i] = 0;
  __syncthreads();
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  for (long long i = lo + tid; i < hi; i += kCsrBlock) atomicAdd(&cnt[warp][digit_of(keys[i], shift)], 1u);
  __syncthreads();
  unsigned s = 0;
  for (int w = 0; w < kCsrBlock / 32; w++) s += cnt[w][tid];
  hist[(long long)tid * gridDim.x + blockIdx.x] = s;
}

// Exclusive scan of a uint32 array into uint64 (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) scan_u32_to_u64(const unsigned* in, unsigned long long* out,
                                                        long long len) {
  __shared__ unsigned long long part[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
}

// Stable scatter of one radix pass. Each CTA walks its chunk tile by tile, in
// order; offs[d * G + g] is where its first key of digit d goes.
__global__ void __launch_bounds__(kCsrBlock, 6) rs_downsweep(const unsigned long long* in,
                                                          unsigned long long* out, long long N,
                                                          long long chunk, int shift,
                                                          const unsigned long long* offs) {
  __shared__ unsigned long long buf[kTile];
  __shared__ __align__(16) unsigned long long stage[kTile];  // the next tile, copied asynchronously
  __shared__ unsigned wbase[kCsrBlock / 32][256];
  __shared__ unsigned local_off[256];
  __shared__ unsigned tile_cnt[256];
  __shared__ unsigned long long run[256];
  __shared__ unsigned part[kCsrBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  run[tid] = offs[(long long)tid * G + blockIdx.x];
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  // 16-byte asynchronous copies of a tile's keys into `stage` (pairs of keys;
  // a last odd key is copied with its neighbour, which lies inside the
  // 256-byte-aligned key buffer and is not used)
  auto prefetch = [&](long long t0) {
    const long long tn = min((long long)kTile, hi - t0);
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(stage);
    for (int c = tid; 2 * c < tn; c += kCsrBlock)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * c), "l"(in + t0 + 2 * c)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (lo < hi) prefetch(lo);
  for (long long ts = lo; ts < hi; ts += kTile) {
    const long long tn = min((long long)kTile, hi - ts);
    for (int i = tid; i < (kCsrBlock / 32) * 256; i += kCsrBlock) (&wbase[0][0])[i] = 0;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    unsigned long long k[kKeysPerThread];
    int dg[kKeysPerThread];
#pragma unroll
    for (int it = 0; it < kKeysPerThread; it++) {
      long long j = (long long)warp * (kKeysPerThread * 32) + it * 32 + lane;
      k[it] = j < tn ? stage[j] : 0;
    }
    __syncthreads();  // the stage is read: copy the next tile into it
    if (ts + kTile < hi) prefetch(ts + kTile);
#pragma unroll
    for (int it = 0; it < kKeysPerThread; it++) {
      long long j = (long long)warp * (kKeysPerThread * 32) + it * 32 + lane;
      dg[it] = 256;  // invalid lane
      if (j < tn) {
        dg[it] = digit_of(k[it], shift);
        atomicAdd(&wbase[warp][dg[it]], 1u);
      }
    }
    __syncthreads();
    // per digit (thread d): tile count, then exclusive scan over digits
    unsigned tc = 0;
    for (int w = 0; w < kCsrBlock / 32; w++) tc += wbase[w][tid];
    tile_cnt[tid] = tc;
    unsigned incl = warp_incl_scan(tc, lane);
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned p = lane < kCsrBlock / 32 ? part[lane] : 0;
      unsigned pi = warp_incl_scan(p, lane);
      if (lane < kCsrBlock / 32) part[lane] = pi - p;
    }
    __syncthreads();
    unsigned lo_d = part[warp] + incl - tc;
    local_off[tid] = lo_d;
    unsigned acc = lo_d;
    for (int w = 0; w < kCsrBlock / 32; w++) {
      unsigned c = wbase[w][tid];
      wbase[w][tid] = acc;
      acc += c;
    }
    __syncthreads();
    // ranks in key order: warps own consecutive sub-ranges, iterations go in order
#pragma unroll
    for (int it = 0; it < kKeysPerThread; it++) {
      unsigned peers = __match_any_sync(kFull, dg[it]);
      int rank = __popc(peers & lanemask_lt());
      unsigned b = 0;
      if (dg[it] < 256) {
        b = wbase[warp][dg[it]];
        buf[b + rank] = k[it];
      }
      __syncwarp();
      if (dg[it] < 256 && rank == 0) wbase[warp][dg[it]] = b + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    for (int j = tid; j < tn; j += kCsrBlock) {
      unsigned long long key = buf[j];
      int d = digit_of(key, shift);
      out[run[d] + (unsigned long long)(j - local_off[d])] = key;
    }
    __syncthreads();
    run[tid] += tile_cnt[tid];
    __syncthreads();
  }
}

// Unique keys of each CTA chunk (a key differing from its predecessor); each
// thread reads kKeysPerThread keys per tile, with their predecessors.
__global__ void __launch_bounds__(kCsrBlock) csr_count_unique(const unsigned long long* k, long long N,
                                                              long long chunk, unsigned* cnt) {
  __shared__ unsigned part[kCsrBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  unsigned c = 0;
  for (long long ts = lo; ts < hi; ts += kTile) {
    unsigned long long x[kKeysPerThread], p[kKeysPerThread];
#pragma unroll
    for (int q = 0; q < kKeysPerThread; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      x[q] = i < hi ? __ldcs(k + i) : kSentinel;
      p[q] = i < hi && i > 0 ? __ldcg(k + i - 1) : kSentinel;
    }
#pragma unroll
    for (int q = 0; q < kKeysPerThread; q++) {
      const long long i = ts + (long long)q * kCsrBlock + tid;
      if (i < hi && x[q] != kSentinel && (i == 0 || p[q] != x[q])) c++;
    }
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

// Ordered emission of the unique keys: adj[pos] = low Bd bits; the first arc
// of each source fixes offsets[] for that source and every source without
// arcs just below it; the last arc fills the offsets of the sources above it.
// A tile of kTile keys is read coalesced into shared memory, each thread then
// takes kKeysPerThread consecutive keys (one block scan orders the whole
// tile), and the tile's unique targets leave through shared memory too.
__global__ void __launch_bounds__(kCsrBlock) csr_emit(const unsigned long long* k, long long N,
                                                      long long chunk, int B, long long n,
                                                      const unsigned long long* base, int* adj,
                                                      long long* off, long long* m_out) {
  __shared__ unsigned long long tk[kTile + 2];  // tk[0]: the key before the tile, tk[kTile + 1]: after it
  __shared__ int ta[kTile];
  __shared__ unsigned part[kCsrBlock / 32];
  __shared__ unsigned long long running;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long mask = (1ull << B) - 1;
  long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  if (tid == 0) running = base[blockIdx.x];
  for (long long ts = lo; ts < hi; ts += kTile) {
    const int tn = (int)min((long long)kTile, hi - ts);
    // tk[j + 1] = key ts + j for j < tn, then the key after the tile (if any)
    for (int j = tid; j <= kTile; j += kCsrBlock) tk[j + 1] = j <= tn && ts + j < N ? k[ts + j] : kSentinel;
    if (tid == 0) tk[0] = ts > 0 ? k[ts - 1] : kSentinel;
    __syncthreads();
    const int j0 = tid * kKeysPerThread;  // this thread's first key, in the tile
    unsigned flags = 0;
#pragma unroll
    for (int q = 0; q < kKeysPerThread; q++) {
      const int j = j0 + q;
      const unsigned long long cur = tk[j + 1], prev = tk[j];
      if (j < tn && cur != kSentinel && (ts + j == 0 || prev != cur)) flags |= 1u << q;
    }
    const unsigned cntf = __popc(flags);
    const unsigned incl = warp_incl_scan(cntf, lane);
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned pp = lane < kCsrBlock / 32 ? part[lane] : 0;
      unsigned pi = warp_incl_scan(pp, lane);
      if (lane < kCsrBlock / 32) part[lane] = pi - pp;
    }
    __syncthreads();
    const unsigned long long r0 = running;
    unsigned local = part[warp] + incl - cntf;  // unique keys of the tile before this thread's first
#pragma unroll
    for (int q = 0; q < kKeysPerThread; q++) {
      const int j = j0 + q;
      if (j >= tn) break;
      const unsigned long long cur = tk[j + 1], prev = tk[j];
      if ((flags >> q) & 1u) {
        const unsigned long long pos = r0 + local;
        ta[local++] = (int)(cur & mask);
        const long long s = (long long)(cur >> B);
        const long long ps = (ts + j == 0 || prev == kSentinel) ? -1 : (long long)(prev >> B);
        if (s != ps)
          for (long long v = ps + 1; v <= s; v++) off[v] = (long long)pos;
      }
      // the last valid key (unique or a repeat) closes the offsets above its source
      if (cur != kSentinel && tk[j + 2] == kSentinel) {
        const long long s = (long long)(cur >> B);
        const long long last = (long long)(r0 + local) - 1;  // position of the latest unique key
        for (long long v = s + 1; v <= n; v++) off[v] = last + 1;
        *m_out = last + 1;
      }
    }
    __syncthreads();
    // the tile's unique targets, coalesced
    if (tid == kCsrBlock - 1) running = r0 + local;
    __syncthreads();
    const unsigned nu = (unsigned)(running - r0);
    for (unsigned j = tid; j < nu; j += kCsrBlock) adj[r0 + j] = ta[j];
    __syncthreads();
  }
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
  // into shared memory while the current one is ranked (44 KB of shared
  // memory, which admits five; 40 registers, held to six CTAs' worth by the
  // kernel's launch bounds): the scatter is latency bound, so resident warps and
  // loads in flight count. Measured on R-MAT 24 (ms per build): 2 CTAs x
  // 4,096-key tiles 56.8, 4 x 4,096 37.7, 6 x 2,048 35.6, 7 x 2,048 38.2,
  // 8 x 1,536 37.3; with the asynchronous copy 5 x 2,048 31.0, 4 x 2,048 31.8
  long long G = (long long)sms * 5;
  long long tiles = (N + kTile - 1) / kTile;
  if (tiles < G) G = tiles < 1 ? 1 : tiles;
  L.grid = (int)G;
  long long chunk = (N + G - 1) / G;
  chunk = (chunk + kTile - 1) / kTile * kTile;
  if (chunk < kTile) chunk = kTile;
  L.chunk = chunk;
  L.N = N;
  L.Bs = bits_for(n);
  // batched: one spare code so that no valid (local) target has all bits set
  // and a valid key can never equal the sentinel in the sorted bits
  L.B = max_graph_n > 0 ? bits_for(max_graph_n + 1) : L.Bs;
  size_t off = 0;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  L.status = off;
  off = al(off + 256);
  L.keys0 = off;
  off = al(off + 8 * (size_t)(N > 0 ? N : 1));
  L.keys1 = off;
  off = al(off + 8 * (size_t)(N > 0 ? N : 1));
  L.hist = off;
  off = al(off + 4 * 256 * (size_t)G);
  L.offs = off;
  off = al(off + 8 * 256 * (size_t)G);
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
  if ((e = cudaMemsetAsync(status, 0, 256, stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(off_out, 0, 8 * (size_t)(n + 1), stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(m_out, 0, 8, stream)) != cudaSuccess) return e;
  if (E == 0) return cudaSuccess;
  const long long N = L.N;
  const int G = L.grid;
  int kb = (int)std::min<long long>((E + kCsrBlock - 1) / kCsrBlock, 65536);
  csr_make_keys<<<kb, kCsrBlock, 0, stream>>>(src, dst, E, n, L.B, gv, eoff, ngraphs, k0, status);
  const int passes = (L.Bs + L.B + 7) / 8;
  for (int p = 0; p < passes; p++) {
    int shift = 8 * p;
    rs_upsweep<<<G, kCsrBlock, 0, stream>>>(k0, N, L.chunk, shift, hist);
    scan_u32_to_u64<<<1, 1024, 0, stream>>>(hist, offs, 256ll * G);
    rs_downsweep<<<G, kCsrBlock, 0, stream>>>(k0, k1, N, L.chunk, shift, offs);
    unsigned long long* t = k0;
    k0 = k1;
    k1 = t;
  }
  csr_count_unique<<<G, kCsrBlock, 0, stream>>>(k0, N, L.chunk, hist);
  scan_u32_to_u64<<<1, 1024, 0, stream>>>(hist, offs, G);
  csr_emit<<<G, kCsrBlock, 0, stream>>>(k0, N, L.chunk, L.B, n, offs, adj_out, off_out, m_out);
  return cudaGetLastError();
}

}  // namespace kc
