// kcore_validate_csr: checks on the device that a CSR is the simple undirected
// graph the peel requires (Sec. 2: an undirected graph without self-loops or
// parallel edges; the input format of every decomposition entry point).
//
// Two launches. The first checks the offsets: monotone, off[0] = 0 and
// off[n] = m. The second, only if they are sound, is a grid-stride pass over
// the arcs: a warp takes 1024 consecutive arcs, each
// lane 32 of them in order; a lane finds the source of its first arc by binary
// search over the offsets and then walks. Per arc: the neighbour id is in
// [0, n), differs from the source, is larger than the previous entry of the
// same list (ascending lists, hence no repeats), and the neighbour's list
// holds the source (binary search: symmetry). The first failure is recorded (check code, vertex, arc); the rest of the
// pass still runs but records nothing more.
#include <cuda_runtime.h>

#include "kcore_peel.h"

namespace kc {

namespace {

__device__ __forceinline__ void record(int* st, int code, long long v, long long arc) {
  if (atomicCAS(st, 0, code) == 0) {
    long long* p = (long long*)(st + 2);
    p[0] = v;
    p[1] = arc;
  }
}

// Pass 1: the offsets. Monotone, within [0, m], off[0] = 0 and off[n] = m.
__global__ void __launch_bounds__(256) csr_validate_offsets(long long n, long long m, const long long* off,
                                                            int* st) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nthreads) {
    const long long a = off[v], b = off[v + 1];
    if (a < 0 || b < a || b > m) record(st, 1, v, a);
  }
  if (tid == 0) {
    if (off[0] != 0) record(st, 2, 0, off[0]);
    else if (off[n] != m) record(st, 2, n, off[n]);
  }
}

// Pass 2: the arcs, only once pass 1 found the offsets sound (the launch
// boundary orders the two, so every offset read below is within [0, m]).
__global__ void __launch_bounds__(256) csr_validate_arcs(long long n, long long m, const long long* off,
                                                         const int* adj, int* st) {
  if (*((volatile int*)st) != 0) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const long long warp = tid >> 5, nwarps = nthreads >> 5;
  for (long long base = warp * 1024; base < m; base += nwarps * 1024) {
    const long long j0 = base + (long long)lane * 32;
    if (j0 >= m) continue;
    // source of arc j0: the last v with off[v] <= j0
    long long lo = 0, hi = n;
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (off[mid] <= j0) lo = mid;
      else hi = mid;
    }
    long long v = lo, vend = off[v + 1];
    const long long jend = j0 + 32 < m ? j0 + 32 : m;
    for (long long j = j0; j < jend; j++) {
      while (j >= vend) {  // next source (lists may be empty; off[n] = m > j ends it)
        v++;
        vend = off[v + 1];
      }
      const int u = adj[j];
      if (u < 0 || (long long)u >= n) {
        record(st, 3, v, j);
        continue;
      }
      if (u == v) {
        record(st, 4, v, j);
        continue;
      }
      if (j > off[v] && adj[j - 1] >= u) {
        record(st, 5, v, j);
        continue;
      }
      // symmetry: v in u's list
      long long a = off[u], b = off[u + 1] - 1;
      bool found = false;
      while (a <= b) {
        const long long mid = (a + b) >> 1;
        const int x = adj[mid];
        if (x == v) {
          found = true;
          break;
        }
        if (x < v) a = mid + 1;
        else b = mid - 1;
      }
      if (!found) record(st, 6, v, j);
    }
  }
}

}  // namespace

cudaError_t validate_launch(long long n, long long m, const long long* off, const int* adj, int* st, int sms,
                            cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(st, 0, 32, stream);
  if (e != cudaSuccess) return e;
  csr_validate_offsets<<<sms * 4, 256, 0, stream>>>(n, m, off, st);
  e = cudaGetLastError();
  if (e != cudaSuccess || m == 0) return e;
  csr_validate_arcs<<<sms * 8, 256, 0, stream>>>(n, m, off, adj, st);
  return cudaGetLastError();
}

}  // namespace kc
