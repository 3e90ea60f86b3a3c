// Final check of a sampled peel (Sec. 4.1, "Recover from Errors").
//
// Every value a peel assigns is at least the vertex's coreness: a vertex gets
// value k only when at most k of its neighbours are untraversed, and every
// traversed one got a value (hence a coreness) of at most k. A sampling error
// can therefore only raise values. Condition (i), that every v has at least
// core[v] neighbours u with core[u] >= core[v], bounds every value by the
// coreness (the set {core >= c} has minimum degree c, so it lies in the
// c-core). Both together: a sampled result that passes (i) is exact, and one
// that fails it is recomputed without sampling.
//
// Two launches: a pass over the arcs (a warp takes 1024 consecutive arcs,
// each lane 32 in order, finding its first arc's source by binary search over
// the offsets) counts, per vertex, the neighbours whose value is at least its
// own; a pass over the vertices compares and clears the counts. Both skip
// their work when the run is already marked for a rerun or raised an error.
#include <climits>

#include "kcore_peel.h"

namespace kc {

namespace {

__global__ void __launch_bounds__(256) check_count(long long n, long long m, const long long* off, const int* adj,
                                                   const int* core, int* acc, const PeelCtl* ctl) {
  if (*((volatile const int*)&ctl->s_redo) || *((volatile const int*)&ctl->status)) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const long long warp = tid >> 5, nwarps = nthreads >> 5;
  for (long long base = warp * 1024; base < m; base += nwarps * 1024) {
    const long long j0 = base + (long long)lane * 32;
    if (j0 >= m) continue;
    long long lo = 0, hi = n;
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (off[mid] <= j0) lo = mid;
      else hi = mid;
    }
    long long v = lo, vend = off[v + 1];
    int cv = core[v], cnt = 0;
    const long long jend = j0 + 32 < m ? j0 + 32 : m;
    for (long long j = j0; j < jend; j++) {
      while (j >= vend && v + 1 < n) {
        if (cnt) atomicAdd(acc + v, cnt);
        cnt = 0;
        v++;
        vend = off[v + 1];
        cv = core[v];
      }
      const int u = adj[j];
      if ((unsigned long long)(unsigned)u < (unsigned long long)n && core[u] >= cv) cnt++;
    }
    if (cnt) atomicAdd(acc + v, cnt);
  }
}

__global__ void __launch_bounds__(256) check_compare(long long n, const int* core, int* acc, PeelCtl* ctl) {
  const bool skip = *((volatile const int*)&ctl->s_redo) != 0 || *((volatile const int*)&ctl->status) != 0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nthreads) {
    if (!skip && acc[v] < core[v]) atomicExch(&ctl->s_redo, 1);
    acc[v] = 0;
  }
}

}  // namespace

cudaError_t sample_check_launch(long long n, long long m, const long long* off, const int* adj, const int* core,
                                int* acc, PeelCtl* ctl, int sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if (m > 0) check_count<<<sms * 8, 256, 0, stream>>>(n, m, off, adj, core, acc, ctl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  check_compare<<<sms * 4, 256, 0, stream>>>(n, core, acc, ctl);
  return cudaGetLastError();
}

}  // namespace kc
