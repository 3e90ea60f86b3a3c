// Host/device shared declarations of the batched peel.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kcore_peel.h"

namespace kc {

constexpr long long kMaxSortGraphs = 16384;  // batches up to this size are ordered by arcs

struct BatchArgs {
  long long G;
  long long N;               // total vertices (gv[G])
  long long m;               // total arcs (bound for offsets)
  const long long* gv;       // [G+1] first vertex of each graph
  const long long* off;      // [N+1] global arc offsets
  const int* adj;            // [m] graph-local neighbour ids
  int* core;                 // [N]
  int* kmax;                 // [G]
  int* deg;                  // [N] induced degrees of graphs too large for shared memory
  int* A0;                   // [N] active lists (ping-pong)
  int* A1;
  int* F0;                   // [N] frontiers (ping-pong)
  int* F1;
  const int* order;          // [G] processing order, or nullptr
  int* next_graph;           // work counter
  int* status;
  int smem_deg_max;          // graphs with at most this many vertices keep d~ in shared memory
};

// One graph of a descriptor-driven launch: offsets hold absolute indices
// into adj (bounded by m); scratch arrays hold n entries each.
struct GraphDesc {
  const long long* off;
  const int* adj;
  int* core;
  int* kmax;
  int* deg;
  int* A0;
  int* A1;
  int* F0;
  int* F1;
  long long n;
  long long m;
};

// Table slots of one descriptor-driven launch (passed by value as a kernel
// parameter, so no host buffer must outlive the launch).
constexpr int kMaxSlotsPerLaunch = 1024;
struct SlotList {
  int count;
  int slot[kMaxSlotsPerLaunch];
};

// cluster 2, 4 or 8: clusters of that many CTAs for the listed graphs of at
// least big_arcs arcs (list them largest first)
cudaError_t desc_launch(const GraphDesc* table, const SlotList& list, int* next, int smem_deg_max,
                        int* status, int grid, size_t smem, cudaStream_t stream, int cluster = 0,
                        long long big_arcs = 0);
size_t desc_static_smem();
// gv = {0, n} on `stream`: the vertex offsets of a batch of one graph
cudaError_t batch_single_gv(long long* gv, long long n, cudaStream_t stream);
int batch_occupancy(int block, size_t smem);
size_t batch_static_smem(int block);
// cluster > 1 (512 or 1024 threads, 2, 4 or 8 CTAs): the clustered form, for
// graphs with at least big_arcs arcs
cudaError_t batch_launch(const BatchArgs& a, int block, int grid, size_t smem, bool sort_graphs,
                         cudaStream_t stream, int cluster = 0, long long big_arcs = 0);

}  // namespace kc
