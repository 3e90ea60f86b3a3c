// Autotuners (host code; declarations and contracts in include/kcore.h): the
// batched peel's launch shape, and the single-graph peel's schedule. Each
// times its candidates on the caller's own input through the public entry
// points, so what it measures is exactly what later calls run.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kcore.h"

namespace {

struct Shape {
  int block, ctas_per_sm, cluster, smem_vertices;  // smem_vertices -1: as many as fit
};

// Candidate shapes: threads per CTA x resident CTAs per SM, within one SM's
// 2048 threads. The shared-memory threshold follows each shape (-1: as many
// vertices as fit with that many CTAs per SM).
std::vector<Shape> candidates() {
  std::vector<Shape> c;
  for (int cps : {1, 2}) c.push_back({1024, cps, 0, -1});
  for (int cps : {1, 2, 3, 4}) c.push_back({512, cps, 0, -1});
  for (int cps : {2, 4, 6, 8}) c.push_back({256, cps, 0, -1});
  // more resident CTAs with less shared memory each: the SM keeps more L1 for
  // the global accesses of the graphs that do not fit
  for (int sv : {8000, 2000}) c.push_back({512, 3, 0, sv});
  // the clustered form for the batch's largest graphs
  for (int cl : {2, 4, 8}) c.push_back({1024, 2, cl, -1});
  c.push_back({512, 2, 4, -1});
  return c;
}

struct OptionSnapshot {
  kcore_handle h;
  int64_t block = 0, sv = 0, cps = 0, cluster = 0, big = 0;
  explicit OptionSnapshot(kcore_handle hh) : h(hh) {
    kcore_get_option(h, KCORE_OPT_BATCH_BLOCK, &block);
    kcore_get_option(h, KCORE_OPT_BATCH_SMEM_VERTICES, &sv);
    kcore_get_option(h, KCORE_OPT_BATCH_CTAS_PER_SM, &cps);
    kcore_get_option(h, KCORE_OPT_BATCH_CLUSTER, &cluster);
    kcore_get_option(h, KCORE_OPT_BATCH_BIG_ARCS, &big);
  }
  void restore() const {
    kcore_set_option(h, KCORE_OPT_BATCH_BLOCK, block);
    kcore_set_option(h, KCORE_OPT_BATCH_SMEM_VERTICES, sv);
    kcore_set_option(h, KCORE_OPT_BATCH_CTAS_PER_SM, cps);
    kcore_set_option(h, KCORE_OPT_BATCH_CLUSTER, cluster);
    kcore_set_option(h, KCORE_OPT_BATCH_BIG_ARCS, big);
  }
};

kcore_status apply(kcore_handle h, const Shape& s) {
  kcore_status st = kcore_set_option(h, KCORE_OPT_BATCH_BLOCK, s.block);
  if (st == KCORE_OK) st = kcore_set_option(h, KCORE_OPT_BATCH_SMEM_VERTICES, s.smem_vertices);
  if (st == KCORE_OK) st = kcore_set_option(h, KCORE_OPT_BATCH_CTAS_PER_SM, s.ctas_per_sm);
  if (st == KCORE_OK) st = kcore_set_option(h, KCORE_OPT_BATCH_CLUSTER, s.cluster);
  if (st == KCORE_OK) st = kcore_set_option(h, KCORE_OPT_BATCH_BIG_ARCS, 0);
  return st;
}

}  // namespace

extern "C" kcore_status kcore_autotune_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                               int64_t total_arcs, const int64_t* graph_vertex_offsets,
                                               const int64_t* offsets, const int32_t* adj,
                                               int32_t* coreness_out, int32_t* kmax_out, int32_t repeats,
                                               kcore_batch_tuning* best_out, kcore_stream_t stream_) {
  if (!h || !best_out || repeats < 1 || repeats > 100 || num_graphs < 1) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  *best_out = kcore_batch_tuning{};
  OptionSnapshot saved(h);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return KCORE_ERR_CUDA;
  }
  Shape best{0, 0, 0, -1};
  double best_ms = 0;
  int timed = 0;
  kcore_status result = KCORE_OK;
  for (const Shape& s : candidates()) {
    if (apply(h, s) != KCORE_OK) continue;  // not a valid shape on this device
    // warm-up call: first launch of a shape sets its attributes; its status
    // also tells whether the input is sound
    kcore_status st = kcore_decompose_batched(h, num_graphs, total_vertices, total_arcs, graph_vertex_offsets,
                                              offsets, adj, coreness_out, kmax_out, stream_);
    if (st == KCORE_OK) st = kcore_sync_status(h);
    if (st == KCORE_ERR_NOT_SIMPLE || st == KCORE_ERR_OOM || st == KCORE_ERR_INVALID) {
      result = st;  // input or memory problem: no shape can fix it
      break;
    }
    if (st != KCORE_OK) continue;  // this shape cannot launch here
    double shape_ms = 1e30;
    for (int r = 0; r < repeats && st == KCORE_OK; r++) {
      cudaEventRecord(e0, stream);
      st = kcore_decompose_batched(h, num_graphs, total_vertices, total_arcs, graph_vertex_offsets, offsets,
                                   adj, coreness_out, kmax_out, stream_);
      cudaEventRecord(e1, stream);
      if (st == KCORE_OK) st = kcore_sync_status(h);
      float ms = 0;
      if (st == KCORE_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) shape_ms = std::min(shape_ms, (double)ms);
    }
    if (st != KCORE_OK) continue;
    timed++;
    if (best.block == 0 || shape_ms < best_ms) {
      best = s;
      best_ms = shape_ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (result != KCORE_OK || best.block == 0) {
    saved.restore();
    return result != KCORE_OK ? result : KCORE_ERR_CUDA;
  }
  apply(h, best);
  // leave the outputs computed with the chosen shape
  kcore_status st = kcore_decompose_batched(h, num_graphs, total_vertices, total_arcs, graph_vertex_offsets,
                                            offsets, adj, coreness_out, kmax_out, stream_);
  if (st == KCORE_OK) st = kcore_sync_status(h);
  if (st != KCORE_OK) return st;
  kcore_stats stats{};
  kcore_get_stats(h, &stats);
  best_out->block = best.block;
  best_out->ctas_per_sm = best.ctas_per_sm;
  best_out->cluster = best.cluster;
  best_out->smem_vertices = (int32_t)stats.batch_smem_vertices;
  best_out->candidates = timed;
  best_out->ms = best_ms;
  return KCORE_OK;
}

// ---- single-graph peel: schedule and tail mode -----------------------------

namespace {

constexpr int64_t kHuge = (int64_t)1 << 30;

// One candidate schedule: every option the single-graph tuner sets.
struct Schedule {
  int64_t sync_mode, batch_update, warp_combine, ctas_per_sm, tail_items, tail_entries, precheck_items,
      local_batches, cluster;
};

// Candidates: the default bulk-synchronous schedule; tail mode at small,
// medium and unbounded thresholds (the last runs the whole peel on one CTA,
// which suits small graphs); without batch update; reading d~ first in
// shorter subrounds; shorter local chains; warp aggregation; one CTA per SM;
// the asynchronous schedule; and the whole graph on one CTA or on one cluster
// of 8 CTAs (mode 4).
std::vector<Schedule> schedule_candidates() {
  return {
      {2, 1, 0, 0, 0, 0, 64, 32, 0},
      {2, 1, 0, 0, 8, 0, 64, 32, 0},
      {2, 1, 0, 0, 64, 4096, 64, 32, 0},
      {2, 1, 0, 0, kHuge, kHuge, 64, 32, 0},
      {2, 0, 0, 0, 0, 0, 64, 32, 0},
      {2, 1, 0, 0, 0, 0, 16, 32, 0},
      {2, 1, 0, 0, 0, 0, 64, 8, 0},
      {2, 1, 1, 0, 0, 0, 64, 32, 0},
      {2, 1, 0, 1, 0, 0, 64, 32, 0},
      {1, 1, 0, 0, 0, 0, 64, 32, 0},
      {4, 1, 0, 0, 0, 0, 64, 32, 0},
      {4, 1, 0, 0, 0, 0, 64, 32, 8},
  };
}

constexpr kcore_option kScheduleOptions[] = {KCORE_OPT_SYNC_MODE,      KCORE_OPT_BATCH_UPDATE,
                                             KCORE_OPT_WARP_COMBINE,   KCORE_OPT_CTAS_PER_SM,
                                             KCORE_OPT_TAIL_ITEMS,     KCORE_OPT_TAIL_ENTRIES,
                                             KCORE_OPT_PRECHECK_ITEMS, KCORE_OPT_LOCAL_BATCHES,
                                             KCORE_OPT_BATCH_CLUSTER};
constexpr int kScheduleFields = 9;

int64_t* field(Schedule& s, int i) {
  int64_t* f[] = {&s.sync_mode,    &s.batch_update, &s.warp_combine,   &s.ctas_per_sm,  &s.tail_items,
                  &s.tail_entries, &s.precheck_items, &s.local_batches, &s.cluster};
  return f[i];
}

Schedule read_schedule(kcore_handle h) {
  Schedule s{};
  for (int i = 0; i < kScheduleFields; i++) kcore_get_option(h, kScheduleOptions[i], field(s, i));
  return s;
}

kcore_status apply_schedule(kcore_handle h, Schedule s) {
  for (int i = 0; i < kScheduleFields; i++) {
    const kcore_status st = kcore_set_option(h, kScheduleOptions[i], *field(s, i));
    if (st != KCORE_OK) return st;
  }
  return KCORE_OK;
}

}  // namespace

extern "C" kcore_status kcore_autotune(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets,
                                       const int32_t* adj, int32_t* coreness_out, int32_t* kmax_out,
                                       int32_t repeats, kcore_tuning* best_out, kcore_stream_t stream_) {
  if (!h || !best_out || repeats < 1 || repeats > 100 || n < 1) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  *best_out = kcore_tuning{};
  const Schedule saved = read_schedule(h);
  int64_t trace = 0;
  kcore_get_option(h, KCORE_OPT_TRACE, &trace);
  kcore_set_option(h, KCORE_OPT_TRACE, 0);  // tracing would slow every candidate
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    kcore_set_option(h, KCORE_OPT_TRACE, trace);
    return KCORE_ERR_CUDA;
  }
  Schedule best{};
  bool have = false;
  double best_ms = 0;
  int timed = 0;
  kcore_status result = KCORE_OK;
  for (const Schedule& s : schedule_candidates()) {
    if (apply_schedule(h, s) != KCORE_OK) continue;  // not valid on this device
    kcore_status st = kcore_decompose(h, n, m, offsets, adj, coreness_out, kmax_out, stream_);
    if (st == KCORE_OK) st = kcore_sync_status(h);
    if (st == KCORE_ERR_NOT_SIMPLE || st == KCORE_ERR_OOM || st == KCORE_ERR_INVALID) {
      result = st;  // input or memory problem: no schedule can fix it
      break;
    }
    if (st != KCORE_OK) continue;
    double ms_best = 1e30;
    for (int r = 0; r < repeats && st == KCORE_OK; r++) {
      cudaEventRecord(e0, stream);
      st = kcore_decompose(h, n, m, offsets, adj, coreness_out, kmax_out, stream_);
      cudaEventRecord(e1, stream);
      if (st == KCORE_OK) st = kcore_sync_status(h);
      float ms = 0;
      if (st == KCORE_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_best = std::min(ms_best, (double)ms);
    }
    if (st != KCORE_OK) continue;
    timed++;
    if (!have || ms_best < best_ms) {
      best = s;
      best_ms = ms_best;
      have = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  kcore_set_option(h, KCORE_OPT_TRACE, trace);
  if (result != KCORE_OK || !have) {
    apply_schedule(h, saved);
    return result != KCORE_OK ? result : KCORE_ERR_CUDA;
  }
  apply_schedule(h, best);
  // leave the outputs computed with the chosen schedule
  kcore_status st = kcore_decompose(h, n, m, offsets, adj, coreness_out, kmax_out, stream_);
  if (st == KCORE_OK) st = kcore_sync_status(h);
  if (st != KCORE_OK) return st;
  best_out->sync_mode = (int32_t)best.sync_mode;
  best_out->batch_update = (int32_t)best.batch_update;
  best_out->warp_combine = (int32_t)best.warp_combine;
  best_out->ctas_per_sm = (int32_t)best.ctas_per_sm;
  best_out->tail_items = best.tail_items;
  best_out->tail_entries = best.tail_entries;
  best_out->cluster = (int32_t)best.cluster;
  best_out->precheck_items = best.precheck_items;
  best_out->local_batches = best.local_batches;
  best_out->candidates = timed;
  best_out->ms = best_ms;
  return KCORE_OK;
}
