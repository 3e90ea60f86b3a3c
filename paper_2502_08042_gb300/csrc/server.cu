// Served k-core peel: a request loop with continuous batching.
//
// The server owns one device memory pool (reserved once at creation) and
// admits a request only when its footprint fits the pool and a slot is free:
// offsets + arcs + coreness + k_max + the peel state it keeps resident while
// in flight (induced degrees, active lists and frontiers, 20 bytes per
// vertex; or the whole-GPU peel's workspace for large requests).
//
// kcore_server_poll advances every request through its stages without
// blocking on the device:
//   copying  - its graph is being copied to the pool (copy stream)
//   ready    - copies done; waiting for the next launch
//   running  - small requests that became ready together run as one
//              descriptor-driven batched peel (one CTA per graph; a cluster of
//              CTAs for each of the largest, which are listed first) on one of
//              several launch streams, so a batch admitted while others are on
//              the GPU overlaps with them; a large request (many vertices or
//              arcs) runs the whole-GPU single-graph peel on its own stream
//   results  - coreness and k_max are being copied back (copy stream)
//   done     - returned by poll; its pool memory is released
// No device code waits on the host: every launch is finite.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kcore.h"
#include "kcore_batched.h"
#include "kcore_peel.h"

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// First-fit allocator over [0, size) with coalescing on free.
class PoolAlloc {
 public:
  explicit PoolAlloc(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al256(std::max<size_t>(bytes, 256));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes;
        size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(std::max<size_t>(bytes, 256));
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

enum ReqState { RS_COPYING = 0, RS_READY, RS_RUNNING, RS_RESULTS, RS_DONE };

struct Request {
  int64_t ticket = 0;
  int64_t n = 0, m = 0;
  int32_t* core_h = nullptr;
  bool large = false;
  size_t pool_off = 0, pool_bytes = 0;
  char* d = nullptr;  // device base of the request's pool block
  size_t o_off = 0, o_adj = 0, o_core = 0, o_kmax = 0, o_state = 0;
  int state = RS_COPYING;
  cudaEvent_t ev = nullptr;  // completion of the current stage
  int batch = -1;
  int slot = -1;             // index of the pinned result words and the descriptor table entry
  int32_t* kmax_slot = nullptr;
  int32_t* status_slot = nullptr;
};

struct Batch {
  std::vector<int64_t> reqs;
  size_t pool_off = 0, pool_bytes = 0;
  cudaEvent_t done = nullptr;
  int* d_status = nullptr;
  bool finished = false;
};

}  // namespace

struct kcore_server_ctx {
  int device = 0;
  int sms = 0;
  int peel_ctas_per_sm = 0;
  kcore_server_config cfg{};
  char* pool = nullptr;
  PoolAlloc* alloc = nullptr;
  cudaStream_t copy = nullptr, large = nullptr;
  std::vector<cudaStream_t> launch;
  int next_launch = 0;
  std::map<int64_t, Request> reqs;  // by ticket
  std::map<int, Batch> batches;
  int next_batch = 0;
  int64_t next_ticket = 1;
  // per request slot: pinned k_max/status words, a pinned descriptor and its
  // device copy in the descriptor table
  int32_t* pinned = nullptr;
  std::vector<int> free_slots;
  kc::GraphDesc* pinned_desc = nullptr;
  kc::GraphDesc* d_table = nullptr;
  size_t smem_vertices = 0;
  int desc_grid_cap = 0;
  std::string err;
};

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

long long isqrt_s(long long m) {
  long long r = (long long)std::sqrt((double)m);
  while (r > 0 && r * r > m) r--;
  while ((r + 1) * (r + 1) <= m) r++;
  return r;
}

// Whole-GPU peel workspace for a large request (same layout as the handle's).
struct LargeLayout {
  size_t ctl, rounds, deg, a0, a1, q, total;
  long long qcap;
  int max_rounds;
};
constexpr int kLargeSlice = 64;
LargeLayout large_layout(long long n, long long m) {
  LargeLayout L{};
  L.qcap = n + (m + kLargeSlice - 1) / kLargeSlice + 1;
  L.max_rounds = (int)std::min<long long>(2 * isqrt_s(m) + 8, 2 * n + 8);
  size_t o = 0;
  L.ctl = o;
  o = al256(o + sizeof(kc::PeelCtl));
  L.rounds = o;
  o = al256(o + sizeof(kc::RoundRec) * (size_t)L.max_rounds);
  L.deg = o;
  o = al256(o + 4 * (size_t)n);
  L.a0 = o;
  o = al256(o + 4 * (size_t)n);
  L.a1 = o;
  o = al256(o + 4 * (size_t)n);
  L.q = o;
  o = al256(o + 8 * (size_t)L.qcap);
  L.total = o;
  return L;
}

void release_request(kcore_server_ctx* s, Request& r) {
  if (r.pool_bytes) s->alloc->release(r.pool_off, r.pool_bytes);
  r.pool_bytes = 0;
  if (r.ev) cudaEventDestroy(r.ev);
  r.ev = nullptr;
  if (r.slot >= 0) s->free_slots.push_back(r.slot);
  r.slot = -1;
  r.kmax_slot = r.status_slot = nullptr;
}

}  // namespace

extern "C" {

kcore_status kcore_server_create(kcore_server* out, int device, const kcore_server_config* cfg) {
  if (!out) return KCORE_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return KCORE_ERR_INVALID;
  }
  DevGuard g(device);
  kcore_server_ctx* s = new kcore_server_ctx();
  s->device = device;
  kcore_server_config c{};
  c.pool_bytes = 0;
  c.max_requests = 4096;
  c.streams = 4;
  c.large_vertices = (int64_t)1 << 20;
  c.large_arcs = (int64_t)1 << 25;
  c.batch_cluster = 4;
  c.batch_big_arcs = 0;
  if (cfg) {
    if (cfg->batch_cluster != 0 && cfg->batch_cluster != 1 && cfg->batch_cluster != 2 &&
        cfg->batch_cluster != 4 && cfg->batch_cluster != 8) {
      delete s;
      return KCORE_ERR_INVALID;
    }
    if (cfg->batch_cluster > 0) c.batch_cluster = cfg->batch_cluster;
    if (cfg->batch_big_arcs < 0) {
      delete s;
      return KCORE_ERR_INVALID;
    }
    c.batch_big_arcs = cfg->batch_big_arcs;
    if (cfg->pool_bytes) c.pool_bytes = cfg->pool_bytes;
    if (cfg->max_requests > 0) c.max_requests = cfg->max_requests;
    if (cfg->streams > 0) c.streams = std::min(cfg->streams, 32);
    if (cfg->large_vertices > 0) c.large_vertices = cfg->large_vertices;
    if (cfg->large_arcs > 0) c.large_arcs = cfg->large_arcs;
  }
  if (c.pool_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c.pool_bytes = fr / 4;
  }
  s->cfg = c;
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, device);
  s->peel_ctas_per_sm = kc::bsp_max_ctas_per_sm();
  if (cudaMalloc(&s->pool, c.pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return KCORE_ERR_OOM;
  }
  s->alloc = new PoolAlloc(c.pool_bytes);
  cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&s->large, cudaStreamNonBlocking);
  s->launch.resize(c.streams);
  for (auto& st : s->launch) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (cudaHostAlloc((void**)&s->pinned, sizeof(int32_t) * 2 * (size_t)c.max_requests, cudaHostAllocDefault) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->pool);
    delete s;
    return KCORE_ERR_OOM;
  }
  for (int i = c.max_requests - 1; i >= 0; i--) s->free_slots.push_back(i);
  if (cudaHostAlloc((void**)&s->pinned_desc, sizeof(kc::GraphDesc) * (size_t)c.max_requests,
                    cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc(&s->d_table, sizeof(kc::GraphDesc) * (size_t)c.max_requests) != cudaSuccess) {
    cudaGetLastError();
    if (s->pinned_desc) cudaFreeHost(s->pinned_desc);
    cudaFreeHost(s->pinned);
    cudaFree(s->pool);
    delete s;
    return KCORE_ERR_OOM;
  }
  // shared memory of the descriptor-driven peel: d~ of graphs up to ~half an SM's shared memory
  int sm_total = 0, dev_smem = 0;
  cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  long long per = std::min<long long>((long long)sm_total / 2, (long long)dev_smem) -
                  (long long)kc::desc_static_smem() - 2048;
  s->smem_vertices = (size_t)std::max<long long>(0, per / 4);
  s->desc_grid_cap = s->sms;
  *out = s;
  return KCORE_OK;
}

kcore_status kcore_server_submit(kcore_server s, int64_t n, int64_t m, const int64_t* offsets_host,
                                 const int32_t* adj_host, int32_t* coreness_host, int64_t* ticket_out) {
  if (!s || !ticket_out || n < 0 || m < 0 || n > INT32_MAX - 1) return KCORE_ERR_INVALID;
  if (n > 0 && (!offsets_host || !coreness_host)) return KCORE_ERR_INVALID;
  if (m > 0 && !adj_host) return KCORE_ERR_INVALID;
  DevGuard g(s->device);
  if (s->free_slots.empty()) return KCORE_ERR_CAPACITY;
  Request r;
  r.n = n;
  r.m = m;
  r.core_h = coreness_host;
  r.large = n > s->cfg.large_vertices || m > s->cfg.large_arcs;
  size_t o = 0;
  r.o_off = o;
  o = al256(o + 8 * (size_t)(n + 1));
  r.o_adj = o;
  o = al256(o + 4 * (size_t)std::max<int64_t>(m, 1));
  r.o_core = o;
  o = al256(o + 4 * (size_t)std::max<int64_t>(n, 1));
  r.o_kmax = o;
  o = al256(o + 8);
  r.o_state = o;
  if (r.large) o += large_layout(n, m).total;
  else o += 5 * al256(4 * (size_t)std::max<int64_t>(n, 1));
  size_t poff = 0;
  if (!s->alloc->alloc(o, &poff)) return KCORE_ERR_CAPACITY;  // not admitted now
  r.pool_off = poff;
  r.pool_bytes = o;
  r.d = s->pool + poff;
  int slot = s->free_slots.back();
  s->free_slots.pop_back();
  r.slot = slot;
  r.kmax_slot = s->pinned + 2 * (size_t)slot;
  r.status_slot = r.kmax_slot + 1;
  *r.kmax_slot = 0;
  *r.status_slot = 0;
  cudaError_t e = cudaSuccess;
  if (n > 0) e = cudaMemcpyAsync(r.d + r.o_off, offsets_host, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, s->copy);
  else e = cudaMemsetAsync(r.d + r.o_off, 0, 8, s->copy);
  if (e == cudaSuccess && m > 0)
    e = cudaMemcpyAsync(r.d + r.o_adj, adj_host, 4 * (size_t)m, cudaMemcpyHostToDevice, s->copy);
  if (e == cudaSuccess && !r.large) {
    // the request's descriptor, in its slot of the device table
    kc::GraphDesc gd{};
    char* st = r.d + r.o_state;
    size_t nn = (size_t)std::max<int64_t>(n, 1);
    gd.off = (const long long*)(r.d + r.o_off);
    gd.adj = (const int*)(r.d + r.o_adj);
    gd.core = (int*)(r.d + r.o_core);
    gd.kmax = (int*)(r.d + r.o_kmax);
    gd.deg = (int*)st;
    gd.A0 = (int*)(st + al256(4 * nn));
    gd.A1 = (int*)(st + 2 * al256(4 * nn));
    gd.F0 = (int*)(st + 3 * al256(4 * nn));
    gd.F1 = (int*)(st + 4 * al256(4 * nn));
    gd.n = n;
    gd.m = m;
    s->pinned_desc[slot] = gd;
    e = cudaMemcpyAsync(s->d_table + slot, s->pinned_desc + slot, sizeof(kc::GraphDesc),
                        cudaMemcpyHostToDevice, s->copy);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.ev, s->copy);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_request(s, r);
    s->err = std::string("submit: ") + cudaGetErrorString(e);
    return KCORE_ERR_CUDA;
  }
  r.ticket = s->next_ticket++;
  r.state = RS_COPYING;
  *ticket_out = r.ticket;
  s->reqs.emplace(r.ticket, r);
  return KCORE_OK;
}

kcore_status kcore_server_poll(kcore_server s, int64_t* tickets_out, int32_t* kmax_out, int32_t* status_out,
                               int max_out, int* n_out) {
  if (!s || !n_out || max_out < 0 || (max_out > 0 && !tickets_out)) return KCORE_ERR_INVALID;
  *n_out = 0;
  DevGuard g(s->device);
  cudaError_t e;
  // 1. copies finished -> ready
  std::vector<int64_t> small_ready;
  for (auto& kv : s->reqs) {
    Request& r = kv.second;
    if (r.state == RS_COPYING && cudaEventQuery(r.ev) == cudaSuccess) r.state = RS_READY;
    if (r.state == RS_READY && !r.large) small_ready.push_back(r.ticket);
  }
  cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error
  // 2a. batched launches for the small requests that became ready together
  for (size_t first = 0; first < small_ready.size(); first += kc::kMaxSlotsPerLaunch) {
    int cnt = (int)std::min<size_t>(small_ready.size() - first, (size_t)kc::kMaxSlotsPerLaunch);
    Batch b;
    if (!s->alloc->alloc(256, &b.pool_off)) break;  // no room for the counters now: next poll
    b.pool_bytes = 256;
    int* ctr = (int*)(s->pool + b.pool_off);
    b.d_status = ctr + 1;
    kc::SlotList list;
    list.count = cnt;
    // largest first: with clusters the cluster-sized graphs lead the list
    std::vector<std::pair<long long, int64_t>> by_arcs;
    long long launch_arcs = 0;
    for (int i = 0; i < cnt; i++) {
      const Request& r = s->reqs[small_ready[first + i]];
      by_arcs.push_back({-(long long)r.m, small_ready[first + i]});
      launch_arcs += (long long)r.m;
    }
    std::sort(by_arcs.begin(), by_arcs.end());
    for (int i = 0; i < cnt; i++) {
      Request& r = s->reqs[by_arcs[i].second];
      list.slot[i] = r.slot;
      r.state = RS_RUNNING;
      r.batch = s->next_batch;
      b.reqs.push_back(r.ticket);
    }
    cudaStream_t st = s->launch[s->next_launch];
    s->next_launch = (s->next_launch + 1) % (int)s->launch.size();
    const int cl = s->cfg.batch_cluster > 1 ? s->cfg.batch_cluster : 0;
    int grid = std::min(cl ? cnt * cl : cnt, s->desc_grid_cap);
    long long big = s->cfg.batch_big_arcs > 0 ? (long long)s->cfg.batch_big_arcs
                                              : std::max<long long>(1, launch_arcs / std::max(grid, 1));
    e = cudaMemsetAsync(ctr, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess)
      e = kc::desc_launch(s->d_table, list, ctr, (int)s->smem_vertices, b.d_status, grid,
                          s->smem_vertices * 4, st, cl, big);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->err = std::string("batched launch: ") + cudaGetErrorString(e);
      return KCORE_ERR_CUDA;
    }
    s->batches.emplace(s->next_batch++, b);
  }
  // 2b. large requests: the whole-GPU single-graph peel, one at a time on its stream
  for (auto& kv : s->reqs) {
    Request& r = kv.second;
    if (r.state != RS_READY || !r.large) continue;
    LargeLayout L = large_layout(r.n, r.m);
    char* ws = r.d + r.o_state;
    kc::PeelArgs a{};
    a.n = r.n;
    a.m = r.m;
    a.off = (const long long*)(r.d + r.o_off);
    a.adj = (const int*)(r.d + r.o_adj);
    a.core = (int*)(r.d + r.o_core);
    a.kmax_out = (int*)(r.d + r.o_kmax);
    a.deg = (int*)(ws + L.deg);
    a.A0 = (int*)(ws + L.a0);
    a.A1 = (int*)(ws + L.a1);
    a.Q = (unsigned long long*)(ws + L.q);
    a.qcap = L.qcap;
    a.rounds = (kc::RoundRec*)(ws + L.rounds);
    a.max_rounds = L.max_rounds;
    a.ctl = (kc::PeelCtl*)(ws + L.ctl);
    a.slice = kLargeSlice;
    a.lq_cap = 32;
    a.max_take = 256;
    a.scan_min = 2048;
    a.idle_sleep_ns = 192;
    a.poll_sleep_ns = 64;
    a.timeout_ns = 2000ull * 1000000ull;
    long long want = (r.n + r.m / 8 + 2047) / 2048;
    long long gmax = (long long)s->sms * s->peel_ctas_per_sm;
    int grid = (int)std::max<long long>(1, std::min(want, gmax));
    a.take_div = grid * (kc::bsp_block_size() / 32);
    a.local_batches = 8;
    a.precheck_items = 64;
    e = cudaMemsetAsync(ws, 0, L.deg, s->large);
    if (e == cudaSuccess) e = kc::bsp_launch(a, grid, s->large);
    if (e == cudaSuccess) e = cudaEventRecord(r.ev, s->large);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->err = std::string("large launch: ") + cudaGetErrorString(e);
      return KCORE_ERR_CUDA;
    }
    r.state = RS_RUNNING;
    r.batch = -1;
  }
  // 3. finished launches -> copy results back
  for (auto& kv : s->batches) {
    Batch& b = kv.second;
    if (b.finished || cudaEventQuery(b.done) != cudaSuccess) continue;
    b.finished = true;
    for (int64_t t : b.reqs) {
      Request& r = s->reqs[t];
      if (r.n > 0) cudaMemcpyAsync(r.core_h, r.d + r.o_core, 4 * (size_t)r.n, cudaMemcpyDeviceToHost, s->copy);
      cudaMemcpyAsync(r.kmax_slot, r.d + r.o_kmax, 4, cudaMemcpyDeviceToHost, s->copy);
      cudaMemcpyAsync(r.status_slot, b.d_status, 4, cudaMemcpyDeviceToHost, s->copy);
      cudaEventRecord(r.ev, s->copy);
      r.state = RS_RESULTS;
    }
  }
  for (auto& kv : s->reqs) {
    Request& r = kv.second;
    if (r.state != RS_RUNNING || !r.large || cudaEventQuery(r.ev) != cudaSuccess) continue;
    LargeLayout L = large_layout(r.n, r.m);
    char* ws = r.d + r.o_state;
    if (r.n > 0) cudaMemcpyAsync(r.core_h, r.d + r.o_core, 4 * (size_t)r.n, cudaMemcpyDeviceToHost, s->copy);
    cudaMemcpyAsync(r.kmax_slot, r.d + r.o_kmax, 4, cudaMemcpyDeviceToHost, s->copy);
    cudaMemcpyAsync(r.status_slot, &((kc::PeelCtl*)(ws + L.ctl))->status, 4, cudaMemcpyDeviceToHost, s->copy);
    cudaEventRecord(r.ev, s->copy);
    r.state = RS_RESULTS;
  }
  cudaGetLastError();
  // 4. results copied -> done
  std::vector<int64_t> done;
  for (auto& kv : s->reqs) {
    Request& r = kv.second;
    if (r.state == RS_RESULTS && cudaEventQuery(r.ev) == cudaSuccess) done.push_back(r.ticket);
  }
  cudaGetLastError();
  for (int64_t t : done) {
    Request& r = s->reqs[t];
    if (*n_out < max_out) {
      tickets_out[*n_out] = t;
      if (kmax_out) kmax_out[*n_out] = r.n > 0 ? *r.kmax_slot : 0;
      if (status_out) status_out[*n_out] = *r.status_slot;
      (*n_out)++;
      int b = r.batch;
      release_request(s, r);
      s->reqs.erase(t);
      if (b >= 0) {
        Batch& bb = s->batches[b];
        bool all = true;
        for (int64_t x : bb.reqs)
          if (s->reqs.count(x)) all = false;
        if (all) {
          s->alloc->release(bb.pool_off, bb.pool_bytes);
          cudaEventDestroy(bb.done);
          s->batches.erase(b);
        }
      }
    }
  }
  return KCORE_OK;
}

kcore_status kcore_server_info(kcore_server s, int64_t* in_flight, int64_t* pool_used, int64_t* pool_bytes) {
  if (!s) return KCORE_ERR_INVALID;
  if (in_flight) *in_flight = (int64_t)s->reqs.size();
  if (pool_used) *pool_used = (int64_t)s->alloc->used();
  if (pool_bytes) *pool_bytes = (int64_t)s->cfg.pool_bytes;
  return KCORE_OK;
}

kcore_status kcore_server_destroy(kcore_server s) {
  if (!s) return KCORE_ERR_INVALID;
  {
    DevGuard g(s->device);
    cudaDeviceSynchronize();
    for (auto& kv : s->reqs)
      if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    for (auto& kv : s->batches)
      if (kv.second.done) cudaEventDestroy(kv.second.done);
    for (auto& st : s->launch) cudaStreamDestroy(st);
    cudaStreamDestroy(s->copy);
    cudaStreamDestroy(s->large);
    cudaFree(s->pool);
    cudaFreeHost(s->pinned);
    cudaFreeHost(s->pinned_desc);
    cudaFree(s->d_table);
    cudaGetLastError();
  }
  delete s->alloc;
  delete s;
  return KCORE_OK;
}

}  // extern "C"
