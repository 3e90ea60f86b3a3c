// C ABI of libkcore: handle, workspace, options and the single-graph entry
// points (declarations and contracts in include/kcore.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "kcore.h"
#include "kcore_batched.h"
#include "kcore_csr.h"
#include "kcore_peel.h"

struct kcore_ctx {
  int device = 0;
  int sms = 0;
  int max_ctas_per_sm = 0;
  int bsp_max_ctas_per_sm = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_external = false;
  std::string err;
  int64_t opt[kc::kNumOptions] = {0, 0, 0, -1, kc::kTimeoutMsDefault, 1, 2048, 0, 0, 192,
                                  kc::kPollSleepDefault, 1024, -1, 0, kc::kLocalBatchesDefault, 0, 1,
                                  0, 0, -1, 1, 1, 0, kc::kPrecheckDefault, kc::kTailItemsDefault,
                                  kc::kTailEntriesDefault, kc::kParkSleepDefault,
                                  kc::kScanMin, 0, 0};  // indexed by kcore_option
  cudaStream_t last_stream = nullptr;
  bool pending = false;
  kc::PeelCtl* last_ctl = nullptr;
  kc::PeelCtl* last_ctl2 = nullptr;  // sampled calls: the control block of the rerun without sampling
  int* last_csr_status = nullptr;  // device status word of the last CSR build
  int* last_batch_status = nullptr;  // device status word of the last batched call
  int* last_validate_status = nullptr;  // device status words of the last CSR check
  int last_batch_block = 0, last_batch_grid = 0, last_batch_smem_vertices = 0, last_batch_cluster = 0;
  bool last_batch_single = false;  // the batched kernel ran one graph of a single-graph call (mode 4)
  unsigned long long* last_trace = nullptr;
  bool last_trace_phases = false;  // the trace holds one record per phase
  int last_max_rounds = 0;
  kcore_stats stats{};
  int last_grid = 0;
  int last_mode = 0;
  int last_slice = 0;
  // device staging for kcore_decompose_host
  void* e2e = nullptr;
  size_t e2e_bytes = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

kcore_status fail(kcore_ctx* h, kcore_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

kcore_status cuda_fail(kcore_ctx* h, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear the sticky-free error state
  return fail(h, KCORE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

long long isqrt_ll(long long m) {
  long long r = (long long)std::sqrt((double)m);
  while (r > 0 && r * r > m) r--;
  while ((r + 1) * (r + 1) <= m) r++;
  return r;
}

struct PeelLayout {
  size_t deg, a0, a1, a2, q, rounds, ctl, trace, hcnt, touched, total;
  // sampling: the rerun's control block and round ring, and the sampler state
  size_t ctl2, rounds2, scnt, stamp, racc, rst, rlist, rq, rqv;
  long long qcap, rqcap;
  int max_rounds;
};
constexpr int kRecountSlice = 1024;  // arcs per recount slice

// Workspace of the single-graph peel: d~[n], two active lists [n], the work
// queue (every vertex pushes ceil(deg/slice) slices once: <= n + m/slice), the
// per-round records (levels <= k_max+1 <= sqrt(m)+1, each followed by at most
// one empty speculative level) and the control block. Everything below `deg`
// is zeroed per call.
PeelLayout peel_layout(long long n, long long m, int slice, bool offline = false, bool sample = false) {
  PeelLayout L{};
  L.qcap = n + (m + slice - 1) / slice + 1;
  L.rqcap = n + (m + kRecountSlice - 1) / kRecountSlice + 1;
  long long mr = 2 * isqrt_ll(m) + 8;
  mr = std::min(mr, 2 * n + 8);
  L.max_rounds = (int)mr;
  size_t off = 0;
  L.ctl = off;
  off = align_up(off + sizeof(kc::PeelCtl), 256);
  L.rounds = off;
  off = align_up(off + sizeof(kc::RoundRec) * (size_t)L.max_rounds, 256);
  L.ctl2 = L.rounds2 = off;
  if (sample) {
    L.ctl2 = off;
    off = align_up(off + sizeof(kc::PeelCtl), 256);
    L.rounds2 = off;
    off = align_up(off + sizeof(kc::RoundRec) * (size_t)kc::kPhaseRing, 256);
  }
  L.deg = off;
  off = align_up(off + 4 * (size_t)n, 256);
  L.a0 = off;
  off = align_up(off + 4 * (size_t)n, 256);
  L.a1 = off;
  off = align_up(off + 4 * (size_t)n, 256);
  L.a2 = off;  // third list buffer of the level window (sync mode 2)
  off = align_up(off + 4 * (size_t)n, 256);
  L.q = off;
  off = align_up(off + 8 * (size_t)L.qcap, 256);
  L.trace = off;
  off = align_up(off + 8 * (size_t)kc::kTraceFields * (size_t)L.max_rounds, 256);
  // offline subrounds (mode 3): decrement counts and the touched list
  L.hcnt = L.touched = off;
  if (offline) {
    L.hcnt = off;
    off = align_up(off + 4 * (size_t)n, 256);
    L.touched = off;
    off = align_up(off + 4 * (size_t)n, 256);
  }
  // sampling: head counts, stamps, recount accumulators and list, recount queue
  L.scnt = L.stamp = L.racc = L.rst = L.rlist = L.rq = L.rqv = off;
  if (sample) {
    size_t* arrays[] = {&L.scnt, &L.stamp, &L.racc, &L.rst, &L.rlist};
    for (size_t* f : arrays) {
      *f = off;
      off = align_up(off + 4 * (size_t)n, 256);
    }
    L.rq = off;
    off = align_up(off + 8 * (size_t)L.rqcap, 256);
    L.rqv = off;
    off = align_up(off + 4 * (size_t)L.rqcap, 256);
  }
  L.total = off;
  return L;
}

// Schedule and slice length a call on this handle uses (option value 0 = auto).
int effective_mode(const kcore_ctx* h) {
  const int64_t m = h->opt[KCORE_OPT_SYNC_MODE];
  return m == 1 ? 1 : (m == 3 ? 3 : (m == 4 ? 4 : 2));
}
// mode 4: the batched peel's kernel on a batch of one graph (defined with the batched entry points)
size_t single_batched_bytes(int64_t n);
kcore_status single_batched_call(kcore_ctx* h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                                 int32_t* out, int32_t* kmax_out, cudaStream_t stream);
// Sampling runs in the bulk-synchronous mode, without the level window and
// not for the k'-core query.
bool sampling_on(const kcore_ctx* h, bool threshold) {
  return h->opt[KCORE_OPT_SAMPLING] != 0 && !threshold && effective_mode(h) == 2 &&
         h->opt[KCORE_OPT_LEVEL_WINDOW] == 0;
}
// mu of the sampling theorem (Sec. 4.1) with c = 8 unless set: ceil(4 (c + 2) ln n).
int sample_mu(const kcore_ctx* h, long long n) {
  if (h->opt[KCORE_OPT_SAMPLE_MU] > 0) return (int)h->opt[KCORE_OPT_SAMPLE_MU];
  return (int)std::ceil(40.0 * std::log((double)std::max(n, 2ll)));
}
int effective_slice(const kcore_ctx* h) {
  if (h->opt[KCORE_OPT_SLICE_ARCS] > 0) return (int)h->opt[KCORE_OPT_SLICE_ARCS];
  return effective_mode(h) == 1 ? 512 : kc::kSliceDefault;
}

kcore_status ensure_ws(kcore_ctx* h, size_t need) {
  if (h->ws_bytes >= need) return KCORE_OK;
  if (h->ws_external)
    return fail(h, KCORE_ERR_OOM,
                "caller workspace too small: need " + std::to_string(need) + " bytes, have " +
                    std::to_string(h->ws_bytes));
  if (h->ws) {
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  size_t grow = std::max(need, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(&h->ws, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return fail(h, KCORE_ERR_OOM, "cudaMalloc of " + std::to_string(grow) + " workspace bytes failed");
  }
  h->ws_bytes = grow;
  return KCORE_OK;
}

}  // namespace

extern "C" {

kcore_status kcore_create(kcore_handle* out, int device) {
  if (!out) return KCORE_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return KCORE_ERR_INVALID;
  }
  kcore_ctx* h = new kcore_ctx();
  h->device = device;
  DeviceGuard g(device);
  if (!g.ok) {
    delete h;
    return KCORE_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
  h->max_ctas_per_sm = kc::peel_max_ctas_per_sm();
  h->bsp_max_ctas_per_sm = kc::bsp_max_ctas_per_sm();
  if (h->max_ctas_per_sm <= 0 || h->bsp_max_ctas_per_sm <= 0 || h->sms <= 0) {
    delete h;
    cudaGetLastError();
    return KCORE_ERR_CUDA;
  }
  *out = h;
  return KCORE_OK;
}

kcore_status kcore_destroy(kcore_handle h) {
  if (!h) return KCORE_ERR_INVALID;
  {
    DeviceGuard g(h->device);
    if (h->pending && h->last_stream) cudaStreamSynchronize(h->last_stream);
    cudaDeviceSynchronize();
    if (h->ws && !h->ws_external) cudaFree(h->ws);
    if (h->e2e) cudaFree(h->e2e);
    cudaGetLastError();
  }
  delete h;
  return KCORE_OK;
}

const char* kcore_last_error(kcore_handle h) { return h ? h->err.c_str() : "null handle"; }

kcore_status kcore_set_option(kcore_handle h, kcore_option opt, int64_t value) {
  if (!h || (int)opt < 0 || (int)opt >= kc::kNumOptions) return KCORE_ERR_INVALID;
  switch (opt) {
    case KCORE_OPT_TAIL_ITEMS:
      if (value < 0 || value > (1ll << 30)) return fail(h, KCORE_ERR_INVALID, "tail items in [0, 2^30]");
      break;
    case KCORE_OPT_TAIL_ENTRIES:
      if (value < 0 || value > INT32_MAX - 1) return fail(h, KCORE_ERR_INVALID, "tail entries in [0, 2^31 - 2]");
      break;
    case KCORE_OPT_SCAN_ENTRIES:
      if (value < 256 || value > (1 << 20)) return fail(h, KCORE_ERR_INVALID, "scan entries in [256, 2^20]");
      break;
    case KCORE_OPT_BATCH_BLOCK:
      if (value != 256 && value != 512 && value != 1024)
        return fail(h, KCORE_ERR_INVALID, "batch block must be 256, 512 or 1024");
      break;
    case KCORE_OPT_BATCH_SMEM_VERTICES:
      if (value < -1 || value > 60000) return fail(h, KCORE_ERR_INVALID, "batch smem vertices in [-1, 60000]");
      break;
    case KCORE_OPT_BATCH_CTAS_PER_SM:
      if (value < 0 || value > 8) return fail(h, KCORE_ERR_INVALID, "batch CTAs per SM in [0, 8]");
      break;
    case KCORE_OPT_BATCH_CLUSTER:
      if (value != 0 && value != 2 && value != 4 && value != 8)
        return fail(h, KCORE_ERR_INVALID, "batch cluster must be 0, 2, 4 or 8");
      break;
    case KCORE_OPT_BATCH_BIG_ARCS:
      if (value < 0 || value > ((int64_t)1 << 40)) return fail(h, KCORE_ERR_INVALID, "big arcs in [0, 2^40]");
      break;
    case KCORE_OPT_LOCAL_BATCHES:
      if (value < 0 || value > (1 << 20)) return fail(h, KCORE_ERR_INVALID, "local batches in [0, 2^20]");
      break;
    case KCORE_OPT_LEVEL_WINDOW:
      if (value < 0 || value > (1 << 20)) return fail(h, KCORE_ERR_INVALID, "level window in [0, 2^20]");
      break;
    case KCORE_OPT_BATCH_UPDATE:
      if (value < 0 || value > 1) return fail(h, KCORE_ERR_INVALID, "batch update must be 0 or 1");
      break;
    case KCORE_OPT_SAMPLING:
    case KCORE_OPT_SAMPLE_CHECK:
    case KCORE_OPT_WARP_COMBINE:
      if (value < 0 || value > 1) return fail(h, KCORE_ERR_INVALID, "sampling switches must be 0 or 1");
      break;
    case KCORE_OPT_SAMPLE_MU:
      if (value < 0 || value > (1 << 24)) return fail(h, KCORE_ERR_INVALID, "sample mu in [0, 2^24]");
      break;
    case KCORE_OPT_SAMPLE_THRESHOLD:
      if (value < -1 || value > INT32_MAX) return fail(h, KCORE_ERR_INVALID, "sample threshold in [-1, 2^31 - 1]");
      break;
    case KCORE_OPT_SAMPLE_SEED:
      break;
    case KCORE_OPT_PRECHECK_ITEMS:
      if (value < 0 || value > (1 << 20)) return fail(h, KCORE_ERR_INVALID, "precheck items in [0, 2^20]");
      break;
    case KCORE_OPT_IDLE_SLEEP_NS:
    case KCORE_OPT_POLL_SLEEP_NS:
    case KCORE_OPT_PARK_SLEEP_NS:
      if (value < 0 || value > 100000) return fail(h, KCORE_ERR_INVALID, "sleep must be in [0, 100000] ns");
      break;
    case KCORE_OPT_TRACE:
      if (value < 0 || value > 2) return fail(h, KCORE_ERR_INVALID, "trace must be 0, 1 or 2");
      break;
    case KCORE_OPT_TEST_STALL:
      if (value < 0 || value > 1) return fail(h, KCORE_ERR_INVALID, "test stall must be 0 or 1");
      break;
    case KCORE_OPT_SYNC_MODE:
      if (value < 0 || value > 4) return fail(h, KCORE_ERR_INVALID, "sync mode must be 0, 1, 2, 3 or 4");
      break;
    case KCORE_OPT_CTAS_PER_SM:
      if (value < 0 || value > h->max_ctas_per_sm)
        return fail(h, KCORE_ERR_INVALID, "CTAs per SM above the occupancy limit");
      break;
    case KCORE_OPT_SLICE_ARCS:
      if (value != 0 && (value < kc::kMinSlice || value > (1 << 20)))
        return fail(h, KCORE_ERR_INVALID, "slice must be 0 (auto) or in [16, 2^20]");
      break;
    case KCORE_OPT_LOCAL_QUEUE:
      if (value < -1 || value > kc::kLocalQueueMax)
        return fail(h, KCORE_ERR_INVALID, "local queue must be -1 (auto) or in [0, 128]");
      break;
    case KCORE_OPT_TIMEOUT_MS:
      if (value < 1 || value > 600000) return fail(h, KCORE_ERR_INVALID, "timeout must be in [1, 600000] ms");
      break;
    case KCORE_OPT_MIN_CTAS:
      if (value < 1) return fail(h, KCORE_ERR_INVALID, "min CTAs must be >= 1");
      break;
    case KCORE_OPT_VERTICES_PER_CTA:
      if (value < 1) return fail(h, KCORE_ERR_INVALID, "vertices per CTA must be >= 1");
      break;
  }
  h->opt[opt] = value;
  return KCORE_OK;
}

kcore_status kcore_get_option(kcore_handle h, kcore_option opt, int64_t* value) {
  if (!h || !value || (int)opt < 0 || (int)opt >= kc::kNumOptions) return KCORE_ERR_INVALID;
  *value = h->opt[opt];
  return KCORE_OK;
}

kcore_status kcore_workspace_size(kcore_handle h, int64_t n, int64_t m, size_t* bytes) {
  if (!h || !bytes || n < 0 || m < 0 || n > INT32_MAX - 1) return KCORE_ERR_INVALID;
  if (effective_mode(h) == 4) {
    *bytes = single_batched_bytes(n);
    return KCORE_OK;
  }
  *bytes = peel_layout(n, m, effective_slice(h),
                       effective_mode(h) == 3 || (effective_mode(h) == 2 && h->opt[KCORE_OPT_BATCH_UPDATE]),
                       sampling_on(h, false))
               .total;
  return KCORE_OK;
}

kcore_status kcore_set_workspace(kcore_handle h, void* ptr, size_t bytes) {
  if (!h) return KCORE_ERR_INVALID;
  if (ptr && ((uintptr_t)ptr % 256) != 0) return fail(h, KCORE_ERR_INVALID, "workspace must be 256-byte aligned");
  DeviceGuard g(h->device);
  if (h->ws && !h->ws_external) {
    cudaDeviceSynchronize();
    cudaFree(h->ws);
  }
  h->ws = ptr;
  h->ws_bytes = ptr ? bytes : 0;
  h->ws_external = ptr != nullptr;
  return KCORE_OK;
}

}  // extern "C"

namespace {

// One single-graph peel on the handle's workspace: the decomposition, or
// (threshold) the k'-core query, which only the bulk-synchronous kernel runs.
kcore_status peel_call(kcore_ctx* h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                       int32_t* out, int32_t* kmax_out, cudaStream_t stream, bool threshold, int32_t kprime,
                       int64_t* size_out) {
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  h->stats = kcore_stats{};
  h->last_ctl = nullptr;
  h->last_csr_status = nullptr;
  h->last_trace = nullptr;
  h->last_stream = stream;
  h->pending = true;
  h->last_validate_status = nullptr;
  if (n == 0) {
    cudaError_t e = cudaSuccess;
    if (kmax_out) e = cudaMemsetAsync(kmax_out, 0, sizeof(int32_t), stream);
    if (e == cudaSuccess && size_out) e = cudaMemsetAsync(size_out, 0, sizeof(int64_t), stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    return KCORE_OK;
  }
  if (!threshold && effective_mode(h) == 4) return single_batched_call(h, n, m, offsets, adj, out, kmax_out, stream);
  const int mode = threshold ? 2 : effective_mode(h);
  const int slice =
      h->opt[KCORE_OPT_SLICE_ARCS] > 0 ? (int)h->opt[KCORE_OPT_SLICE_ARCS] : (mode == 1 ? 512 : kc::kSliceDefault);
  const bool hybrid = mode == 2 && !threshold && h->opt[KCORE_OPT_BATCH_UPDATE] != 0 &&
                      h->opt[KCORE_OPT_LEVEL_WINDOW] == 0;
  const bool sample = sampling_on(h, threshold);
  PeelLayout L = peel_layout(n, m, slice, mode == 3 || hybrid, sample);
  kcore_status st = ensure_ws(h, L.total);
  if (st != KCORE_OK) return st;
  char* ws = (char*)h->ws;
  kc::PeelArgs a{};
  a.n = n;
  a.m = m;
  a.off = (const long long*)offsets;
  a.adj = adj;
  a.core = out;
  a.kmax_out = kmax_out;
  a.deg = (int*)(ws + L.deg);
  a.A0 = (int*)(ws + L.a0);
  a.A1 = (int*)(ws + L.a1);
  a.Q = (unsigned long long*)(ws + L.q);
  a.qcap = L.qcap;
  a.rounds = (kc::RoundRec*)(ws + L.rounds);
  a.max_rounds = L.max_rounds;
  a.ctl = (kc::PeelCtl*)(ws + L.ctl);
  a.slice = slice;
  a.lq_cap = h->opt[KCORE_OPT_LOCAL_QUEUE] >= 0 ? (int)h->opt[KCORE_OPT_LOCAL_QUEUE]
                                                : (mode == 1 ? 32 : kc::kLocalQueueDefault);
  a.max_take = 256;
  a.timeout_ns = (unsigned long long)h->opt[KCORE_OPT_TIMEOUT_MS] * 1000000ull;
  a.scan_min = (int)h->opt[KCORE_OPT_SCAN_ENTRIES];
  a.idle_sleep_ns = (int)h->opt[KCORE_OPT_IDLE_SLEEP_NS];
  a.poll_sleep_ns = (int)h->opt[KCORE_OPT_POLL_SLEEP_NS];
  a.inject_stall = (int)h->opt[KCORE_OPT_TEST_STALL];
  a.trace = h->opt[KCORE_OPT_TRACE] ? (unsigned long long*)(ws + L.trace) : nullptr;
  a.trace_phases = h->opt[KCORE_OPT_TRACE] == 2 && mode != 1 ? 1 : 0;
  a.local_batches = h->opt[KCORE_OPT_LOCAL_BATCHES] > 0 ? (int)h->opt[KCORE_OPT_LOCAL_BATCHES] : INT32_MAX;
  a.threshold = threshold ? 1 : 0;
  a.offline = mode == 3 ? 1 : 0;
  a.window = mode == 2 ? (int)h->opt[KCORE_OPT_LEVEL_WINDOW] : 0;
  a.hybrid = hybrid ? 1 : 0;
  a.A2 = (int*)(ws + L.a2);
  a.hcnt = (int*)(ws + L.hcnt);
  a.touched = (int*)(ws + L.touched);
  a.kprime = threshold ? std::max<int32_t>(kprime, 0) : 0;
  a.size_out = (long long*)size_out;
  a.combine = mode == 2 && h->opt[KCORE_OPT_WARP_COMBINE] != 0 ? 1 : 0;
  a.precheck_items = (int)h->opt[KCORE_OPT_PRECHECK_ITEMS];
  a.tail_items = mode == 2 ? h->opt[KCORE_OPT_TAIL_ITEMS] : 0;
  a.tail_entries = mode == 2 ? h->opt[KCORE_OPT_TAIL_ENTRIES] : 0;
  a.park_sleep_ns = (int)h->opt[KCORE_OPT_PARK_SLEEP_NS];

  if (mode != 1 && m >= ((int64_t)1 << 40))
    return fail(h, KCORE_ERR_INVALID, "the bulk-synchronous modes take at most 2^40 arcs");
  const int mode_max = mode != 1 ? h->bsp_max_ctas_per_sm : h->max_ctas_per_sm;
  int per_sm = h->opt[KCORE_OPT_CTAS_PER_SM] > 0 ? (int)h->opt[KCORE_OPT_CTAS_PER_SM] : mode_max;
  per_sm = std::min(per_sm, mode_max);
  long long gmax = (long long)h->sms * per_sm;
  long long work = n + m / 8;
  long long want = (work + h->opt[KCORE_OPT_VERTICES_PER_CTA] - 1) / h->opt[KCORE_OPT_VERTICES_PER_CTA];
  long long grid = std::max<long long>(h->opt[KCORE_OPT_MIN_CTAS], std::min(want, gmax));
  grid = std::min(grid, gmax);
  a.take_div = (int)std::max<long long>(1, grid * (kc::peel_block_size() / 32));

  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, L.deg, stream)) != cudaSuccess) return cuda_fail(h, e, "memset ctl");
  // the asynchronous mode polls queue slots for the item tag; the
  // bulk-synchronous mode reads only slots written before its barrier
  if (mode == 1 && (e = cudaMemsetAsync(ws + L.q, 0xff, 8 * (size_t)L.qcap, stream)) != cudaSuccess)
    return cuda_fail(h, e, "memset queue");
  if (a.trace && (e = cudaMemsetAsync(a.trace, 0, 8 * (size_t)kc::kTraceFields * (size_t)L.max_rounds,
                                      stream)) != cudaSuccess)
    return cuda_fail(h, e, "memset trace");
  if ((mode == 3 || hybrid) && (e = cudaMemsetAsync(a.hcnt, 0, 4 * (size_t)n, stream)) != cudaSuccess)
    return cuda_fail(h, e, "memset counts");
  h->last_ctl2 = nullptr;
  if (sample) {
    // the sampled run, its final check, and the rerun without sampling that
    // runs only when the sampled result is not exact
    kc::PeelArgs sa = a;
    sa.sample = 1;
    sa.hybrid = 0;
    sa.window = 0;
    sa.trace = nullptr;
    sa.mu = sample_mu(h, n);
    sa.sthreshold = h->opt[KCORE_OPT_SAMPLE_THRESHOLD] >= 0 ? h->opt[KCORE_OPT_SAMPLE_THRESHOLD] : 8ll * sa.mu;
    sa.seed = (unsigned long long)h->opt[KCORE_OPT_SAMPLE_SEED];
    sa.coin_lim = ((unsigned long long)(10ull * (unsigned long long)sa.mu) << 32) / 9ull;
    sa.scnt = (int*)(ws + L.scnt);
    sa.stamp = (int*)(ws + L.stamp);
    sa.racc = (int*)(ws + L.racc);
    sa.rst = (int*)(ws + L.rst);
    sa.rlist = (int*)(ws + L.rlist);
    sa.RQ = (unsigned long long*)(ws + L.rq);
    sa.RQv = (int*)(ws + L.rqv);
    sa.rqcap = L.rqcap;
    sa.rslice = kRecountSlice;
    if ((e = kc::bsp_launch(sa, (int)grid, stream)) != cudaSuccess) return cuda_fail(h, e, "sampled peel launch");
    if (h->opt[KCORE_OPT_SAMPLE_CHECK] &&
        (e = kc::sample_check_launch(n, m, (const long long*)offsets, adj, out, sa.racc, sa.ctl, h->sms,
                                     stream)) != cudaSuccess)
      return cuda_fail(h, e, "sampled result check launch");
    a.ctl = (kc::PeelCtl*)(ws + L.ctl2);
    a.rounds = (kc::RoundRec*)(ws + L.rounds2);
    a.run_if = &sa.ctl->s_redo;
    if ((e = kc::bsp_launch(a, (int)grid, stream)) != cudaSuccess) return cuda_fail(h, e, "rerun launch");
    h->last_ctl = sa.ctl;
    h->last_ctl2 = a.ctl;
  } else {
    e = mode != 1 ? kc::bsp_launch(a, (int)grid, stream) : kc::peel_launch(a, (int)grid, stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "peel launch");
    h->last_ctl = a.ctl;
  }
  h->last_trace = sample ? nullptr : a.trace;  // the sampled peel records no timeline
  h->last_trace_phases = a.trace_phases != 0;
  h->last_max_rounds = L.max_rounds;
  h->last_grid = (int)grid;
  h->last_mode = mode;
  h->last_slice = slice;
  return KCORE_OK;
}

}  // namespace

extern "C" {

kcore_status kcore_decompose(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets,
                             const int32_t* adj, int32_t* coreness_out, int32_t* kmax_out,
                             kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  if (n < 0 || m < 0 || n > INT32_MAX - 1) return fail(h, KCORE_ERR_INVALID, "n or m out of range");
  if (!kmax_out) return fail(h, KCORE_ERR_INVALID, "kmax_out is null");
  if (n > 0 && (!offsets || !coreness_out)) return fail(h, KCORE_ERR_INVALID, "null offsets/coreness");
  if (m > 0 && !adj) return fail(h, KCORE_ERR_INVALID, "null adj with m > 0");
  return peel_call(h, n, m, offsets, adj, coreness_out, kmax_out, (cudaStream_t)stream_, false, 0, nullptr);
}

kcore_status kcore_core_mask(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                             int32_t kprime, int32_t* mask_out, int64_t* size_out, kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  if (n < 0 || m < 0 || n > INT32_MAX - 1) return fail(h, KCORE_ERR_INVALID, "n or m out of range");
  if (n > 0 && (!offsets || !mask_out)) return fail(h, KCORE_ERR_INVALID, "null offsets/mask");
  if (m > 0 && !adj) return fail(h, KCORE_ERR_INVALID, "null adj with m > 0");
  return peel_call(h, n, m, offsets, adj, mask_out, nullptr, (cudaStream_t)stream_, true, kprime, size_out);
}

kcore_status kcore_validate_csr(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                               kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  if (n < 0 || m < 0 || n > INT32_MAX - 1) return fail(h, KCORE_ERR_INVALID, "n or m out of range");
  if (n == 0 && m > 0) return fail(h, KCORE_ERR_INVALID, "arcs given for an empty vertex set");
  if (n > 0 && !offsets) return fail(h, KCORE_ERR_INVALID, "null offsets");
  if (m > 0 && !adj) return fail(h, KCORE_ERR_INVALID, "null adj with m > 0");
  cudaStream_t stream = (cudaStream_t)stream_;
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  h->stats = kcore_stats{};
  h->last_ctl = nullptr;
  h->last_csr_status = nullptr;
  h->last_batch_status = nullptr;
  h->last_trace = nullptr;
  h->last_validate_status = nullptr;
  h->last_stream = stream;
  h->pending = true;
  h->last_validate_status = nullptr;
  if (n == 0) return KCORE_OK;
  kcore_status st = ensure_ws(h, 64);
  if (st != KCORE_OK) return st;
  cudaError_t e = kc::validate_launch(n, m, (const long long*)offsets, adj, (int*)h->ws, h->sms, stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "CSR check launch");
  h->last_validate_status = (int*)h->ws;
  return KCORE_OK;
}

kcore_status kcore_build_csr_workspace_size(kcore_handle h, int64_t n, int64_t num_edges, size_t* bytes) {
  if (!h || !bytes || n < 0 || n > INT32_MAX - 1 || num_edges < 0) return KCORE_ERR_INVALID;
  *bytes = kc::csr_layout(n, num_edges, h->sms).total;
  return KCORE_OK;
}

kcore_status kcore_build_csr(kcore_handle h, int64_t n, int64_t num_edges, const int32_t* src,
                             const int32_t* dst, int64_t* offsets_out, int32_t* adj_out,
                             int64_t* m_out, kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n < 0 || n > INT32_MAX - 1 || num_edges < 0 || num_edges > ((int64_t)1 << 40))
    return fail(h, KCORE_ERR_INVALID, "n or number of edges out of range");
  if (!offsets_out || !m_out) return fail(h, KCORE_ERR_INVALID, "null offsets_out/m_out");
  if (num_edges > 0 && (!src || !dst || !adj_out)) return fail(h, KCORE_ERR_INVALID, "null edge or adj pointer");
  if (n == 0 && num_edges > 0) return fail(h, KCORE_ERR_INVALID, "edges given for an empty vertex set");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  h->last_ctl = nullptr;
  h->last_trace = nullptr;
  h->last_batch_status = nullptr;
  h->last_stream = stream;
  h->pending = true;
  h->last_validate_status = nullptr;
  kc::CsrLayout L = kc::csr_layout(n, num_edges, h->sms);
  kcore_status st = ensure_ws(h, L.total);
  if (st != KCORE_OK) return st;
  cudaError_t e = kc::csr_build_launch(L, (char*)h->ws, n, num_edges, src, dst, nullptr, nullptr, 0,
                                       (long long*)offsets_out, adj_out, (long long*)m_out, stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "CSR build launch");
  h->last_csr_status = (int*)((char*)h->ws + L.status);
  return KCORE_OK;
}

namespace {
struct BatchLayout {
  size_t ctl, order, deg, a0, a1, f0, f1, total;
};
BatchLayout batch_layout(int64_t G, int64_t N) {
  BatchLayout L{};
  size_t off = 0;
  L.ctl = off;
  off = align_up(off + 256, 256);
  L.order = off;
  off = align_up(off + 4 * (size_t)std::max<int64_t>(G, 1), 256);
  L.deg = off;
  off = align_up(off + 4 * (size_t)N, 256);
  L.a0 = off;
  off = align_up(off + 4 * (size_t)N, 256);
  L.a1 = off;
  off = align_up(off + 4 * (size_t)N, 256);
  L.f0 = off;
  off = align_up(off + 4 * (size_t)N, 256);
  L.f1 = off;
  off = align_up(off + 4 * (size_t)N, 256);
  L.total = off;
  return L;
}

// Batched launch shape from the handle's options: block size, vertices kept in
// shared memory, CTAs per SM.
void batch_shape(kcore_ctx* h, int* block, int* smem_vertices, int* grid, size_t* smem) {
  int b = (int)h->opt[KCORE_OPT_BATCH_BLOCK];
  int sv = (int)h->opt[KCORE_OPT_BATCH_SMEM_VERTICES];
  int cps = (int)h->opt[KCORE_OPT_BATCH_CTAS_PER_SM];
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  int sm_total = 0;
  cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  size_t stat = kc::batch_static_smem(b);
  if (sv < 0) {
    // default: two CTAs per SM share the SM's shared memory
    int want = cps > 0 ? cps : 2;
    long long per = (long long)sm_total / want - (long long)stat - 2048;
    per = std::min<long long>(per, (long long)dev_smem - (long long)stat - 1024);
    sv = (int)std::max<long long>(0, per / 4);
  }
  size_t sm = (size_t)sv * 4;
  if (sm + stat > (size_t)dev_smem) {
    sv = (int)(((size_t)dev_smem - stat - 1024) / 4);
    sm = (size_t)sv * 4;
  }
  int occ = kc::batch_occupancy(b, sm);
  if (occ < 1) occ = 1;
  if (cps > 0) occ = std::min(occ, cps);
  *block = b;
  *smem_vertices = sv;
  *grid = h->sms * occ;
  *smem = sm;
}

}  // namespace
extern "C++" {
namespace {
size_t single_batched_bytes(int64_t n) { return batch_layout(1, n).total + 256; }

// Mode 4: the whole graph on one CTA of 1,024 threads (induced degrees in
// shared memory when they fit in one SM's), or on one thread-block cluster of
// KCORE_OPT_BATCH_CLUSTER CTAs: the batched peel's kernel on a batch of one.
kcore_status single_batched_call(kcore_ctx* h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                                 int32_t* out, int32_t* kmax_out, cudaStream_t stream) {
  const BatchLayout L = batch_layout(1, n);
  kcore_status st = ensure_ws(h, L.total + 256);
  if (st != KCORE_OK) return st;
  char* ws = (char*)h->ws;
  int dev_smem = 0, sm_total = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  const long long stat = (long long)kc::batch_static_smem(1024) + 256;  // + the cluster counters
  const long long per = std::min<long long>((long long)sm_total - stat - 2048, (long long)dev_smem - stat - 1024);
  // shared memory only as large as the graph's induced degrees (32 bits, or 16
  // when every degree is below 2^16, which the kernel finds out); none when
  // even 16 bits do not fit, so the SM keeps its L1 for the global accesses
  const long long cap = std::max<long long>(0, per / 4);
  const int sv = (int)(n <= cap ? n : ((n + 1) / 2 <= cap ? (n + 1) / 2 : 0));
  const int cluster = h->opt[KCORE_OPT_BATCH_CLUSTER] > 1 ? (int)h->opt[KCORE_OPT_BATCH_CLUSTER] : 0;
  kc::BatchArgs a{};
  a.G = 1;
  a.N = n;
  a.m = m;
  a.gv = (const long long*)(ws + L.total);
  a.off = (const long long*)offsets;
  a.adj = adj;
  a.core = out;
  a.kmax = kmax_out;
  a.deg = (int*)(ws + L.deg);
  a.A0 = (int*)(ws + L.a0);
  a.A1 = (int*)(ws + L.a1);
  a.F0 = (int*)(ws + L.f0);
  a.F1 = (int*)(ws + L.f1);
  a.order = nullptr;
  a.next_graph = (int*)(ws + L.ctl);
  a.status = (int*)(ws + L.ctl) + 32;
  a.smem_deg_max = sv;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws + L.ctl, 0, 256, stream)) != cudaSuccess) return cuda_fail(h, e, "memset");
  if ((e = kc::batch_single_gv((long long*)(ws + L.total), n, stream)) != cudaSuccess)
    return cuda_fail(h, e, "graph offsets");
  if ((e = kc::batch_launch(a, 1024, cluster ? cluster : 1, (size_t)sv * 4, false, stream, cluster, 1)) !=
      cudaSuccess)
    return cuda_fail(h, e, "single-graph launch on the batched kernel");
  h->last_batch_status = a.status;
  h->last_batch_block = 1024;
  h->last_batch_grid = cluster ? cluster : 1;
  h->last_batch_smem_vertices = sv;
  h->last_batch_cluster = cluster;
  h->last_batch_single = true;
  return KCORE_OK;
}
}  // namespace
}  // extern "C++"

kcore_status kcore_batched_workspace_size(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                          size_t* bytes) {
  if (!h || !bytes || num_graphs < 0 || total_vertices < 0) return KCORE_ERR_INVALID;
  *bytes = batch_layout(num_graphs, total_vertices).total;
  return KCORE_OK;
}

kcore_status kcore_decompose_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                     int64_t total_arcs, const int64_t* graph_vertex_offsets,
                                     const int64_t* offsets, const int32_t* adj, int32_t* coreness_out,
                                     int32_t* kmax_out, kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (num_graphs < 0 || total_vertices < 0 || total_arcs < 0 || num_graphs > ((int64_t)1 << 24))
    return fail(h, KCORE_ERR_INVALID, "batch sizes out of range");
  if (num_graphs > 0 && (!graph_vertex_offsets || !kmax_out))
    return fail(h, KCORE_ERR_INVALID, "null graph offsets / kmax");
  if (total_vertices > 0 && (!offsets || !coreness_out)) return fail(h, KCORE_ERR_INVALID, "null offsets / coreness");
  if (total_arcs > 0 && !adj) return fail(h, KCORE_ERR_INVALID, "null adj");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  h->stats = kcore_stats{};
  h->last_ctl = nullptr;
  h->last_trace = nullptr;
  h->last_csr_status = nullptr;
  h->last_batch_status = nullptr;
  h->last_stream = stream;
  h->pending = true;
  h->last_validate_status = nullptr;
  if (num_graphs == 0) return KCORE_OK;
  BatchLayout L = batch_layout(num_graphs, total_vertices);
  kcore_status st = ensure_ws(h, L.total);
  if (st != KCORE_OK) return st;
  char* ws = (char*)h->ws;
  int block, sv, grid;
  size_t smem;
  batch_shape(h, &block, &sv, &grid, &smem);
  kc::BatchArgs a{};
  a.G = num_graphs;
  a.N = total_vertices;
  a.m = total_arcs;
  a.gv = (const long long*)graph_vertex_offsets;
  a.off = (const long long*)offsets;
  a.adj = adj;
  a.core = coreness_out;
  a.kmax = kmax_out;
  a.deg = (int*)(ws + L.deg);
  a.A0 = (int*)(ws + L.a0);
  a.A1 = (int*)(ws + L.a1);
  a.F0 = (int*)(ws + L.f0);
  a.F1 = (int*)(ws + L.f1);
  bool sort_graphs = num_graphs <= kc::kMaxSortGraphs && num_graphs > 1;
  a.order = sort_graphs ? (const int*)(ws + L.order) : nullptr;
  a.next_graph = (int*)(ws + L.ctl);
  a.status = (int*)(ws + L.ctl) + 32;
  a.smem_deg_max = sv;
  const int cluster = (int)h->opt[KCORE_OPT_BATCH_CLUSTER];
  if (cluster > 1 && block != 512 && block != 1024)
    return fail(h, KCORE_ERR_INVALID, "a clustered batch needs 512 or 1024 threads per CTA");
  long long big_arcs = (long long)h->opt[KCORE_OPT_BATCH_BIG_ARCS];
  if (big_arcs == 0) big_arcs = std::max<long long>(1, total_arcs / std::max(grid, 1));
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws + L.ctl, 0, 256, stream)) != cudaSuccess) return cuda_fail(h, e, "memset");
  if ((e = kc::batch_launch(a, block, grid, smem, sort_graphs, stream, cluster, big_arcs)) != cudaSuccess)
    return cuda_fail(h, e, "batched launch");
  h->last_batch_cluster = cluster > 1 ? cluster : 0;
  h->last_batch_single = false;
  h->last_batch_status = a.status;
  h->last_batch_block = block;
  h->last_batch_grid = grid;
  h->last_batch_smem_vertices = sv;
  return KCORE_OK;
}

kcore_status kcore_build_csr_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                     int64_t num_edges, int64_t max_graph_vertices,
                                     const int64_t* graph_vertex_offsets, const int64_t* graph_edge_offsets,
                                     const int32_t* src, const int32_t* dst, int64_t* offsets_out,
                                     int32_t* adj_out, int64_t* m_out, kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (num_graphs < 1 || total_vertices < 0 || total_vertices > INT32_MAX - 1 || num_edges < 0 ||
      num_edges > ((int64_t)1 << 40) || max_graph_vertices < 1 || max_graph_vertices > total_vertices + 1)
    return fail(h, KCORE_ERR_INVALID, "batch CSR sizes out of range");
  if (!graph_vertex_offsets || !graph_edge_offsets || !offsets_out || !m_out)
    return fail(h, KCORE_ERR_INVALID, "null pointer");
  if (num_edges > 0 && (!src || !dst || !adj_out)) return fail(h, KCORE_ERR_INVALID, "null edge or adj pointer");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  h->last_ctl = nullptr;
  h->last_trace = nullptr;
  h->last_batch_status = nullptr;
  h->last_stream = stream;
  h->pending = true;
  h->last_validate_status = nullptr;
  kc::CsrLayout L = kc::csr_layout(total_vertices, num_edges, h->sms, max_graph_vertices);
  kcore_status st = ensure_ws(h, L.total);
  if (st != KCORE_OK) return st;
  cudaError_t e = kc::csr_build_launch(L, (char*)h->ws, total_vertices, num_edges, src, dst,
                                       (const long long*)graph_vertex_offsets,
                                       (const long long*)graph_edge_offsets, num_graphs,
                                       (long long*)offsets_out, adj_out, (long long*)m_out, stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched CSR build launch");
  h->last_csr_status = (int*)((char*)h->ws + L.status);
  return KCORE_OK;
}

kcore_status kcore_sync_status(kcore_handle h) {
  if (!h) return KCORE_ERR_INVALID;
  DeviceGuard g(h->device);
  if (!h->pending) return KCORE_OK;
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  h->pending = false;
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  if (h->last_batch_status) {
    int bs[4] = {0, 0, 0, 0};
    e = cudaMemcpy(bs, h->last_batch_status, sizeof(bs), cudaMemcpyDeviceToHost);
    h->last_batch_status = nullptr;
    if (e != cudaSuccess) return cuda_fail(h, e, "read status");
    h->stats.grid = h->last_batch_grid;
    h->stats.batch_block = h->last_batch_block;
    h->stats.batch_smem_vertices = h->last_batch_smem_vertices;
    h->stats.batch_cluster = h->last_batch_cluster;
    if (h->last_batch_single) h->stats.sync_mode = 4;
    if (bs[0] == kc::ST_NOT_SIMPLE) {
      long long val = (long long)(unsigned)bs[2] | ((long long)bs[3] << 32);
      if (h->last_batch_single)
        return fail(h, KCORE_ERR_NOT_SIMPLE,
                    "malformed CSR detected on the device (check " + std::to_string(bs[1]) + ", value " +
                        std::to_string(val) + "); k_max is -1");
      return fail(h, KCORE_ERR_NOT_SIMPLE,
                  "malformed segmented CSR detected on the device (check " + std::to_string(bs[1]) +
                      ", value " + std::to_string(val) + "); the graphs concerned report k_max -1");
    }
    if (bs[0] != 0) return fail(h, KCORE_ERR_CUDA, "unknown device status " + std::to_string(bs[0]));
    return KCORE_OK;
  }
  if (h->last_validate_status) {
    long long vs[4] = {0, 0, 0, 0};
    e = cudaMemcpy(vs, h->last_validate_status, sizeof(vs), cudaMemcpyDeviceToHost);
    h->last_validate_status = nullptr;
    if (e != cudaSuccess) return cuda_fail(h, e, "read status");
    const int code = (int)(vs[0] & 0xffffffff);
    static const char* what[] = {"",
                                 "offsets not monotone or outside [0, m]",
                                 "offsets[0] != 0 or offsets[n] != m",
                                 "neighbour id outside [0, n)",
                                 "self-loop",
                                 "list not strictly ascending (repeated arc or unsorted)",
                                 "arc without its reverse (not symmetric)"};
    if (code == 0) return KCORE_OK;
    if (code < 0 || code > 6) return fail(h, KCORE_ERR_CUDA, "unknown check code " + std::to_string(code));
    h->stats.invalid_check = code;
    h->stats.invalid_vertex = vs[1];
    h->stats.invalid_arc = vs[2];
    return fail(h, KCORE_ERR_NOT_SIMPLE,
                std::string("CSR is not simple: ") + what[code] + " (vertex " + std::to_string(vs[1]) +
                    ", arc " + std::to_string(vs[2]) + ")");
  }
  if (h->last_csr_status) {
    int cs = 0;
    e = cudaMemcpy(&cs, h->last_csr_status, sizeof(int), cudaMemcpyDeviceToHost);
    h->last_csr_status = nullptr;
    if (e != cudaSuccess) return cuda_fail(h, e, "read status");
    if (cs != 0) return fail(h, KCORE_ERR_INVALID, "edge list holds a vertex id outside [0, n)");
    return KCORE_OK;
  }
  if (!h->last_ctl) return KCORE_OK;
  kc::PeelCtl c;
  e = cudaMemcpy(&c, h->last_ctl, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "read status");
  if (h->last_ctl2) {
    // sampled call: sampling counters from its run; the peel counters from the
    // rerun when it ran
    h->stats.sample_vertices = c.s_sampled;
    h->stats.sample_recounts = c.s_recounts;
    h->stats.sample_bag = c.s_bag;
    h->stats.sample_failed_validations = c.s_failed;
    h->stats.sample_heads = c.s_heads;
    h->stats.sample_reruns = c.s_redo ? 1 : 0;
    h->stats.sample_miss_round = c.s_miss ? c.s_miss_round : -1;
    if (c.s_redo && c.status == 0) {
      e = cudaMemcpy(&c, h->last_ctl2, sizeof(c), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(h, e, "read status");
    }
  }
  h->stats.rounds = c.rounds;
  h->stats.empty_rounds = c.empty_rounds;
  h->stats.items = (int64_t)c.items;
  h->stats.local_items = (int64_t)c.local_items;
  h->stats.scanned = c.scanned;
  h->stats.kmax = c.kmax;
  h->stats.grid = h->last_grid;
  h->stats.sync_mode = h->last_mode;
  h->stats.passes = c.passes;
  h->stats.barriers = c.barriers;
  h->stats.tail_phases = c.tail_phases;
  h->stats.tail_episodes = c.tail_episodes;
  h->stats.slice_arcs = h->last_slice;
  switch (c.status) {
    case 0:
      return KCORE_OK;
    case kc::ST_TIMEOUT:
      return fail(h, KCORE_ERR_TIMEOUT, "a device-side wait exceeded its time limit");
    case kc::ST_NOT_SIMPLE:
      return fail(h, KCORE_ERR_NOT_SIMPLE, "malformed CSR detected on the device (offsets or ids out of range)");
    case kc::ST_CAPACITY:
      return fail(h, KCORE_ERR_CAPACITY, "an internal bound was exceeded");
    default:
      return fail(h, KCORE_ERR_CUDA, "unknown device status " + std::to_string(c.status));
  }
}

kcore_status kcore_get_trace(kcore_handle h, uint64_t* out, int64_t max_rounds, int64_t* rounds_out) {
  if (!h || !out || !rounds_out || max_rounds < 0) return KCORE_ERR_INVALID;
  *rounds_out = 0;
  if (!h->last_trace) return fail(h, KCORE_ERR_INVALID, "the last decomposition ran without tracing");
  DeviceGuard g(h->device);
  // the bulk-synchronous modes record one entry per non-empty level, or per
  // phase (grid barrier or tail phase) with trace mode 2
  const int64_t have = h->last_trace_phases ? h->stats.barriers + h->stats.tail_phases
                       : h->last_mode != 1  ? h->stats.rounds - h->stats.empty_rounds
                                            : h->stats.rounds;
  int64_t r = std::min<int64_t>(std::min<int64_t>(max_rounds, have), h->last_max_rounds);
  if (r > 0) {
    cudaError_t e = cudaMemcpy(out, h->last_trace, sizeof(uint64_t) * kc::kTraceFields * (size_t)r,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "read trace");
  }
  *rounds_out = r;
  return KCORE_OK;
}

kcore_status kcore_barrier_latency(kcore_handle h, int64_t grid, int32_t iters, double* ns_out) {
  if (!h || !ns_out || iters < 1 || iters > 1000000 || grid < 0) return KCORE_ERR_INVALID;
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, KCORE_ERR_CUDA, "cudaSetDevice failed");
  h->err.clear();
  const long long gmax = (long long)h->sms * h->bsp_max_ctas_per_sm;
  if (grid > gmax) return fail(h, KCORE_ERR_INVALID, "grid above the co-resident maximum");
  const int ctas = grid > 0 ? (int)grid : (int)gmax;
  if (h->pending && h->last_stream) cudaStreamSynchronize(h->last_stream);
  h->pending = false;
  h->last_ctl = nullptr;
  h->last_trace = nullptr;
  h->last_csr_status = nullptr;
  h->last_batch_status = nullptr;
  h->last_validate_status = nullptr;
  const size_t ctl_bytes = align_up(sizeof(kc::PeelCtl), 256);
  kcore_status st = ensure_ws(h, ctl_bytes + 256);
  if (st != KCORE_OK) return st;
  char* ws = (char*)h->ws;
  kc::PeelArgs a{};
  a.ctl = (kc::PeelCtl*)ws;
  a.timeout_ns = (unsigned long long)h->opt[KCORE_OPT_TIMEOUT_MS] * 1000000ull;
  a.poll_sleep_ns = (int)h->opt[KCORE_OPT_POLL_SLEEP_NS];
  unsigned long long* d_ns = (unsigned long long*)(ws + ctl_bytes);
  cudaError_t e;
  unsigned long long ns = 0;
  int status = 0;
  if ((e = cudaMemset(ws, 0, ctl_bytes + 256)) != cudaSuccess) return cuda_fail(h, e, "memset");
  if ((e = kc::bsp_barrier_probe(a, ctas, iters, d_ns, nullptr)) != cudaSuccess)
    return cuda_fail(h, e, "barrier probe launch");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(h, e, "barrier probe");
  if ((e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(h, e, "read probe");
  if ((e = cudaMemcpy(&status, &a.ctl->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(h, e, "read status");
  if (status == kc::ST_TIMEOUT) return fail(h, KCORE_ERR_TIMEOUT, "a barrier wait exceeded its time limit");
  *ns_out = (double)ns / iters;
  return KCORE_OK;
}

kcore_status kcore_get_stats(kcore_handle h, kcore_stats* out) {
  if (!h || !out) return KCORE_ERR_INVALID;
  *out = h->stats;
  return KCORE_OK;
}

kcore_status kcore_decompose_host(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets_host,
                                  const int32_t* adj_host, int32_t* coreness_host,
                                  int32_t* kmax_host, kcore_stream_t stream_) {
  if (!h) return KCORE_ERR_INVALID;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n < 0 || m < 0 || n > INT32_MAX - 1) return fail(h, KCORE_ERR_INVALID, "n or m out of range");
  if (!kmax_host || (n > 0 && (!offsets_host || !coreness_host)) || (m > 0 && !adj_host))
    return fail(h, KCORE_ERR_INVALID, "null host pointer");
  DeviceGuard g(h->device);
  size_t b_off = align_up(8 * (size_t)(n + 1), 256), b_adj = align_up(4 * (size_t)m, 256);
  size_t b_core = align_up(4 * (size_t)n, 256);
  size_t need = b_off + b_adj + b_core + 256;
  if (h->e2e_bytes < need) {
    if (h->e2e) {
      cudaDeviceSynchronize();
      cudaFree(h->e2e);
      h->e2e = nullptr;
      h->e2e_bytes = 0;
    }
    if (cudaMalloc(&h->e2e, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, KCORE_ERR_OOM, "cudaMalloc of host-path staging failed");
    }
    h->e2e_bytes = need;
  }
  char* p = (char*)h->e2e;
  int64_t* d_off = (int64_t*)p;
  int32_t* d_adj = (int32_t*)(p + b_off);
  int32_t* d_core = (int32_t*)(p + b_off + b_adj);
  int32_t* d_kmax = (int32_t*)(p + b_off + b_adj + b_core);
  cudaError_t e;
  if (n > 0 && (e = cudaMemcpyAsync(d_off, offsets_host, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
    return cuda_fail(h, e, "copy offsets");
  if (m > 0 && (e = cudaMemcpyAsync(d_adj, adj_host, 4 * (size_t)m, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
    return cuda_fail(h, e, "copy adj");
  kcore_status st = kcore_decompose(h, n, m, d_off, d_adj, d_core, d_kmax, stream_);
  if (st != KCORE_OK) return st;
  if (n > 0 && (e = cudaMemcpyAsync(coreness_host, d_core, 4 * (size_t)n, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return cuda_fail(h, e, "copy coreness");
  if ((e = cudaMemcpyAsync(kmax_host, d_kmax, 4, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return cuda_fail(h, e, "copy kmax");
  return kcore_sync_status(h);
}

}  // extern "C"
