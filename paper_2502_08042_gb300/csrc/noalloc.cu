// kcore_decompose_static: the single-graph decomposition for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: the device memory of their process may
// be fully reserved by another allocator (a framework's caching pool), their
// policy may forbid allocation once start-up is over, or they cannot afford
// the device-wide synchronisation an allocation can cause. This entry point
// runs the same peel kernel as kcore_decompose, with the same launch settings
// as a handle's defaults (bulk-synchronous schedule, batch-updated heavy
// subrounds, tail mode off), but its scratch memory (the induced degrees, the two
// active lists, the work queue, the batch-update counts, the three phase
// records and the control block) lives in one file-scope __device__ array of
// fixed size. The caller still provides the graph and the output arrays.
//
// The library is built without relocatable device code, so this file is a
// module of its own: under lazy module loading (the CUDA default) the array
// is created on a device when the first call there looks up its address, and
// it stays until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "kcore.h"
#include "kcore_peel.h"

namespace {

constexpr long long kStaticMaxN = KCORE_STATIC_MAX_VERTICES;
constexpr long long kStaticMaxM = KCORE_STATIC_MAX_ARCS;
constexpr int kStaticSlice = kc::kSliceDefault;
constexpr long long kStaticQcap = kStaticMaxN + (kStaticMaxM + kStaticSlice - 1) / kStaticSlice + 1;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffCtl = 0;
// the bulk-synchronous kernel uses its round records as a ring of three
constexpr size_t kOffRounds = al256(sizeof(kc::PeelCtl));
constexpr size_t kOffDeg = al256(kOffRounds + sizeof(kc::RoundRec) * (size_t)kc::kPhaseRing);
constexpr size_t kOffA0 = al256(kOffDeg + 4 * (size_t)kStaticMaxN);
constexpr size_t kOffA1 = al256(kOffA0 + 4 * (size_t)kStaticMaxN);
constexpr size_t kOffCnt = al256(kOffA1 + 4 * (size_t)kStaticMaxN);
constexpr size_t kOffQ = al256(kOffCnt + 4 * (size_t)kStaticMaxN);
constexpr size_t kStaticBytes = al256(kOffQ + 8 * (size_t)kStaticQcap);
static_assert(kStaticBytes < ((size_t)32 << 20), "the fixed scratch stays below 32 MB");

constexpr int kMaxDevices = 64;
struct StaticDev {
  bool ready = false;
  char* scratch = nullptr;  // device address of g_kcore_static_scratch on this device
  int sms = 0;
  int ctas_per_sm = 0;
};
StaticDev g_dev[kMaxDevices];
std::mutex g_setup_mu;

kcore_status status_of(int device_status) {
  switch (device_status) {
    case kc::ST_OK: return KCORE_OK;
    case kc::ST_TIMEOUT: return KCORE_ERR_TIMEOUT;
    case kc::ST_NOT_SIMPLE: return KCORE_ERR_NOT_SIMPLE;
    case kc::ST_CAPACITY: return KCORE_ERR_CAPACITY;
    default: return KCORE_ERR_CUDA;
  }
}

}  // namespace

// The scratch array. In host code this name is only a stand-in for the symbol,
// never a device address: its address on each device is looked up once with
// cudaGetSymbolAddress while that device is current.
static __device__ __align__(256) unsigned char g_kcore_static_scratch[kStaticBytes];

extern "C" kcore_status kcore_decompose_static(int64_t n, int64_t m, const int64_t* offsets,
                                               const int32_t* adj, int32_t* coreness_out,
                                               int32_t* kmax_out, kcore_stream_t stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n < 0 || m < 0 || !kmax_out) return KCORE_ERR_INVALID;
  if (n > kStaticMaxN || m > kStaticMaxM) return KCORE_ERR_CAPACITY;  // beyond the fixed scratch
  if (n > 0 && (!offsets || !coreness_out)) return KCORE_ERR_INVALID;
  if (m > 0 && !adj) return KCORE_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KCORE_ERR_CUDA;
  }
  {
    // one-time set-up on this device (the device is current here); the
    // address lookup is also what loads this file's module, array included
    std::lock_guard<std::mutex> lock(g_setup_mu);
    StaticDev& d = g_dev[dev];
    if (!d.ready) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_kcore_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KCORE_ERR_CUDA;
      }
      if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return KCORE_ERR_CUDA;
      }
      d.ctas_per_sm = kc::bsp_max_ctas_per_sm();
      if (d.ctas_per_sm <= 0 || d.sms <= 0) return KCORE_ERR_CUDA;
      d.scratch = (char*)p;
      d.ready = true;
    }
  }
  const StaticDev& d = g_dev[dev];
  cudaError_t e;
  int status = 0;
  if (n == 0) {
    if ((e = cudaMemsetAsync(kmax_out, 0, sizeof(int32_t), stream)) != cudaSuccess) goto cuda_error;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) goto cuda_error;
    return KCORE_OK;
  }
  {
    char* ws = d.scratch;
    kc::PeelArgs a{};
    a.n = n;
    a.m = m;
    a.off = (const long long*)offsets;
    a.adj = adj;
    a.core = coreness_out;
    a.kmax_out = kmax_out;
    a.deg = (int*)(ws + kOffDeg);
    a.A0 = (int*)(ws + kOffA0);
    a.A1 = (int*)(ws + kOffA1);
    a.A2 = nullptr;  // third list buffer: only the level window uses it
    a.hcnt = (int*)(ws + kOffCnt);
    a.Q = (unsigned long long*)(ws + kOffQ);
    a.qcap = n + (m + kStaticSlice - 1) / kStaticSlice + 1;
    a.rounds = (kc::RoundRec*)(ws + kOffRounds);
    a.max_rounds = kc::kPhaseRing;  // bounds trace records only; no trace is written here
    a.ctl = (kc::PeelCtl*)(ws + kOffCtl);
    // the settings of a handle's default decomposition (sync mode 2)
    a.slice = kStaticSlice;
    a.lq_cap = kc::kLocalQueueDefault;
    a.max_take = 256;
    a.scan_min = kc::kScanMin;
    a.poll_sleep_ns = kc::kPollSleepDefault;
    a.timeout_ns = (unsigned long long)kc::kTimeoutMsDefault * 1000000ull;
    a.local_batches = kc::kLocalBatchesDefault;
    a.precheck_items = kc::kPrecheckDefault;
    a.hybrid = 1;
    a.tail_items = kc::kTailItemsDefault;
    a.tail_entries = kc::kTailEntriesDefault;
    a.park_sleep_ns = (int)kc::kParkSleepDefault;
    a.trace = nullptr;
    const long long gmax = (long long)d.sms * d.ctas_per_sm;
    const long long want = (n + m / 8 + 2047) / 2048;
    const int grid = (int)std::max<long long>(1, std::min(want, gmax));
    a.take_div = grid * (kc::bsp_block_size() / 32);
    // the array keeps the previous call's contents: clear what must start at
    // zero (control block, phase records; the batch-update counts, which a
    // call that ended early may leave behind); the bulk-synchronous peel reads
    // only queue slots written earlier in the same call
    if ((e = cudaMemsetAsync(ws + kOffCtl, 0, kOffDeg, stream)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMemsetAsync(a.hcnt, 0, 4 * (size_t)n, stream)) != cudaSuccess) goto cuda_error;
    if ((e = kc::bsp_launch(a, grid, stream)) != cudaSuccess) goto cuda_error;
    // the device status is read on the caller's stream (pageable destination:
    // the copy returns once the stream has reached it)
    if ((e = cudaMemcpyAsync(&status, &((kc::PeelCtl*)(ws + kOffCtl))->status, sizeof(int),
                             cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      goto cuda_error;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) goto cuda_error;
    return status_of(status);
  }
cuda_error:
  cudaGetLastError();
  return KCORE_ERR_CUDA;
}
