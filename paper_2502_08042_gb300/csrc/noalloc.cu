// kcore_decompose_static: the single-graph decomposition for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: the device memory of their process may
// be fully reserved by another allocator (a framework's caching pool), their
// policy may forbid allocation once start-up is over, or they cannot afford
// the device-wide synchronisation an allocation can cause. This entry point
// runs the same peel kernel as kcore_decompose, but its scratch memory (the
// induced degrees, the two active lists, the work queue, the per-round records
// and the control block) lives in one file-scope __device__ array of fixed
// size, which every GPU that loads the library holds until the process exits.
// The caller still provides the graph and the output arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "kcore.h"
#include "kcore_peel.h"

namespace {

constexpr long long kStaticMaxN = KCORE_STATIC_MAX_VERTICES;
constexpr long long kStaticMaxM = KCORE_STATIC_MAX_ARCS;
constexpr int kStaticSlice = 128;
constexpr long long kStaticQcap = kStaticMaxN + (kStaticMaxM + kStaticSlice - 1) / kStaticSlice + 1;
// levels: 2 * sqrt(m) + 8 rounds at most (see the handle's workspace layout)
constexpr int kStaticMaxRounds = 2 * 4096 + 8;
static_assert((long long)4096 * 4096 == kStaticMaxM, "round bound assumes m <= 2^24");

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffRounds = al256(sizeof(kc::PeelCtl));
constexpr size_t kOffDeg = al256(kOffRounds + sizeof(kc::RoundRec) * (size_t)kStaticMaxRounds);
constexpr size_t kOffA0 = al256(kOffDeg + 4 * (size_t)kStaticMaxN);
constexpr size_t kOffA1 = al256(kOffA0 + 4 * (size_t)kStaticMaxN);
constexpr size_t kOffQ = al256(kOffA1 + 4 * (size_t)kStaticMaxN);
constexpr size_t kStaticBytes = al256(kOffQ + 8 * (size_t)kStaticQcap);

constexpr int kMaxDevices = 64;
struct StaticDev {
  bool ready = false;
  char* scratch = nullptr;  // device address of g_kcore_static_scratch on this device
  int sms = 0;
  int ctas_per_sm = 0;
};
StaticDev g_dev[kMaxDevices];
std::mutex g_setup_mu;

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
    // one-time set-up on this device (the device is current here)
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
  if (n == 0) {
    if ((e = cudaMemsetAsync(kmax_out, 0, sizeof(int32_t), stream)) != cudaSuccess) goto cuda_error;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) goto cuda_error;
    return KCORE_OK;
  }
  {
    long long isq = (long long)std::sqrt((double)m);
    while (isq > 0 && isq * isq > m) isq--;
    while ((isq + 1) * (isq + 1) <= m) isq++;
    int max_rounds = (int)std::min<long long>(2 * isq + 8, 2 * n + 8);
    long long qcap = n + (m + kStaticSlice - 1) / kStaticSlice + 1;
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
    a.Q = (unsigned long long*)(ws + kOffQ);
    a.qcap = qcap;
    a.rounds = (kc::RoundRec*)(ws + kOffRounds);
    a.max_rounds = max_rounds;
    a.ctl = (kc::PeelCtl*)(ws + kOffCtl);
    a.slice = kStaticSlice;
    a.lq_cap = 32;
    a.max_take = 256;
    a.scan_min = 2048;
    a.idle_sleep_ns = 192;
    a.poll_sleep_ns = 64;
    a.timeout_ns = 2000ull * 1000000ull;
    a.inject_stall = 0;
    a.trace = nullptr;
    long long gmax = (long long)d.sms * d.ctas_per_sm;
    long long want = (n + m / 8 + 2047) / 2048;
    int grid = (int)std::max<long long>(1, std::min(want, gmax));
    a.take_div = grid * (kc::bsp_block_size() / 32);
    a.local_batches = 8;
    a.precheck_items = 64;
    // the array keeps the previous call's contents: clear what must start at
    // zero (control block, this call's round records); the bulk-synchronous
    // peel reads only queue slots written earlier in the same call
    if ((e = cudaMemsetAsync(ws + kOffCtl, 0, kOffRounds + sizeof(kc::RoundRec) * (size_t)max_rounds,
                             stream)) != cudaSuccess)
      goto cuda_error;
    if ((e = kc::bsp_launch(a, grid, stream)) != cudaSuccess) goto cuda_error;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) goto cuda_error;
    int status = 0;
    if ((e = cudaMemcpy(&status, &((kc::PeelCtl*)(ws + kOffCtl))->status, sizeof(int),
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
      goto cuda_error;
    switch (status) {
      case 0: return KCORE_OK;
      case kc::ST_TIMEOUT: return KCORE_ERR_TIMEOUT;
      case kc::ST_NOT_SIMPLE: return KCORE_ERR_NOT_SIMPLE;
      case kc::ST_CAPACITY: return KCORE_ERR_CAPACITY;
      default: return KCORE_ERR_CUDA;
    }
  }
cuda_error:
  cudaGetLastError();
  return KCORE_ERR_CUDA;
}
