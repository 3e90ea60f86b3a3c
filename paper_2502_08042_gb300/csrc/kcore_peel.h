// Host/device shared declarations of the single-graph peel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kc {

// Device status codes (same values as kcore_status).
enum : int { ST_OK = 0, ST_TIMEOUT = 4, ST_NOT_SIMPLE = 5, ST_CAPACITY = 6 };

constexpr int kLocalQueueMax = 128;

// Per-round record (zeroed before launch).
struct RoundRec {
  unsigned long long cnt;    // (scan tokens << 40) + outstanding work items
  unsigned long long found;  // frontier vertices claimed by the scan
  unsigned long long alen;   // length of the next active list
  int minkey;                // max over survivors of INT_MAX - d~ (0: no survivor)
  int pad;
};

// Device control block (zeroed before launch); hot words on their own lines.
struct PeelCtl {
  unsigned long long qtail;
  char pad0[120];
  unsigned long long qhead;
  char pad1[120];
  int status;
  int pad2[31];
  unsigned long long progress;
  char pad4[120];
  unsigned long long items, local_items;
  long long rounds, empty_rounds, scanned, kmax;
  char pad3[80];
};

struct PeelArgs {
  long long n, m;
  const long long* off;
  const int* adj;
  int* core;
  int* kmax_out;
  int* deg;
  int* A0;
  int* A1;
  unsigned long long* Q;
  long long qcap;
  RoundRec* rounds;
  int max_rounds;
  PeelCtl* ctl;
  int slice;
  int lq_cap;
  int max_take;
  int take_div;
  int max_backoff_ns;
  unsigned long long timeout_ns;
  int inject_stall;
};

int peel_max_ctas_per_sm();
int peel_block_size();
cudaError_t peel_launch(const PeelArgs& args, int grid, cudaStream_t stream);

}  // namespace kc
