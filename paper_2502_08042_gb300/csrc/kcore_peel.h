// Host/device shared declarations of the single-graph peel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kc {

// Device status codes (same values as kcore_status).
enum : int { ST_OK = 0, ST_TIMEOUT = 4, ST_NOT_SIMPLE = 5, ST_CAPACITY = 6 };

constexpr int kLocalQueueMax = 128;
constexpr int kHandoff = 8;  // words of loop state CTA 0 hands the parked CTAs (tail mode)
// Options of a handle (kcore_option values 0 .. kNumOptions - 1) and the
// tail-mode defaults: off, because every threshold measured on GB300 was
// slower on R-MAT scale 24 and the kNN workload (kcore_autotune tries it).
constexpr int kNumOptions = 30;
constexpr long long kTailItemsDefault = 0;
constexpr long long kTailEntriesDefault = 0;
constexpr long long kParkSleepDefault = 256;
// Defaults of the bulk-synchronous schedule (sync mode 2), shared by the
// handle's options and the no-allocation entry point.
constexpr int kSliceDefault = 32;          // arcs per work item (measured on R-MAT 24: 32 16.45 ms,
                                           // 64 16.65; kNN equal)
constexpr int kLocalQueueDefault = 128;    // per-warp local queue (items)
constexpr int kLocalBatchesDefault = 32;   // local batches per chunk taken
constexpr int kPrecheckDefault = 64;       // per-warp share from which d~ is read first
constexpr int kPollSleepDefault = 64;      // grid-barrier poll sleep (ns)
constexpr int kTimeoutMsDefault = 2000;    // limit of every device-side wait
constexpr int kScanMin = 512;              // active-list entries per scanning CTA (at least; measured
                                           // on R-MAT 24 / kNN: 2048 17.0 / 6.03 ms, 1024 16.8 / 5.82,
                                           // 512 16.7 / 5.72)
constexpr int kMinSlice = 16;  // keeps slice indices below 2^27 (27-bit field of a work item)

// Per-round record (zeroed before launch). Each hot word has its own 128-byte
// line: the termination counter, the queue's claim and append counters.
struct RoundRec {
  unsigned long long cnt;  // (scan tokens << 40) + outstanding work items
  char pad0[120];
  unsigned long long head;  // tickets handed out in this round's queue segment
  char pad1[120];
  unsigned long long tail;  // items appended to this round's queue segment
  char pad2[120];
  unsigned long long found;  // frontier vertices claimed by the scan
  unsigned long long alen;   // length of the next active list
  int minkey;                // max over survivors of INT_MAX - d~ (0: no survivor)
  int pad3;
  unsigned long long rcount;  // sampling: vertices appended to the recount list
  unsigned long long rqtail;  // sampling: recount slices appended
  char pad4[88];
};

// Round-completion broadcast: the thread whose counter update finishes round r
// copies the round's results here and then publishes round = r + 1. Each CTA
// polls one of kDoneLines copies, so no single cache line takes every poll.
constexpr int kDoneLines = 16;
struct DoneLine {
  int round;
  int minkey;
  unsigned long long found, alen, tail;
  char pad[96];
};

// Device control block (zeroed before launch).
struct PeelCtl {
  DoneLine done[kDoneLines];
  int status;
  int pad1[31];
  unsigned long long progress;  // heartbeat of long single-warp chains
  char pad2[120];
  unsigned long long items, local_items;
  long long rounds, empty_rounds, scanned, kmax;
  char pad3[80];
  // bulk-synchronous mode: the grid barrier's words (barrier g uses word
  // g % 3: arrivals, the phase's queue appends, the abort bit; reset two
  // phases ahead), subround passes and barriers taken
  struct {
    unsigned long long v;
    char pad[120];
  } bar_ring[3];
  long long passes, barriers;
  unsigned long long tr_arcs, tr_decs;  // bulk-synchronous mode, with tracing: running sums
  unsigned long long crossed;           // k'-core query: vertices removed by a decrement
  char pad7[88];
  // sampling (Sec. 4.1): vertices sampled by the first InitSampler, recounts,
  // counting-bag insertions, failed validations, heads; a detected miss (the
  // flag, its round and vertex) and a failed final check
  long long s_sampled, s_recounts, s_bag, s_failed, s_heads;
  int s_miss, s_miss_round;
  long long s_miss_vertex;
  int s_redo;  // 1: the sampled run's result is not exact (miss or failed check); rerun without sampling
  int pad8[23];
  // tail mode (bulk-synchronous mode): CTA 0's releases of the parked CTAs
  // (bit 63: a status was raised), the loop state it hands over with each
  // release, and its counts of tail phases and episodes
  unsigned long long tail_word;
  char pad9[120];
  unsigned long long handoff[kHandoff];
  long long tail_phases, tail_episodes;
  char pad10[48];
};

// The bulk-synchronous mode uses round records 0..2 as a ring: phase p uses
// record p % 3 (reset during phase p - 1, last read during phase p - 2).
constexpr int kPhaseRing = 3;

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
  int scan_min;  // active-list entries per scanning CTA (at least)
  unsigned long long timeout_ns;
  int idle_sleep_ns;  // sleep of a waiting warp between looks at its ticket slots
  int poll_sleep_ns;  // sleep of the CTA's round poller between polls
  int inject_stall;
  unsigned long long* trace;  // optional: kTraceFields words per round (nullptr = off)
  int trace_phases;           // bulk-synchronous mode: one trace record per phase instead of per level
  int local_batches;          // bulk-synchronous mode: local batches per chunk taken
  int precheck_items;         // bulk-synchronous mode: per-warp share of a pass from which d~ is read first
  // k'-core query (bulk-synchronous mode only): one peel at level kprime - 1
  // taking every vertex below kprime; core[] receives 1 (in the k'-core) or 0
  int threshold;
  int kprime;
  long long* size_out;  // optional: the k'-core's vertex count
  // offline subrounds (sync mode 3, Algorithm 2): per-vertex decrement
  // counts (zero at launch, left zero) and the touched list of a subround
  int offline;
  int* hcnt;
  int* touched;
  // level window (bucketing of the active list, sync mode 2): 0 = off, else
  // the number of levels a rebuild scan serves; A2 is the third list buffer
  int window;
  int* A2;
  // heavy subrounds over a short active list use Algorithm 2's batch update
  // (counts in hcnt, zero at launch and left zero)
  int hybrid;

  // sampling (Sec. 4.1, Algorithms 4-5; bulk-synchronous mode): a vertex in
  // sample mode keeps -1 - D in deg[] (D: its induced degree at InitSampler).
  // scnt: heads since InitSampler; stamp: the pass that traverses a vertex's
  // arcs (INT_MAX before it is assigned); racc / rst: recount accumulators
  // (zero between recounts); rlist: vertices to recount; RQ / RQv: their
  // adjacency slices and owners (rqcap entries of rslice arcs at most).
  int sample;
  int mu;                  // heads that fill the counting bag
  long long sthreshold;    // sample mode needs D > sthreshold (and D r > k)
  unsigned long long seed; // Philox key of the coins
  unsigned long long coin_lim;  // floor(10 mu 2^32 / 9): a coin x is a head when D (x + 1) <= coin_lim
  int* scnt;
  int* stamp;
  int* racc;
  int* rst;
  int* rlist;
  unsigned long long* RQ;
  int* RQv;
  long long rqcap;
  int rslice;
  // when set, the kernel runs only if *run_if != 0 (the rerun after a sampled
  // run that was not exact)
  const int* run_if;
  // bulk-synchronous mode: the lanes of a warp that decrement the same vertex
  // in the same step send one atomic of their count (warp aggregation)
  int combine;
  // tail mode (bulk-synchronous mode, plain schedule): a subround pass of at
  // most tail_items queue items, or a scan of at most tail_entries active-list
  // entries, runs on CTA 0 alone (0 disables either); the other CTAs park,
  // sleeping park_sleep_ns between polls
  long long tail_items, tail_entries;
  int park_sleep_ns;
};

// Per-round trace record (KCORE_OPT_TRACE): globaltimer at round start (CTA 0),
// when the last scan token arrived, when the round finished; the level, the
// active-list length scanned, frontier vertices found, items queued, the
// scanning CTAs, arcs read, decrements issued, the longest scan of one CTA
// (ns), the latest round start of a CTA after CTA 0's (ns), the summed time
// warps spent in work batches (ns) and the number of batches. The
// bulk-synchronous mode writes one record per non-empty level, with 0 in
// fields 10..12 and its subround passes in field 13.
constexpr int kTraceFields = 14;

int peel_max_ctas_per_sm();
int peel_block_size();
cudaError_t peel_launch(const PeelArgs& args, int grid, cudaStream_t stream);

// Bulk-synchronous mode (grid barrier between scan and subround phases).
int bsp_max_ctas_per_sm();
int bsp_block_size();
cudaError_t bsp_launch(const PeelArgs& args, int grid, cudaStream_t stream);
// Grid-barrier latency probe: `iters` barriers with no work between them
// (ctl zeroed by the caller); *out_ns (device) receives the elapsed time.
cudaError_t bsp_barrier_probe(const PeelArgs& args, int grid, int iters, unsigned long long* out_ns,
                              cudaStream_t stream);

// Final check of a sampled run (sample.cu): every v must have at least
// core[v] neighbours u with core[u] >= core[v]; a failure sets ctl->s_redo.
// Skipped when ctl->s_redo is already set. acc: device int[n], zero on entry
// and left zero.
cudaError_t sample_check_launch(long long n, long long m, const long long* off, const int* adj, const int* core,
                                int* acc, PeelCtl* ctl, int sms, cudaStream_t stream);

// Simple-CSR check (validate.cu). st: device int[8] (code, pad, vertex, arc as
// int64); zeroed by the launch, code 0 when the CSR is simple.
cudaError_t validate_launch(long long n, long long m, const long long* off, const int* adj, int* st, int sms,
                            cudaStream_t stream);

}  // namespace kc
