/*
 * kcore.h - C ABI of the GB300 (sm_103a) k-core decomposition library.
 *
 * Problem (arXiv 2502.08042, Sec. 2 "Notations"): for a simple undirected
 * graph G, the k-core G_k is the largest subgraph in which every vertex has
 * degree at least k; the coreness of v is the largest k with v in G_k, and
 * k_max is the largest coreness. The library computes the coreness of every
 * vertex by parallel peeling (Algorithm 1 with the online Peel of
 * Algorithm 3): level by level, the live vertices whose induced degree is at
 * most k get coreness k, their live neighbours' induced degrees are decremented
 * atomically, and a neighbour whose decrement lands it on k joins the same
 * level's work.
 *
 * Conventions shared by every entry point:
 *  - Graphs are CSR: int64 offsets[n+1] (offsets[0] = 0, offsets[n] = m) and
 *    int32 adj[m]. m counts arcs: each undirected edge appears twice (u->v and
 *    v->u), so the number of undirected edges is m/2. The graph must be simple
 *    (symmetric, no self-loops, no repeated arcs); kcore_build_csr produces
 *    such a CSR from any edge list. 0 <= n <= 2^31 - 2.
 *  - Pointers marked "device" must be device memory (or managed memory)
 *    readable/writable by the handle's device; "host" pointers are host memory.
 *    The caller owns every array it passes and keeps it alive until the work
 *    queued on `stream` has passed the call.
 *  - Calls taking a stream are asynchronous: they queue work on `stream` and
 *    return. Argument errors are reported synchronously by the return value
 *    and nothing is queued. Errors found on the device (a wait that ran past
 *    its time limit, a malformed graph detected on the device) are reported by
 *    kcore_sync_status. Outputs are undefined after an error.
 *  - No entry point throws; none calls exit(); none takes a torch type.
 *  - A handle is bound to one device and is not thread-safe: use one handle
 *    per host thread (handles share nothing).
 */
#ifndef KCORE_H_
#define KCORE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kcore_ctx* kcore_handle;
typedef struct CUstream_st* kcore_stream_t; /* same type as cudaStream_t; NULL = legacy default stream */

typedef enum {
  KCORE_OK = 0,
  KCORE_ERR_INVALID = 1,    /* bad argument (null pointer, negative size, n too large, ...) */
  KCORE_ERR_OOM = 2,        /* device memory for the workspace could not be obtained */
  KCORE_ERR_CUDA = 3,       /* a CUDA runtime call failed; see kcore_last_error */
  KCORE_ERR_TIMEOUT = 4,    /* a device-side wait exceeded its time limit; the kernel returned */
  KCORE_ERR_NOT_SIMPLE = 5, /* the graph failed a simple-CSR check */
  KCORE_ERR_CAPACITY = 6    /* an internal bound was exceeded (reported, never overrun) */
} kcore_status;

/* Tunables (kcore_set_option). Defaults are chosen per device at kcore_create
 * and may be overridden; kcore_get_option reads them back. */
typedef enum {
  KCORE_OPT_SYNC_MODE = 0,     /* single-graph peel schedule: 0 auto (= 2); 1 asynchronous
                                  persistent kernel (rounds end on device-wide counters, work
                                  overlaps across subrounds); 2 bulk-synchronous persistent kernel
                                  (a bounded grid barrier after the scan and after every subround);
                                  3 the offline peel of Algorithm 2 on the same kernel: each subround
                                  counts the frontier's decrements per neighbour (histogram), then
                                  applies them in one step per vertex, so every crossing is decided
                                  by one owner; no local queues (its subrounds are Algorithm 1's);
                                  4 the whole graph on one CTA of 1024 threads (CTA barriers only,
                                  induced degrees in shared memory when they fit), or on one
                                  thread-block cluster of KCORE_OPT_BATCH_CLUSTER CTAs (the
                                  hardware cluster barrier): the batched peel's kernel on a batch
                                  of one, for small deep graphs whose many phases cost more in
                                  grid barriers than one SM's work; not for the k'-core query,
                                  which runs mode 2; trace and sampling options do not apply */
  KCORE_OPT_CTAS_PER_SM = 1,   /* CTAs per SM of the persistent kernel (0 = occupancy maximum) */
  KCORE_OPT_SLICE_ARCS = 2,    /* arcs per work item (16 .. 2^20; 0 = auto: 32 in modes 2 and 3,
                                  512 in mode 1): longer lists are split in slices */
  KCORE_OPT_LOCAL_QUEUE = 3,   /* per-warp local queue capacity (work items, 0 .. 128; 0 disables
                                  it; -1 = auto: 128 in mode 2, 32 in mode 1) */
  KCORE_OPT_TIMEOUT_MS = 4,    /* limit for every device-side wait, milliseconds */
  KCORE_OPT_MIN_CTAS = 5,      /* lower bound of the grid for small graphs */
  KCORE_OPT_VERTICES_PER_CTA = 6, /* grid sizing: about one CTA per this many vertices+arcs/8 */
  KCORE_OPT_TEST_STALL = 7,      /* test hook, default 0: 1 makes CTA 0 withhold its round-1
                                    completion token (mode 1) or its arrival at the first grid
                                    barrier (mode 2), so every device wait must run out its
                                    time limit and the call ends with KCORE_ERR_TIMEOUT */
  KCORE_OPT_TRACE = 8,           /* 1 records a per-round timeline (kcore_get_trace); 2 (modes 2
                                    and 3) one record per phase instead; calls with
                                    KCORE_OPT_SAMPLING record none */
  KCORE_OPT_IDLE_SLEEP_NS = 9,   /* nanosleep of a warp waiting for work (0 .. 100000) */
  KCORE_OPT_POLL_SLEEP_NS = 10,  /* nanosleep of a CTA's round-end poller (0 .. 100000) */
  KCORE_OPT_BATCH_BLOCK = 11,    /* batched peel: threads per CTA (256, 512 or 1024; default 1024) */
  KCORE_OPT_BATCH_SMEM_VERTICES = 12, /* batched peel: graphs with at most this many vertices keep
                                         their induced degrees in shared memory (-1 = as many as
                                         fit with the CTAs per SM below) */
  KCORE_OPT_BATCH_CTAS_PER_SM = 13,   /* batched peel: resident CTAs per SM (0 = occupancy limit) */
  KCORE_OPT_LOCAL_BATCHES = 14,       /* mode 2: local-queue batches a warp may run after each chunk it
                                         takes (0 .. 2^20, 0 = no limit; default 32); the rest of its local queue
                                         then goes to the work queue, so a large cascade is shared by
                                         all warps in the next subround instead of one warp */
  KCORE_OPT_LEVEL_WINDOW = 15,        /* mode 2: bucketing of the active list (Sec. 5, the fixed number
                                         of buckets): 0 = off (default); W > 0 = a rebuild scan splits
                                         the live vertices into those below k+W (scanned level by
                                         level) and an overflow list (scanned again only at the next
                                         rebuild); a vertex enters the window when a decrement of its
                                         induced degree returns k+W */
  KCORE_OPT_BATCH_UPDATE = 16         /* mode 2: 1 (default) = a heavy subround (at least a quarter of
                                         an item per warp and one per active vertex) counts its
                                         decrements per neighbour with reductions and then applies
                                         them walking the active list (Algorithm 2's batch update);
                                         0 = every subround decrements with returning atomics */,
  /* Sampling (Sec. 4.1, Algorithms 4 and 5; mode 2, not with LEVEL_WINDOW or
   * the k'-core query): a vertex whose induced degree D exceeds
   * SAMPLE_THRESHOLD and 10 k is put in sample mode; a peeled neighbour then
   * tosses a coin of probability mu / (0.9 D) (Philox4x32-10 of the arc index
   * and SAMPLE_SEED) instead of decrementing it; mu heads, or a failed
   * validation at a level's start, make the vertex recount its untraversed
   * neighbours. A recount that finds the vertex missed an earlier level, or
   * a failed final check (every v has at least core[v] neighbours of
   * coreness >= core[v], SAMPLE_CHECK), makes the call recompute the result
   * without sampling in the same stream (Las Vegas: the result is always
   * exact; kcore_stats.sample_reruns says whether it happened). */
  KCORE_OPT_SAMPLING = 17,            /* 0 (default) off, 1 on */
  KCORE_OPT_SAMPLE_MU = 18,           /* heads per sampling period (1 .. 2^24); 0 = auto:
                                         ceil(4 (c + 2) ln n) with c = 8 (the sampling
                                         theorem of Sec. 4.1) */
  KCORE_OPT_SAMPLE_THRESHOLD = 19,    /* degree above which a vertex may be sampled; -1 = auto (8 mu) */
  KCORE_OPT_SAMPLE_SEED = 20,         /* Philox key of the coins (default 1) */
  KCORE_OPT_SAMPLE_CHECK = 21,        /* 1 (default) runs the final check; 0 relies on the
                                         recount test of Sec. 4.1 alone */
  KCORE_OPT_WARP_COMBINE = 22,        /* mode 2: 1 = the lanes of a warp that decrement the same
                                         vertex in one step send one atomic of their count (warp
                                         aggregation, the GPU alternative to sampling for hub
                                         contention); 0 (default) = one atomic per arc */
  KCORE_OPT_PRECHECK_ITEMS = 23,      /* mode 2: a subround whose queue range gives every warp at
                                         least this many items reads d~ before decrementing (sparing
                                         atomics on neighbours already peeled); shorter subrounds
                                         decrement unconditionally (sparing a dependent read).
                                         Default 64; 0 = always read first */
  /* Tail mode (mode 2, not with LEVEL_WINDOW, not the k'-core query): the
   * many short phases of a long peel (Algorithm 1's subrounds of a few
   * vertices, scans of a short active list; Sec. 3.2 counts each as a
   * synchronisation of the burdened span) run on one CTA, closed by a CTA
   * barrier instead of the grid barrier. The other CTAs park on a bounded
   * wait (KCORE_OPT_TIMEOUT_MS, KCORE_ERR_TIMEOUT) until CTA 0 meets a
   * larger phase and hands them the loop state. */
  KCORE_OPT_TAIL_ITEMS = 24,          /* a subround pass of at most this many work items runs on one
                                         CTA (0 .. 2^30; 0 = never) */
  KCORE_OPT_TAIL_ENTRIES = 25,        /* a scan of at most this many active-list entries runs on one
                                         CTA (0 .. 2^31 - 2; 0 = never) */
  KCORE_OPT_PARK_SLEEP_NS = 26,       /* nanosleep of a parked CTA between polls (0 .. 100000) */
  KCORE_OPT_SCAN_ENTRIES = 27,        /* modes 1 and 2: a scan gives each CTA at least this many active-list
                                         entries (256 .. 2^20; default 512), so short lists are
                                         scanned by fewer CTAs */
  KCORE_OPT_BATCH_CLUSTER = 28,       /* batched peel: 0 (default) = one CTA per graph; 2, 4 or 8 = a
                                         graph with at least KCORE_OPT_BATCH_BIG_ARCS arcs is peeled
                                         by a thread-block cluster of that many CTAs (512 or 1024
                                         threads per CTA), so a batch's largest graphs no longer
                                         hold it up; smaller graphs still take one CTA each. Sync
                                         mode 4 of a single graph: the cluster size (0 = one CTA) */
  KCORE_OPT_BATCH_BIG_ARCS = 29       /* batched peel with clusters: the arcs from which a graph takes a
                                         cluster (0 = the batch's arcs divided by its CTAs, default;
                                         else 1 .. 2^40) */
} kcore_option;

/* Counters of the last decomposition, or of the last CSR check (the three
 * invalid_* fields), valid after kcore_sync_status. */
typedef struct {
  int64_t rounds;          /* levels visited, empty speculative levels included */
  int64_t empty_rounds;    /* visited levels that held no vertex */
  int64_t items;           /* work items (vertex slices) processed through the global queue */
  int64_t local_items;     /* work items (slices) processed from warp-local queues */
  int64_t scanned;         /* sum over rounds of the active-set size scanned (Theorem 1) */
  int64_t kmax;            /* largest coreness */
  int64_t grid;            /* CTAs of the persistent kernel */
  int64_t sync_mode;       /* mode actually used: 1 asynchronous, 2 bulk-synchronous, 3 offline */
  int64_t passes;          /* modes 2 and 3: subround passes over the work queue */
  int64_t barriers;        /* bulk-synchronous mode: grid barriers taken */
  int64_t batch_block;     /* batched calls: threads per CTA used */
  int64_t batch_smem_vertices; /* batched calls: largest graph kept in shared memory */
  int64_t slice_arcs;      /* arcs per work item the last decomposition used */
  int64_t sample_vertices;  /* sampling: vertices put in sample mode by the first InitSampler */
  int64_t sample_recounts;  /* sampling: SetSampler recounts */
  int64_t sample_bag;       /* sampling: counting-bag insertions (mu heads reached) */
  int64_t sample_failed_validations; /* sampling: Error(v, k) failures at level starts */
  int64_t sample_heads;     /* sampling: coin heads */
  int64_t sample_reruns;    /* sampling: 1 if the sampled result was recomputed without sampling */
  int64_t sample_miss_round; /* sampling: level of a miss found by a recount, else -1 */
  int64_t invalid_check;   /* kcore_validate_csr: first failed check (1..6), 0 if the CSR is simple */
  int64_t invalid_vertex;  /* kcore_validate_csr: the vertex of that failure */
  int64_t invalid_arc;     /* kcore_validate_csr: the failing arc (index into adj); for codes 1
                              and 2 the offending offset value instead */
  int64_t tail_phases;     /* mode 2: phases run by one CTA in tail mode (not counted in barriers) */
  int64_t tail_episodes;   /* mode 2: times the grid parked while one CTA ran tail phases */
  int64_t batch_cluster;   /* batched calls: CTAs per cluster for the large graphs (0: none) */
} kcore_stats;

/* Creates a handle on `device` (CUDA ordinal). The handle owns a workspace
 * that grows on demand, a small pinned status buffer and its tuning values.
 * Errors: KCORE_ERR_INVALID (null out / bad device), KCORE_ERR_CUDA. */
kcore_status kcore_create(kcore_handle* out, int device);

/* Frees everything the handle owns. Waits for the handle's queued work. */
kcore_status kcore_destroy(kcore_handle h);

/* Human-readable description of the last error on this handle ("" if none).
 * The string is owned by the handle and valid until its next call. */
const char* kcore_last_error(kcore_handle h);

kcore_status kcore_set_option(kcore_handle h, kcore_option opt, int64_t value);
kcore_status kcore_get_option(kcore_handle h, kcore_option opt, int64_t* value);

/* Device bytes of workspace kcore_decompose needs for a graph of n vertices
 * and m arcs (host call, no device work). */
kcore_status kcore_workspace_size(kcore_handle h, int64_t n, int64_t m, size_t* bytes);

/* Hands the handle caller-owned device memory to use as workspace (e.g. from
 * a caching allocator). The caller keeps it alive until the handle's work has
 * finished or another workspace is set; ptr = NULL returns to handle-owned
 * memory. ptr must be 256-byte aligned. */
kcore_status kcore_set_workspace(kcore_handle h, void* ptr, size_t bytes);

/* Coreness of every vertex (Algorithm 1 with online peeling, Algorithm 3).
 *   n, m           vertices, arcs (m = offsets[n] = twice the undirected edges)
 *   offsets        device int64[n+1], borrowed
 *   adj            device int32[m], borrowed; simple undirected CSR
 *   coreness_out   device int32[n]: coreness of each vertex
 *   kmax_out       device int32[1]: largest coreness (0 when n == 0)
 *   stream         CUDA stream the work is queued on
 * Asynchronous. Uses the handle's workspace (grown with cudaMalloc if the
 * caller set none; growing synchronises the device). Errors: INVALID, OOM,
 * CUDA synchronously; TIMEOUT via kcore_sync_status. */
kcore_status kcore_decompose(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets,
                             const int32_t* adj, int32_t* coreness_out, int32_t* kmax_out,
                             kcore_stream_t stream);

/* Same computation from HOST arrays, end to end: copies offsets and adj to the
 * device, decomposes, copies coreness and k_max back, and waits. Host buffers
 * may be pageable or pinned (pinned is faster). Synchronous; returns the
 * device status as kcore_sync_status would. */
kcore_status kcore_decompose_host(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets_host,
                                  const int32_t* adj_host, int32_t* coreness_host,
                                  int32_t* kmax_host, kcore_stream_t stream);

/* Checks that a CSR is the simple undirected graph every decomposition entry
 * point requires (Sec. 2: undirected, no self-loops, no parallel edges) and
 * that kcore_build_csr produces. Optional: the decompositions assume it and do
 * not check it (a malformed graph gives undefined coreness, never an access
 * outside the arrays described by offsets). Checks, in this order of codes:
 *   1  offsets monotone and within [0, m]      2  offsets[0] = 0, offsets[n] = m
 *   3  every neighbour id in [0, n)            4  no self-loop
 *   5  each list strictly ascending (no repeated arc)
 *   6  symmetry: u in list(v) implies v in list(u) (binary search in list(u))
 *   n, m         vertices and arcs (0 <= n <= 2^31 - 2; m = 0 when n = 0)
 *   offsets, adj device int64[n+1], int32[m], borrowed, read only
 * Asynchronous: two kernels on `stream`, O(m log d_max) work. kcore_sync_status
 * returns KCORE_OK for a simple CSR, else KCORE_ERR_NOT_SIMPLE with the first
 * failure recorded (which one, when several threads fail at once, is
 * unspecified) in kcore_stats.invalid_check / invalid_vertex / invalid_arc and
 * in kcore_last_error. Uses 64 bytes of the handle's workspace. */
kcore_status kcore_validate_csr(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets,
                                const int32_t* adj, kcore_stream_t stream);

/* Simple undirected CSR of an edge list (a1 of the pipeline; the paper
 * symmetrises directed inputs, Sec. 6.1 "Datasets"): every pair (src[i],
 * dst[i]) with src[i] != dst[i] contributes the arcs src->dst and dst->src;
 * self-loops are dropped and repeated arcs kept once; each adjacency list is
 * ascending.
 *   n               vertices (ids in [0, n)); 0 <= n <= 2^31 - 2
 *   num_edges       pairs in src/dst (may contain duplicates, both directions,
 *                   self-loops)
 *   src, dst        device int32[num_edges], borrowed
 *   offsets_out     device int64[n+1]
 *   adj_out         device int32 with room for 2 * num_edges entries (the
 *                   worst case); the first m are written
 *   m_out           device int64[1]: m, the number of arcs written
 * Asynchronous; uses the handle's workspace (kcore_build_csr_workspace_size
 * bytes: two key buffers of 2 * num_edges uint64 plus histograms). A vertex id
 * outside [0, n) is reported as KCORE_ERR_INVALID by kcore_sync_status. */
kcore_status kcore_build_csr(kcore_handle h, int64_t n, int64_t num_edges, const int32_t* src,
                             const int32_t* dst, int64_t* offsets_out, int32_t* adj_out,
                             int64_t* m_out, kcore_stream_t stream);

/* Workspace bytes kcore_build_csr needs (host call). */
kcore_status kcore_build_csr_workspace_size(kcore_handle h, int64_t n, int64_t num_edges, size_t* bytes);

/* Coreness of many independent graphs in one launch (the batched form of the
 * same peel; the paper peels one graph at a time). The graphs form a
 * segmented CSR: graph g owns global vertices [graph_vertex_offsets[g],
 * graph_vertex_offsets[g+1]), offsets[] is one global int64 offsets array over
 * all N vertices (offsets[N] = total_arcs), and each adjacency list holds
 * GRAPH-LOCAL ids (0 .. n_g - 1). Each graph must be a simple undirected graph.
 *   num_graphs            G (0 <= G <= 2^24)
 *   total_vertices        N = graph_vertex_offsets[G]
 *   total_arcs            offsets[N]
 *   graph_vertex_offsets  device int64[G+1], starts at 0, non-decreasing
 *   offsets, adj          device int64[N+1], int32[total_arcs]
 *   coreness_out          device int32[N]: coreness of every vertex in its graph
 *   kmax_out              device int32[G]: largest coreness of each graph (0 if empty)
 * Asynchronous; one persistent kernel (each graph peeled by one CTA, induced
 * degrees in shared memory when the graph fits, largest graphs first; with
 * KCORE_OPT_BATCH_CLUSTER, the graphs above KCORE_OPT_BATCH_BIG_ARCS arcs by a
 * thread-block cluster each, induced degrees in L2). Uses
 * kcore_batched_workspace_size bytes of workspace (20 bytes per vertex).
 * Malformed offsets or ids are reported as KCORE_ERR_NOT_SIMPLE by
 * kcore_sync_status. */
kcore_status kcore_decompose_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                     int64_t total_arcs, const int64_t* graph_vertex_offsets,
                                     const int64_t* offsets, const int32_t* adj, int32_t* coreness_out,
                                     int32_t* kmax_out, kcore_stream_t stream);

/* Segmented CSR of a batch of edge lists (the batched form of
 * kcore_build_csr): graph g owns vertices [graph_vertex_offsets[g],
 * graph_vertex_offsets[g+1]) and edges [graph_edge_offsets[g],
 * graph_edge_offsets[g+1]) of src/dst, whose ids are GRAPH-LOCAL. The output is
 * the input of kcore_decompose_batched: one global offsets array over all
 * vertices and graph-local adjacency ids, each graph symmetrised, without
 * self-loops or repeated arcs, each list ascending.
 *   num_graphs >= 1; total_vertices = graph_vertex_offsets[G] <= 2^31 - 2
 *   max_graph_vertices    the largest n_g (host value; sizes the sort keys)
 *   graph_vertex_offsets, graph_edge_offsets   device int64[G+1]
 *   src, dst              device int32[num_edges], local ids
 *   offsets_out           device int64[total_vertices + 1]
 *   adj_out               device int32 with room for 2 * num_edges
 *   m_out                 device int64[1]: arcs written
 * Asynchronous; a local id outside its graph is reported as KCORE_ERR_INVALID
 * by kcore_sync_status. Workspace as kcore_build_csr. */
kcore_status kcore_build_csr_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                     int64_t num_edges, int64_t max_graph_vertices,
                                     const int64_t* graph_vertex_offsets, const int64_t* graph_edge_offsets,
                                     const int32_t* src, const int32_t* dst, int64_t* offsets_out,
                                     int32_t* adj_out, int64_t* m_out, kcore_stream_t stream);

/* Workspace bytes kcore_decompose_batched needs (host call). */
kcore_status kcore_batched_workspace_size(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                          size_t* bytes);

/* Result of kcore_autotune_batched. */
typedef struct {
  int32_t block;         /* threads per CTA chosen (KCORE_OPT_BATCH_BLOCK) */
  int32_t ctas_per_sm;   /* resident CTAs per SM chosen (KCORE_OPT_BATCH_CTAS_PER_SM) */
  int32_t smem_vertices; /* largest graph kept in shared memory under that shape */
  int32_t candidates;    /* launch shapes timed */
  double ms;             /* best time of one batched call with the chosen shape */
  int32_t cluster;       /* CTAs per cluster for the large graphs chosen (KCORE_OPT_BATCH_CLUSTER) */
} kcore_batch_tuning;

/* Autotuner of the batched peel (not in the paper: the launch shape of the
 * batched form). Times each candidate launch shape -- 1024, 512 or 256
 * threads per CTA with 1..8 resident CTAs per SM, the shared-memory threshold
 * following the shape, 512 threads x 3 CTAs with thresholds of 8,000 and
 * 2,000 vertices, and the clustered form with clusters of 2, 4 or 8 CTAs
 * of 1024 threads or 4 of 512 -- on the caller's own batch (the arguments of
 * kcore_decompose_batched), best of `repeats` (1..100) calls after one
 * warm-up each, with CUDA events on `stream`. It then sets the handle's batch
 * options (KCORE_OPT_BATCH_BIG_ARCS back to 0) to the fastest shape, runs the
 * batch once more with it and fills *best_out. Synchronous; the outputs hold that last, exact result.
 * Errors: KCORE_ERR_INVALID (bad arguments; options unchanged), the first
 * input or memory error any call reports (KCORE_ERR_NOT_SIMPLE, _OOM;
 * options restored), KCORE_ERR_CUDA if no shape could run. */
kcore_status kcore_autotune_batched(kcore_handle h, int64_t num_graphs, int64_t total_vertices,
                                    int64_t total_arcs, const int64_t* graph_vertex_offsets,
                                    const int64_t* offsets, const int32_t* adj, int32_t* coreness_out,
                                    int32_t* kmax_out, int32_t repeats, kcore_batch_tuning* best_out,
                                    kcore_stream_t stream);

/* Result of kcore_autotune: the option values chosen (see kcore_option). */
typedef struct {
  int32_t sync_mode;      /* KCORE_OPT_SYNC_MODE */
  int32_t batch_update;   /* KCORE_OPT_BATCH_UPDATE */
  int32_t warp_combine;   /* KCORE_OPT_WARP_COMBINE */
  int32_t ctas_per_sm;    /* KCORE_OPT_CTAS_PER_SM (0 = occupancy maximum) */
  int64_t tail_items;     /* KCORE_OPT_TAIL_ITEMS */
  int64_t tail_entries;   /* KCORE_OPT_TAIL_ENTRIES */
  int64_t precheck_items; /* KCORE_OPT_PRECHECK_ITEMS */
  int64_t local_batches;  /* KCORE_OPT_LOCAL_BATCHES */
  int32_t candidates;     /* schedules timed */
  double ms;              /* best time of one decomposition with the chosen schedule */
  int32_t cluster;        /* KCORE_OPT_BATCH_CLUSTER (used by sync mode 4) */
} kcore_tuning;

/* Autotuner of the single-graph peel's schedule (Algorithm 1's subround and
 * round scheduling, Sec. 3.2: how the many synchronisations of a long peel
 * are paid). Times each candidate schedule -- the bulk-synchronous default;
 * tail mode at a few thresholds, including the whole peel on one CTA; no
 * batch update; d~ read first in shorter subrounds; shorter local chains;
 * warp aggregation; one CTA per SM; the asynchronous schedule; mode 4 on one
 * CTA and on a cluster of 8 -- on the caller's own graph (the arguments of kcore_decompose), best of `repeats`
 * (1..100) calls after one warm-up each, with CUDA events on `stream`. It then
 * sets the handle's options to the fastest schedule, decomposes once more
 * with it and fills *best_out. Tracing is off while it times. Synchronous; the
 * outputs hold that last, exact result. Errors: KCORE_ERR_INVALID (bad
 * arguments, n < 1; options unchanged), the first input or memory error a call
 * reports (KCORE_ERR_NOT_SIMPLE, _OOM; options restored), KCORE_ERR_CUDA if no
 * schedule could run. */
kcore_status kcore_autotune(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                            int32_t* coreness_out, int32_t* kmax_out, int32_t repeats, kcore_tuning* best_out,
                            kcore_stream_t stream);

/* ------------------------------------------------------------------------
 * Served peel (the paper peels one graph at a time; this is the request-loop
 * form of the same peel). A server owns a device memory pool reserved at
 * creation and admits a request only when its footprint (offsets, arcs,
 * coreness and the peel state kept resident while it is in flight) fits and a
 * slot is free. kcore_server_poll moves requests through copy-in, launch,
 * copy-out without blocking on the device: the small requests that became
 * ready together run as one batched launch (one CTA per graph, or a cluster
 * of CTAs for each of its largest graphs, listed first) on one of
 * several streams, so requests admitted while others are on the GPU overlap
 * with them; large requests run the whole-GPU peel on their own stream.
 * One host thread drives a server (not thread-safe). */
typedef struct kcore_server_ctx* kcore_server;

typedef struct {
  size_t pool_bytes;      /* device pool for requests in flight (0: a quarter of free memory) */
  int max_requests;       /* requests in flight at most (0: 4096) */
  int streams;            /* launch streams for batched launches (0: 4, at most 32) */
  int64_t large_vertices; /* requests with more vertices use the whole-GPU peel (0: 2^20) */
  int64_t large_arcs;     /* ... or more arcs (0: 2^25) */
  int batch_cluster;      /* batched launches: the graphs with at least batch_big_arcs arcs are peeled
                             by a thread-block cluster of this many CTAs (2, 4 or 8), the others by
                             one CTA each; 1 = one CTA per graph; 0 = the default (4) */
  int64_t batch_big_arcs; /* batched launches with clusters: the arcs from which a graph takes a
                             cluster (0: the launch's arcs divided by its CTAs) */
} kcore_server_config;

/* cfg may be NULL (defaults). Errors: INVALID, OOM (pool or pinned buffers). */
kcore_status kcore_server_create(kcore_server* out, int device, const kcore_server_config* cfg);

/* Queues one graph (simple undirected CSR in HOST memory, layout as for
 * kcore_decompose) and returns its ticket. Non-blocking: offsets_host,
 * adj_host and coreness_host must stay valid until the ticket is returned by
 * kcore_server_poll (pinned host memory makes the copies asynchronous).
 * KCORE_ERR_CAPACITY: not admitted now (pool or slots full); poll and retry. */
kcore_status kcore_server_submit(kcore_server s, int64_t n, int64_t m, const int64_t* offsets_host,
                                 const int32_t* adj_host, int32_t* coreness_host, int64_t* ticket_out);

/* Advances all requests and returns up to max_out completed ones: their
 * tickets, k_max and device status (0 = OK, else a kcore_status value); their
 * coreness is in the coreness_host buffer given at submit. *n_out = count. */
kcore_status kcore_server_poll(kcore_server s, int64_t* tickets_out, int32_t* kmax_out, int32_t* status_out,
                               int max_out, int* n_out);

/* Requests in flight and pool bytes in use / reserved (any pointer may be NULL). */
kcore_status kcore_server_info(kcore_server s, int64_t* in_flight, int64_t* pool_used, int64_t* pool_bytes);

/* Waits for the device and frees everything; results not yet polled are dropped. */
kcore_status kcore_server_destroy(kcore_server s);

/* Largest graph kcore_decompose_static accepts. */
#define KCORE_STATIC_MAX_VERTICES (1LL << 20)
#define KCORE_STATIC_MAX_ARCS (1LL << 24)

/* kcore_decompose for callers that cannot allocate device memory. The paper has
 * no counterpart: this is a deployment variant of the same peel.
 *
 * Some callers cannot call cudaMalloc: another allocator may own all of their
 * device memory, their policy may forbid allocation after start-up, or they
 * cannot accept the device-wide synchronisation an allocation can cause. This
 * call allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine) and needs no handle: its scratch memory is one fixed array in the
 * library's device memory (under 32 MB). It runs the peel with the settings of
 * a handle's defaults. The caller still passes the graph and the output arrays,
 * exactly as for kcore_decompose (same layout and meaning):
 *   n <= KCORE_STATIC_MAX_VERTICES, m <= KCORE_STATIC_MAX_ARCS; larger graphs
 *   are rejected with KCORE_ERR_CAPACITY before any work is queued.
 * It runs on the calling thread's current device and is synchronous: it waits
 * for `stream` before returning the device status (KCORE_OK,
 * KCORE_ERR_TIMEOUT, ...).
 * The first call on a device does a one-time set-up: it looks up the array's
 * device address, and under CUDA's default lazy module loading that lookup is
 * what creates the array on the device (one allocation by the CUDA runtime,
 * kept until the process exits). So make the first call on each device at
 * start-up, before another allocator reserves the device memory, or run with
 * CUDA_MODULE_LOADING=EAGER (the array then exists from the moment the
 * library's code is loaded); make that first call before any stream capture.
 * Later calls change nothing in the device's memory use.
 * Every call uses the same array and leaves its contents behind (each call
 * clears what must start from zero); calls that overlap on the GPU, from two
 * threads or two streams, race on it and must not be made. */
kcore_status kcore_decompose_static(int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                                    int32_t* coreness_out, int32_t* kmax_out, kcore_stream_t stream);

/* The maximum k'-core query (App. B, "Maximum k-Core Subgraph": the peeling
 * framework with a single threshold instead of increasing levels). mask_out[v]
 * receives 1 when v lies in the k'-core -- the largest subgraph in which every
 * vertex has degree >= kprime, i.e. the vertices of coreness >= kprime -- and
 * 0 otherwise; *size_out (device int64, may be NULL) receives the k'-core's
 * vertex count. One peel at level kprime - 1 on the bulk-synchronous kernel:
 * a scan takes every vertex whose degree is below kprime, and subround passes
 * remove the vertices whose decrement lands them below kprime. kprime <= 0
 * keeps every vertex. Input layout, workspace and errors as kcore_decompose
 * (asynchronous on `stream`; kcore_sync_status reports device errors). */
kcore_status kcore_core_mask(kcore_handle h, int64_t n, int64_t m, const int64_t* offsets, const int32_t* adj,
                             int32_t kprime, int32_t* mask_out, int64_t* size_out, kcore_stream_t stream);

/* Waits for the stream of the handle's last call and returns the status the
 * device recorded (KCORE_OK, KCORE_ERR_TIMEOUT, ...). */
kcore_status kcore_sync_status(kcore_handle h);

/* Latency of the bulk-synchronous schedule's grid barrier (the synchronisation
 * each phase of Algorithm 1's rounds and subrounds ends with; the burdened
 * span of Sec. 3.2 charges one per subround): `iters` (1 .. 10^6) barriers of
 * `grid` co-resident CTAs (0 = the grid kcore_decompose uses for a large
 * graph) run back to back with no work between them; *ns_out receives the
 * mean time of one, in nanoseconds. Waits for the handle's last call and for
 * the device; uses the handle's workspace. Errors: INVALID (bad arguments, a
 * grid above the co-resident maximum), OOM, CUDA, TIMEOUT. */
kcore_status kcore_barrier_latency(kcore_handle h, int64_t grid, int32_t iters, double* ns_out);

/* Counters of the last decomposition; call after kcore_sync_status. */
kcore_status kcore_get_stats(kcore_handle h, kcore_stats* out);

/* Per-round timeline of the last decomposition when KCORE_OPT_TRACE was 1
 * (call after kcore_sync_status). out receives 14 uint64 per round:
 * [0] device time (ns) the round started, [1] when its scan finished,
 * [2] when the round finished, [3] its level k, [4] active-list entries
 * scanned, [5] frontier vertices found by the scan, [6] work items queued,
 * [7] CTAs that scanned, [8] arcs read, [9] decrements issued, [10] longest
 * scan of one CTA (ns), [11] latest round start of a CTA after CTA 0 (ns),
 * [12] summed time warps spent in work batches (ns), [13] work batches.
 * In mode 2 there is one entry per non-empty level: [1] is when its scan
 * phases ended, [10..12] are 0 and [13] counts its subround passes.
 * With KCORE_OPT_TRACE = 2 (modes 2 and 3) there is one entry per phase
 * (grid barrier or tail phase) instead: [0] device time (ns) the phase
 * ended, [1] its kind (0 scan, 1 subround pass, 2 counting phase, 3 apply
 * phase, 4 second scan of an empty level), [2] the level, [3] the range it
 * worked on (list entries of a scan, queue items of a pass), [4] items it
 * appended, [5] frontier vertices a scan found, [6] arcs a pass read, [7] 1
 * if one CTA ran it (tail mode); [8..13] are 0.
 * Tracing adds atomics and slows the run. At most max_rounds rounds are
 * copied; *rounds_out receives the number copied. */
kcore_status kcore_get_trace(kcore_handle h, uint64_t* out, int64_t max_rounds, int64_t* rounds_out);

#ifdef __cplusplus
}
#endif

#endif /* KCORE_H_ */
