/*
 * coremaint.h -- C ABI of the GB300 (sm_103a) core-maintenance library.
 *
 * Method: batched incremental and decremental k-core maintenance by
 * superior edge sets (N. Wang, D. Yu, H. Jin, C. Qian, X. Xie, Q.-S. Hua,
 * "Parallel Algorithms for Core Maintenance in Dynamic Graphs",
 * arXiv 1612.09368).  Core number: Section III, Definitions 1-2.  Superior
 * edge / k-superior edge set / superior edge set: Section IV, Definition 6
 * and the paragraph after it.  Incremental problem: Section III, Definition
 * 4 and Section V (Algorithms 1-4).  Decremental problem: Definition 5 and
 * Section VI (Algorithms 5-7).  Vertex insertion and deletion reduced to
 * edge operations: Section I.
 *
 * General conventions
 *  - Graphs are undirected and simple.  Vertex ids are dense int32 in
 *    [0, n_total); new vertices get appended ids that are never reused.
 *  - An edge list is an int32 array of 2*k entries (u0, v0, u1, v1, ...).
 *    The order inside a pair does not matter; repeats collapse to one
 *    (the first occurrence); self-loops are dropped; inserting an edge that
 *    is present, or deleting one that is absent, is skipped and not an
 *    error.  n_applied (nullable) reports how many edges were applied.
 *  - Every pointer argument named "host or device" may be either: the
 *    library detects device memory (cudaPointerGetAttributes) and copies
 *    host memory in.  The caller owns its buffers; the library reads them
 *    before the call returns and keeps no reference.  The library owns all
 *    graph state in device memory.
 *  - Calls run on the handle's CUDA stream and return after the work has
 *    completed (synchronous semantics).  One handle must not be used from
 *    two threads at once; distinct handles are independent.
 *  - Return value: CM_OK (0) or a negative CM_ERR_* code.  Validation
 *    happens before any mutation, so CM_ERR_INVALID and CM_ERR_OOM leave
 *    the graph unchanged.  CM_ERR_CUDA and CM_ERR_LIMIT (a device wait or
 *    iteration limit ran out) poison the handle: every later call except
 *    cm_destroy / cm_last_error returns CM_ERR_STATE.
 *  - cm_last_error() describes the most recent failure of a handle.
 */
#ifndef COREMAINT_H
#define COREMAINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CM_OK 0
#define CM_ERR_INVALID (-1)   /* bad argument: id out of range, dead vertex, NULL, negative size */
#define CM_ERR_OOM (-2)       /* device or host allocation failed; graph unchanged */
#define CM_ERR_CAPACITY (-3)  /* a size exceeds a documented maximum; graph unchanged */
#define CM_ERR_LIMIT (-4)     /* a bounded device wait or iteration cap ran out; handle poisoned */
#define CM_ERR_CUDA (-5)      /* a CUDA runtime call failed; handle poisoned */
#define CM_ERR_STATE (-6)     /* handle poisoned by an earlier failure, or cores stale */

#define CM_OP_INSERT 0
#define CM_OP_DELETE 1

typedef struct cm_graph cm_graph;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes usable on `stream`,
 * or NULL; free releases it.  When both are NULL the library uses
 * cudaMalloc / cudaFree. */
typedef void* (*cm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cm_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct cm_options {
    int32_t slack_pct;      /* per-vertex adjacency headroom in percent (default 25) */
    int32_t min_cap;        /* minimum adjacency slots per vertex, rounded up to 4 (default 4) */
    int32_t block_threads;  /* unused (kept for layout): every persistent kernel runs 512-thread blocks */
    int32_t blocks_per_sm;  /* resident blocks per SM of the persistent kernels; 0 = occupancy limit */
    int32_t max_sms;        /* SMs the persistent kernels may fill; 0 = all (lower it to share the GPU) */
    int32_t block_mode_edges; /* single-block mode only while at most this many edges remain (16384;
                                 negative = never leave grid mode) */
    int64_t spin_limit_ns;  /* limit of every grid-barrier wait (default 4e9 ns); CM_ERR_LIMIT past it */
    cm_alloc_fn alloc;      /* optional allocator, see above */
    cm_free_fn free;
    void* alloc_ctx;
    int32_t debug_flags;    /* test hooks, 0 in production (CM_DEBUG_*) */
    int32_t block_mode_enter; /* grid -> single block after an iteration touching <= this many items (1024) */
    int32_t block_mode_leave; /* single block -> grid after an iteration touching more (8192) */
    int32_t hub_slots;      /* grid mode: a vertex with at least this many adjacency slots is scanned by
                               all warps in chunks of 512 (1024; negative = never) */
    int32_t block_slots;    /* grid mode, insert: a vertex with at least this many slots (below hub_slots)
                               is scanned by a whole block instead of one warp (4096) */
    int32_t block_slots_delete; /* the same for delete calls (1024) */
    int32_t task_claim;     /* grid mode: most search tasks a warp claims at once (1..8, default 1) */
    int32_t select_order;   /* order of the greedy superior-edge-set selection (Section IV,
                               Definition 6 and Algorithm 2): CM_SELECT_HASH (default) ranks an edge
                               by fmix64 of its canonical key (lo << 32 | hi), a fixed pseudo-random
                               order; CM_SELECT_KEY by the canonical key itself (lexicographic) */
    int32_t select_rounds;  /* claim rounds per iteration: 0 (default) = until the selected set is
                               maximal; R > 0 = at most R rounds (still a superior edge set, perhaps
                               not a maximal one: fewer barriers per iteration, perhaps more
                               iterations).  Final cores do not depend on either choice. */
    int32_t expand_early;   /* insert search (Algorithm 3): 0 (default) or 1 = a frontier vertex visits
                               its candidates in the same pass that sums its CSD, before its support
                               is known; -1 = the paper's order (sum first, expand only if the
                               support exceeds k).  Visiting early can only add vertices to the
                               search; the cores do not change. */
    int32_t reserved[2];
} cm_options;

#define CM_SELECT_HASH 0
#define CM_SELECT_KEY 1

/* Test hook: every grid barrier of the next maintenance launch waits for
 * one more block than exists, so each wait runs out after spin_limit_ns and
 * the call returns CM_ERR_LIMIT (no fault, no hang). */
#define CM_DEBUG_BARRIER_NEVER_RELEASES 1
/* Test hook: the next maintenance call may run one superior-edge-set
 * iteration only; a batch that needs more stops with CM_ERR_LIMIT. */
#define CM_DEBUG_ITER_CAP 2
/* Test hook: the next maintenance call runs grid-wide and its search counts
 * one task that is never queued, so the search never becomes quiescent:
 * every warp's wait on the task queue runs out after spin_limit_ns and the
 * call returns CM_ERR_LIMIT (no fault, no hang). */
#define CM_DEBUG_TASK_WAIT_NEVER_ENDS 4
/* Debug mode, in effect while set (not cleared by a call): every update
 * call of a single graph (edges and vertices, insert and delete) ends each
 * maintenance launch after one superior-edge-set iteration and its SD
 * fix-up, and runs cm_check on the store before the next; the first
 * inconsistency fails the call with CM_ERR_LIMIT (handle poisoned).  The
 * selected sets, iterations and cores are those of the normal mode.  Slow:
 * for tests. */
#define CM_DEBUG_CHECK_ITERATIONS 8

/* Counters of the most recent update call (or of cm_recompute_cores). */
typedef struct cm_stats {
    int64_t applied;         /* edges applied by the call */
    int64_t iterations;      /* superior-edge-set iterations (Algorithm 1 / 5 while-loop) */
    int64_t select_rounds;   /* claim rounds summed over iterations */
    int64_t selected;        /* edges selected, summed over iterations (= applied) */
    int64_t remaining_sum;   /* remaining edges at iteration start, summed */
    int64_t visited;         /* vertices entered into the candidate set (insert) */
    int64_t visited_slots;   /* adjacency slots of those vertices */
    int64_t evicted;         /* vertices evicted by support waves */
    int64_t evicted_slots;
    int64_t changed;         /* vertices whose core moved by one */
    int64_t changed_slots;
    int64_t waves;           /* discovery + eviction waves */
    int64_t alg_bytes;       /* algorithmic HBM bytes of the maintenance kernel; for cm_recompute_cores,
                                of the peel and the SD pass (see design notes) */
    int64_t launches;        /* kernels this library launched during the call */
    double maintain_ms;      /* device time of the maintenance kernel (CUDA events on the handle's stream) */
    double call_ms;          /* device time of the whole call, first copy to last kernel */
    int64_t peel_levels;     /* cm_recompute_cores / cm_create: peeling levels */
    int64_t barriers;        /* barriers executed by the maintenance launches */
    int64_t grid_iterations; /* iterations run grid-wide (the rest ran in one block) */
    int64_t phase_ns[7];     /* device time per phase: claim, check, apply, discover, evict, commit, fix-up;
                                for cm_recompute_cores / cm_create: level scans, sub-waves, chunk phases
                                of the peel (the rest zero) */
    int64_t reserved[4];
} cm_stats;

/* Fills *opt with the defaults. */
void cm_default_options(cm_options* opt);

/* Creates a graph with n vertices (ids 0..n-1) from m undirected edges
 * (host or device, 2*m int32).  cores (host or device, n int32, nullable):
 * the exact core numbers of this graph, the input of Algorithms 1 and 5;
 * when NULL they are computed on the GPU by bucket peeling (the static
 * decomposition the paper cites as [O(m)]).  Passing wrong cores gives
 * wrong maintenance results; they are not verified.  stream: a
 * cudaStream_t (NULL = legacy default stream) on which every later call of
 * this handle runs.  Repeated edges and self-loops in the list are dropped.
 * Errors: CM_ERR_INVALID (out, n < 0, m < 0, id out of range), CM_ERR_OOM,
 * CM_ERR_CUDA. */
int cm_create(cm_graph** out, int32_t n, const int32_t* edges, int64_t m, const int32_t* cores,
              const cm_options* opt, void* stream);

/* Frees the handle and all its device memory.  NULL is ignored. */
void cm_destroy(cm_graph* g);

/* Incremental core maintenance (Algorithm 1): inserts the k edges
 * (host or device, 2*k int32) and updates every core number.  Each
 * iteration selects a maximal superior edge set from the remaining edges
 * (Algorithm 2 with a fixed priority), inserts it, finds per core level the
 * vertices whose core rises (Algorithms 3-4) and raises them by one.
 * Errors: CM_ERR_INVALID (an id out of range or dead; nothing applied). */
int cm_insert_edges(cm_graph* g, const int32_t* edges, int64_t k, int64_t* n_applied);

/* Decremental core maintenance (Algorithm 5, with Algorithms 6-7): deletes
 * the k edges and updates every core number.  Errors as cm_insert_edges. */
int cm_delete_edges(cm_graph* g, const int32_t* edges, int64_t k, int64_t* n_applied);

/* Vertex insertion (Section I): appends `count` vertices with ids
 * n_total .. n_total+count-1 and core 0, then inserts their edges as one
 * batch.  Vertex i's neighbours are nbrs[nbr_off[i] .. nbr_off[i+1]);
 * nbr_off (count+1 int64) and nbrs may be host or device.  A neighbour may
 * be a live existing vertex or another vertex of this call, but not the
 * vertex itself.  *first_id (nullable) receives n_total before the call.
 * Errors: CM_ERR_INVALID (bad neighbour, self-loop), CM_ERR_OOM. */
int cm_insert_vertices(cm_graph* g, int32_t count, const int64_t* nbr_off, const int32_t* nbrs,
                       int32_t* first_id, int64_t* n_applied);

/* One vertex with d neighbours; *new_id receives its id. */
int cm_insert_vertex(cm_graph* g, const int32_t* nbrs, int32_t d, int32_t* new_id);

/* Vertex deletion (Section I): deletes every edge incident to the given
 * live vertices (host or device, count int32; repeats allowed) as one
 * batch, then marks them dead: they keep their ids, report core -1 and
 * reject later edges.  While their edges go, the deleted vertices are
 * pinned (their cores stay fixed, so they constrain no edge and never
 * drop): Definition 6 then only limits the other endpoints, and a deleted
 * hub loses all its edges in one iteration instead of one per iteration.
 * The other vertices end with the cores of the graph without the deleted
 * ones.  n_applied: edges deleted.  Errors: CM_ERR_INVALID (id out of range
 * or already dead; nothing changed). */
int cm_delete_vertices(cm_graph* g, int32_t count, const int32_t* ids, int64_t* n_applied);

/* One vertex. */
int cm_delete_vertex(cm_graph* g, int32_t v);

/* Copies the core number of every vertex (n_total int32, dead = -1) into
 * out (host or device; NULL only queries the size).  *n_total (nullable)
 * receives the vertex count.  CM_ERR_STATE if cores are stale (after
 * cm_apply_edges without cm_recompute_cores). */
int cm_get_cores(const cm_graph* g, int32_t* out, int32_t* n_total);

/* Copies SD(v), the superior degree of Section IV, Definition 7 (the number
 * of neighbours w with core(w) >= core(v)), of every vertex into out (host
 * or device, n_total int32; dead vertices -1; NULL only queries the size).
 * The library keeps SD with the cores: Algorithms 3 and 6 read it, and every
 * update call leaves it consistent with the cores it returns.  Same errors
 * as cm_get_cores. */
int cm_get_superior_degrees(const cm_graph* g, int32_t* out, int32_t* n_total);

/* Result of cm_check. */
typedef struct cm_check_report {
    int64_t vertices_checked;   /* every vertex id, live or dead */
    int64_t sd_mismatches;      /* live vertices whose stored SD differs from a recount of Definition 7
                                   (neighbours whose core is >= its own) */
    int64_t key_mismatches;     /* vertices whose 4-byte scan key is not core << 1 | (SD > core), or not
                                   the dead key for a deleted vertex */
    int64_t degree_mismatches;  /* live vertices whose degree differs from the non-hole slots of their list */
    int64_t bad_neighbour_ids;  /* list slots naming no live vertex */
    int64_t kcore_violations;   /* live vertices with fewer than core(v) neighbours of core >= core(v)
                                   (a k-core needs at least k of them, Definition 1) */
    int64_t first_bad_vertex;   /* smallest vertex that failed a check, -1 if none */
    int64_t reserved;
} cm_check_report;

/* Checks the device store against its own definitions, every vertex from
 * scratch (a debug check; one pass over all lists, O(n + m)).  Vertices
 * pinned by a vertex deletion in progress are not compared on SD, key or
 * the k-core condition.  *out is filled and CM_OK returned whether or not
 * mismatches were found; CM_ERR_STATE if the handle is poisoned or its cores
 * are stale, CM_ERR_OOM if the 64-byte counter buffer cannot be allocated,
 * CM_ERR_INVALID for NULL arguments.  Synchronises the handle's stream. */
int cm_check(cm_graph* g, cm_check_report* out);

/* Copies the current edge list (canonical pairs lo < hi, any order) into
 * host or device memory of capacity cap pairs; *m receives the edge count.
 * With cm_get_cores this is a complete checkpoint: cm_create(edges, cores)
 * resumes it.  CM_ERR_CAPACITY (nothing copied) when cap < m. */
int cm_get_edges(const cm_graph* g, int32_t* out, int64_t cap, int64_t* m);

/* Vertex count (including dead ids) and live edge count. */
int32_t cm_num_vertices(const cm_graph* g);
int64_t cm_num_edges(const cm_graph* g);

/* Applies an edge batch to the graph structure only (op CM_OP_INSERT or
 * CM_OP_DELETE), leaving core numbers stale until cm_recompute_cores.
 * Together they form the full re-peel comparator: the alternative to
 * maintenance that the paper argues against (Section I). */
int cm_apply_edges(cm_graph* g, int32_t op, const int32_t* edges, int64_t k, int64_t* n_applied);

/* Recomputes every core number from scratch by GPU bucket peeling (the
 * [O(m)] decomposition the paper cites, level-synchronous) and rebuilds
 * the per-vertex superior degrees. */
int cm_recompute_cores(cm_graph* g);

/* Counters of the most recent call. */
int cm_get_stats(const cm_graph* g, cm_stats* out);

/* Changes the stream of the handle (cudaStream_t). */
int cm_set_stream(cm_graph* g, void* stream);

/* Description of the most recent failure of g (or of the last failed
 * cm_create when g is NULL); never NULL. */
const char* cm_last_error(const cm_graph* g);

/* ---------------- many independent graphs in one handle ----------------
 * A multi-graph handle stores `ngraphs` independent graphs as one disjoint
 * union: local vertex v of graph i has global id base[i] + v.  Because no
 * edge joins two graphs, one maintenance launch serves every graph's batch
 * at once and each graph's core numbers are exactly those of the graph on
 * its own. */

/* ns[i]: vertex count of graph i; ms[i]: its edge count; edges: the graphs'
 * edge lists (local ids) concatenated in graph order (host or device);
 * cores: NULL (peel) or the concatenated core numbers.  ns and ms are host
 * arrays. */
int cm_create_multi(cm_graph** out, int32_t ngraphs, const int32_t* ns, const int64_t* ms,
                    const int32_t* edges, const int32_t* cores, const cm_options* opt, void* stream);

/* Number of graphs and the base id of each (host array of ngraphs). */
int cm_multi_bases(const cm_graph* g, int32_t* bases, int32_t* ngraphs);

/* One insert or delete batch per graph, run as a single fused call:
 * counts[i] (host) edges of graph i, local ids, concatenated in graph order
 * (host or device).  n_applied (host, nullable, ngraphs entries) receives
 * per-graph applied counts. */
int cm_update_multi(cm_graph* g, int32_t op, const int64_t* counts, const int32_t* edges,
                    int64_t* n_applied);

/* ---------------- captured update steps (many graphs, one launch) ----------------
 * Not in the paper: the batching the method's data-parallel structure
 * allows.  A step applies one insert batch and then one delete batch to
 * every graph of a handle (a multi-graph handle, or a plain one with
 * ngraphs = 1) as ONE CUDA graph replay: both batches are localised and
 * validated, then each phase ingests its batch, relocates overfull lists
 * behind a device-side capacity check, and runs the superior-edge-set
 * iterations (Algorithms 1 and 5) as a conditional loop node over the
 * grid-wide and single-block maintenance kernels.  The host only stages
 * inputs before the replay and reads one log after it.
 *
 * The handle must run on a created stream (cm_set_stream / the stream of
 * cm_create), not the legacy default stream.  Results equal two calls
 * cm_update_multi(INSERT) then cm_update_multi(DELETE) (same selection
 * rule, so the same iterations).  The captured graph bakes in device
 * pointers and the configuration; the step re-captures by itself when any
 * of them changed (buffer growth, new vertices, cm_step_set_config).  If
 * the adjacency pool cannot take a step's relocations, the replay changes
 * nothing and the step runs both phases on the ordinary path instead
 * (counted as a fallback).  Destroy steps before their handle. */
typedef struct cm_step cm_step;

/* The schedule knobs a step bakes in (the autotuner's search space). */
typedef struct cm_step_config {
    int32_t block_mode_edges;  /* as in cm_options; negative = grid mode only */
    int32_t block_mode_enter;
    int32_t block_mode_leave;
    int32_t hub_slots;         /* frontier granularity: grid-wide chunked scans from this many slots (0 = 1024, -1 never) */
    int32_t blocks_per_sm;     /* block shape of the grid-mode launch: resident 512-thread blocks per SM (0 = max) */
    int32_t block_slots;       /* frontier granularity: block-wide scans from this many slots, insert phase (0 = 4096) */
    int32_t task_claim;        /* most search tasks a warp claims at once (0 = 1) */
    int32_t reserved;
} cm_step_config;

/* max_insert / max_delete: capacity (edges) of the step's two batches.
 * cfg NULL: the handle's options.  Errors: CM_ERR_INVALID, CM_ERR_STATE
 * (default stream, poisoned handle), CM_ERR_OOM. */
int cm_step_create(cm_step** out, cm_graph* g, int64_t max_insert, int64_t max_delete, const cm_step_config* cfg);

/* Runs one step.  ins_counts / del_counts (host, ngraphs entries, NULL =
 * all zero): edges per graph; ins_edges / del_edges: the batches in local
 * ids, concatenated in graph order (host or device).  ins_applied /
 * del_applied (host, nullable, ngraphs entries) receive per-graph applied
 * counts.  Errors: CM_ERR_CAPACITY (a batch above the step's capacity;
 * nothing runs), CM_ERR_INVALID (an id out of range or deleted in either
 * batch; nothing changes), CM_ERR_STATE, CM_ERR_LIMIT / CM_ERR_CUDA
 * (poison the handle).  cm_get_stats then reports both phases together. */
int cm_step_run(cm_step* s, const int64_t* ins_counts, const int32_t* ins_edges, const int64_t* del_counts,
                const int32_t* del_edges, int64_t* ins_applied, int64_t* del_applied);

int cm_step_get_config(const cm_step* s, cm_step_config* cfg);
int cm_step_set_config(cm_step* s, const cm_step_config* cfg);
/* Captures made, replays run, replays that fell back to the ordinary path. */
int cm_step_counters(const cm_step* s, int64_t* captures, int64_t* replays, int64_t* fallbacks);

typedef struct cm_tune_report {
    cm_step_config best;
    double best_ms;   /* median replay time of the chosen configuration */
    double first_ms;  /* median replay time of the configuration the step had before */
    int32_t tried;    /* configurations timed */
    int32_t reps;     /* replays per configuration */
} cm_tune_report;

/* Autotuner: times the step's current configuration, then tunes one knob
 * at a time (coordinate descent, 15 candidates): hub_slots in {512, 1024, 4096,
 * never}, block_slots in {256, 1024, 4096}, blocks_per_sm in {1, 2}, three
 * execution-mode threshold sets and task_claim in {1, 2, 8}, each knob keeping the fastest
 * value with the others at the best found so far.  Each candidate is timed
 * on the given batches, `reps` replays (median), restoring the graph's
 * device state and the batch before every replay; the fastest is kept on
 * the step.  The graph
 * is left exactly as before the call.  Needs device memory for one copy of
 * the graph's state.  Same batch arguments and errors as cm_step_run. */
int cm_step_autotune(cm_step* s, const int64_t* ins_counts, const int32_t* ins_edges, const int64_t* del_counts,
                     const int32_t* del_edges, int32_t reps, cm_tune_report* report);

void cm_step_destroy(cm_step* s);

/* ---------------- serving: resident graphs, continuous batching ----------------
 * Not in the paper: a request loop over graphs kept on the device.  Each
 * graph gets an equal slice of `device_budget_bytes`, split into a ring of
 * staged insert batches and a ring of staged delete batches: a request is
 * admitted (its edges copied to the device on a stream of its own, while
 * the graph's current call runs) once its ring has contiguous room, in
 * arrival order.  The graph's worker thread then takes the oldest admitted
 * requests as one round: the longest run, in arrival order, whose inserted
 * edges and deleted edges are disjoint, at most max_round_edges edges (<= 0:
 * no limit).  Applying all of its inserts and then all of its deletes is then
 * exactly applying the requests one by one, and a round is ONE update step
 * (cm_step: both batches in one CUDA graph replay; two plain calls on a
 * handle that runs on the legacy default stream).  Graphs are served by
 * separate threads, so their calls overlap on the device when the handles
 * run on separate created streams; give each handle a share of the SMs
 * (cm_options.max_sms) to let the grid-wide launches of different graphs run
 * side by side.  Each graph ends in the state of applying its requests one
 * by one, whatever the timing or the other graphs' traffic.  A request that
 * names an invalid vertex fails alone (its round is replayed request by
 * request).  Besides the budget, each graph holds one captured step sized
 * for min(slice / 16 bytes, max_round_edges) edges per operation.  The
 * server does not own the handles; while it runs, touch them only through
 * it.  Requests use local ids and host buffers (copied at submit). */
typedef struct cm_server cm_server;

typedef struct cm_request_result {
    int32_t status;          /* CM_OK or the error of the request's round */
    int32_t pad;
    int64_t round;           /* server-wide round number that applied it */
    int64_t round_applied;   /* edges the round applied (all its requests together) */
    int64_t round_edges;     /* edges the round was given */
    int64_t round_requests;  /* requests merged into the round */
    int64_t latency_ns;      /* submit -> end of its round */
    int64_t queue_ns;        /* submit -> admitted (on the device) */
} cm_request_result;

typedef struct cm_server_stats {
    int64_t submitted, completed, rounds, coalesced, failed, edges;
    int64_t p50_ns, p99_ns;  /* over completed requests, submit -> done */
    int64_t reserved[4];
} cm_server_stats;

/* Errors: CM_ERR_INVALID (bad arguments, budget below 16 bytes per graph), CM_ERR_OOM. */
int cm_server_create(cm_server** out, cm_graph* const* graphs, int32_t ngraphs, int64_t device_budget_bytes,
                     int64_t max_round_edges);
/* Queues a batch of k edges for graph `graph`; returns at once.  Errors:
 * CM_ERR_INVALID, CM_ERR_CAPACITY (k above the graph's ring for that operation, slice / 16 bytes:
 * it could never be admitted). */
int cm_server_submit(cm_server* s, int32_t graph, int32_t op, const int32_t* edges, int64_t k, int64_t* request_id);
/* Blocks until the request's round finished; returns the round's status. */
int cm_server_wait(cm_server* s, int64_t request_id, cm_request_result* out);
/* Blocks until every submitted request finished (CM_ERR_STATE if any failed). */
int cm_server_drain(cm_server* s);
/* Core numbers of a resident graph between two of its rounds (host or device out). */
int cm_server_get_cores(cm_server* s, int32_t graph, int32_t* out);
int cm_server_get_stats(cm_server* s, cm_server_stats* out);
/* Open-loop trace: request i (graph[i], op[i], counts[i] edges, edges
 * concatenated) is submitted at arrival_ns[i] after the call starts, by a
 * driver thread, whether or not earlier requests finished.  latency_ns[i]
 * (nullable) = end of its round - its scheduled arrival; round_of[i]
 * (nullable) = its round; wall_s = start -> last completion. */
int cm_server_run_trace(cm_server* s, int64_t nreq, const int64_t* arrival_ns, const int32_t* graph,
                        const int32_t* op, const int64_t* counts, const int32_t* edges, int64_t* latency_ns,
                        int64_t* round_of, double* wall_s);
void cm_server_destroy(cm_server* s);

/* ---------------- decomposition without device allocation ----------------
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot call cudaMalloc -- a process whose framework already reserved the
 * device memory for its own pool, or a latency-critical loop that must not
 * wait on the allocator (cudaMalloc / cudaFree may synchronise the device).
 *
 * Computes the core number of every vertex of a static simple undirected
 * graph given as CSR in DEVICE memory: row_off (n+1 int64, non-decreasing,
 * row_off[0] = 0) and adj (row_off[n] int32 neighbour ids, every edge listed
 * in both endpoints' rows).  cores (device, n int32) receives the result.
 * Runs on `stream` (cudaStream_t) and returns after completion.  It
 * allocates nothing: its scratch is one static device array sized for at
 * most 1,048,576 vertices (16 MiB, plus 2 MiB of chunk tasks for the lists
 * of high-degree vertices and a 4 KiB control block), held by every
 * GPU that loads the library until the process exits.  All calls share that
 * array: calls whose work overlaps on the GPU (for example on two streams)
 * race on it and must not be issued.  The first call on a device looks up
 * the array's device address (once per device); make that first call
 * before any stream capture.  Each call synchronises `stream` before it
 * returns (it reads the kernel's error word back to the host).
 * Errors: CM_ERR_INVALID (n < 0, NULL or host pointers), CM_ERR_CAPACITY
 * (n > 1,048,576; nothing runs), CM_ERR_LIMIT (a bounded device wait ran
 * out), CM_ERR_CUDA. */
int cm_core_numbers_noalloc(int32_t n, const int64_t* row_off, const int32_t* adj, int32_t* cores, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* COREMAINT_H */
