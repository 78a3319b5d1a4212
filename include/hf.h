/*
 * hf.h -- C ABI of a B300 (sm_103a) executor for task dependency graphs.
 *
 * Task model (Heteroflow, "Concurrent CPU-GPU Task Programming using Modern C++",
 * Section III-A): a graph is a DAG of tasks of four kinds -- host, pull, push and kernel --
 * joined by explicit dependency edges; a task runs only after every task that precedes it
 * has finished, the library adds no implicit edge, and the graph must be acyclic. Running a
 * graph is non-blocking (Section III-B): hf_run only enqueues work on a CUDA stream.
 *
 * Every task carries an FP32 arrival time (timing-graph max-plus propagation, the paper's
 * timing-analysis setting, Section IV-A): a task with no predecessor starts at its source
 * arrival (default +0), every other task ends with
 *         arr[v] = max over edges (u, v) of  arr[u] + d(u, v)
 * where each sum is one binary32 add rounded to nearest even and the max uses the total
 * order -inf < ... < -0 < +0 < ... < +inf. Results are bit-identical for every schedule.
 *
 * Conventions for every call:
 *   - returns hf_status; no C++ exception crosses this boundary;
 *   - "device" pointers are CUDA device (or managed) addresses on the current device,
 *     "host" pointers are host addresses; pull/push host buffers must be page-locked
 *     (cudaHostAlloc / cudaHostRegister), the executors read and write them directly;
 *   - a stream argument is a cudaStream_t passed as void* (NULL = legacy default stream);
 *   - the library owns every device buffer it allocates for a graph (through the allocator
 *     installed with hf_set_allocator, else cudaMalloc/cudaFree) and frees it in
 *     hf_graph_destroy / hf_batch_destroy;
 *   - buffers named in payloads are BORROWED: the caller keeps them alive and leaves them
 *     alone until the run that uses them has completed (the paper's stateful, by-reference
 *     task arguments, Section III-A "Pull Task");
 *   - one graph is not thread-safe for mutation; distinct graphs may run concurrently on
 *     distinct streams.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hf_graph hf_graph;     /* opaque, created by hf_graph_create */
typedef struct hf_batch hf_batch;     /* opaque, created by hf_batch_create */
typedef int32_t hf_task;              /* dense task id, 0..n-1 in creation order (a task handle) */

typedef enum {
    HF_OK = 0,
    HF_EINVAL = 1,     /* bad argument: id out of range, NaN/inf delay, bad payload, NULL pointer */
    HF_ENOMEM = 2,     /* host or device allocation failed */
    HF_ECYCLE = 3,     /* the dependency edges form a cycle (self-loops included) */
    HF_ESTATE = 4,     /* call not valid now: graph mutated while in a batch or run in flight, ... */
    HF_ETIMEDOUT = 5,  /* the persistent executor saw no progress for spin_limit_ns and gave up */
    HF_EQUEUE = 6,     /* a device queue overflowed (internal error; never expected) */
    HF_ECUDA = 7,      /* a CUDA runtime call failed; hf_last_error() has its message */
    HF_ENOTSUP = 8     /* valid request this build does not support (e.g. a validate run of the team executor) */
} hf_status;

/* The paper's four task kinds (Section I; Section III-A). */
typedef enum { HF_HOST = 0, HF_PULL = 1, HF_PUSH = 2, HF_KERNEL = 3 } hf_kind;

/* Built-in kernel payloads. HF_K_SAXPY_I32 is Listing 1's kernel (y = a*x + y on int32,
 * two's-complement wrap); HF_K_SAXPY_F32 its FP32 form with one fused multiply-add. */
typedef enum { HF_K_MAXPLUS = 0, HF_K_SAXPY_F32 = 1, HF_K_SAXPY_I32 = 2 } hf_kernel_op;

/* --- payloads, copied at hf_add_task time (pointers inside are borrowed) ---------------- */

/* kind HF_KERNEL, op HF_K_MAXPLUS: arrival propagation only. arr0 is the arrival used when
 * the task has no predecessor (finite; default +0 when payload is NULL). */
typedef struct { int32_t op; float arr0; } hf_maxplus_payload;

/* kind HF_KERNEL, op HF_K_SAXPY_F32 / HF_K_SAXPY_I32: y[i] = a*x[i] + y[i], i < n.
 * x comes from pull task x_pull (its device buffer, Section III-A "Kernel Task": pull tasks
 * are the data gateway) or, when x_pull == -1, from device pointer x_dev; likewise y.
 * A pull used as an operand must hold at least n * 4 bytes. Device pointers must be 4-byte
 * aligned; n >= 0. The library adds no edge from the pull: order it with hf_precede. */
typedef struct {
    int32_t op;
    int32_t a_i;     /* scalar for HF_K_SAXPY_I32 */
    float a_f;       /* scalar for HF_K_SAXPY_F32 */
    hf_task x_pull;  /* -1: use x_dev */
    hf_task y_pull;  /* -1: use y_dev */
    int32_t pad_;
    int64_t n;       /* elements */
    void* x_dev;
    void* y_dev;
} hf_saxpy_payload;

/* kind HF_PULL: copy `bytes` from page-locked host memory into a device buffer that the
 * library allocates for this task (Section III-A "Pull Task"). */
typedef struct { const void* host_ptr; size_t bytes; } hf_pull_payload;

/* kind HF_PUSH: copy `bytes` into page-locked host memory from pull task src_pull's device
 * buffer (Section III-A "Push Task") or, when src_pull == -1, from device pointer src_dev. */
typedef struct { hf_task src_pull; int32_t pad_; const void* src_dev; void* host_ptr; size_t bytes; } hf_push_payload;

/* kind HF_HOST: fn(arg) runs on a CPU thread (Section III-A "Host Task"). The level-synchronous
 * executor makes it a host node of its CUDA graph. The team and persistent executors post it to
 * a mailbox in mapped page-locked memory, where a proxy thread of the library runs the posted
 * tasks in posting order and raises each one's done flag; the device waits for the flag
 * (bounded by spin_limit_ns: HF_ETIMEDOUT) before the task's successors run. The team executor
 * posts a level's host tasks once the level's device work is done; the persistent executor
 * posts a host task when it becomes ready, and only the warp that took it waits. Callbacks must
 * not wait for the run itself. */
typedef struct { void (*fn)(void* arg); void* arg; } hf_host_payload;

/* --- run options ---------------------------------------------------------------------- */

/* HF_MODE_TEAM: persistent executor for batches of independent graphs. One launch; each graph
 * is a job, taken from a job queue longest predicted first and run level by level with a
 * barrier between levels instead of a kernel boundary: one CTA and CTA barriers for most
 * graphs, the CTAs of one thread-block cluster and the hardware cluster barrier for the longest
 * ones. The next levels' task lists and in-edges are staged in shared memory by TMA bulk
 * copies while the current level runs. The cluster size and which graphs get a cluster come
 * from predicted task costs (HF_PRIO_HEURISTIC, or HF_PRIO_LEARNED with a cost model attached;
 * HF_PRIO_FIFO: one CTA per graph in batch order). Payload pieces default to 512 elements. */
typedef enum { HF_MODE_LEVELSYNC = 0, HF_MODE_PERSISTENT = 1, HF_MODE_AUTO = 2, HF_MODE_TEAM = 3 } hf_mode;
typedef enum { HF_PRIO_FIFO = 0, HF_PRIO_HEURISTIC = 1, HF_PRIO_LEARNED = 2 } hf_priority;

typedef struct {
    int32_t mode;           /* hf_mode */
    int32_t priority;       /* hf_priority (persistent executor) */
    int32_t ctas;           /* persistent: CTAs launched; 0 = two per SM (within occupancy), one
                               per SM with work stealing */
    int32_t warps_per_cta;  /* persistent: fixed at 8 in this build (the field is ignored) */
    int32_t claim;          /* persistent: most queue slots a warp claims at once (it claims its
                               fair share of the backlog), 1..32; default 8 */
    int32_t local_keep;     /* persistent: ready tasks a warp keeps in shared memory, 0..16;
                               negative = default (16) */
    int64_t chunk_elems;    /* payload split size in elements (saxpy) or 4-byte words (copies);
                               0 = 16384 (persistent) / 512 (level-sync); in HF_MODE_AUTO it
                               applies only when the persistent executor is chosen */
    uint64_t spin_limit_ns; /* persistent: give up (HF_ETIMEDOUT) after this long without any
                               task completing; 0 = 2 s */
    int32_t instrument;     /* bit 0: record per-task %globaltimer start/end (hf_get_task_times;
                               persistent executor) or per-graph start/end (team executor,
                               hf_batch_get_graph_times); bit 1: record persistent-executor
                               counters (hf_batch_get_stats); bit 2: record per-task costs in the
                               team executor (hf_batch_get_task_costs) */
    int32_t validate;       /* record per-task start/finish tickets and execution counts */
    int32_t stall_task;     /* failure-injection hook for tests: -1 = off; else this task's
                               pending-predecessor counter starts one too high, so it never
                               becomes ready and a persistent run ends with HF_ETIMEDOUT */
    int32_t time_kernel;    /* record CUDA events around the executor's main work (read with
                               hf_kernel_ms / hf_batch_kernel_ms) */
    int32_t payload_warps;  /* persistent: warps per CTA (0..7) that only run payload tasks,
                               taken from a separate payload queue; 0 = every warp runs both */
    int32_t team_size;      /* team: thread-block cluster size for every graph, 1..16 (above 16:
                               16); 0 = cluster size and clustered graphs chosen from predicted
                               costs (one CTA per graph under HF_PRIO_FIFO) */
    int32_t team_scale;     /* team planner: factor on the predicted payload cost, standing for
                               the slowdown of memory traffic when every graph streams at once;
                               larger values give payload-heavy graphs larger teams; s > 0: s,
                               s < 0: 1 / -s; 0 = 4 for heuristic costs (a 512-element piece:
                               ~0.75 us for a warp alone, ~3 us when every SM streams, measured on
                               B300), 1 for learned costs (recorded under the team executor's
                               real load) */
    int32_t steal_ring;     /* persistent: 0 = one global ready queue; > 0 = work stealing
                               (Section III-C): every CTA owns a ring of this many slots (rounded
                               up to a power of two, 64..16384) that its warps push ready tasks
                               and payload pieces to and take from first; a warp with nothing in
                               its ring or the global queue (sources, ring overflow) steals half
                               of the published front of a random other CTA's ring */
    int32_t copy_warps;     /* persistent: warps per CTA (0..2) that run only pull copies, and as
                               many that run only push copies, each direction from a queue of its
                               own, so that host-to-device and device-to-host copies share the
                               host link's two directions instead of queueing behind each other
                               and behind the other tasks; 0 = copies run like other payloads.
                               (The level-synchronous executor always runs copies as copy-engine
                               nodes of its CUDA graph, each ordered only by its own edges.) */
    int32_t team_fold;      /* team planner (team_size 0): 0 = one launch per team size, run
                               concurrently (each launched once the larger clusters before it
                               are resident); K in {2, 4, 8, 16} = one launch with cluster size K:
                               every graph gets a K-CTA cluster or one CTA, the clusters take their
                               graphs first and then, like the other CTAs, single-CTA graphs; -1 =
                               one launch, K chosen by the planner's predicted makespan */
    int32_t team_global_keys; /* team executor, batches without payloads: 0 = a graph run on a
                               thread-block cluster of 2^j CTAs whose arrival keys fit in the
                               cluster's shared memory (task count / cluster size entries per CTA,
                               every CTA of its class still resident) keeps them there for the
                               whole job, loaded and stored through distributed shared memory, and
                               writes them out after its last level; 1 = every key in global
                               memory. Single-CTA jobs always keep theirs in global memory.
                               Results are identical either way. */
} hf_run_opts;

void hf_run_opts_default(hf_run_opts* opts);

/* --- graph construction (Section III-A) ------------------------------------------------ */

hf_status hf_graph_create(hf_graph** out, int64_t reserve_tasks, int64_t reserve_edges);
hf_status hf_graph_destroy(hf_graph* g);   /* waits for the graph's last run to finish */

/* Adds one task; *out receives its id. payload/payload_bytes must match the kind:
 * HF_KERNEL: hf_maxplus_payload or hf_saxpy_payload (selected by its op field), or NULL for
 * max-plus with arr0 = +0; HF_PULL: hf_pull_payload; HF_PUSH: hf_push_payload; HF_HOST:
 * hf_host_payload. References to other tasks (x_pull, src_pull, ...) must name existing
 * pull tasks. */
hf_status hf_add_task(hf_graph* g, hf_kind kind, const void* payload, size_t payload_bytes, hf_task* out);

/* Adds n max-plus kernel tasks with ids first..first+n-1; arr0 (host, n floats) or NULL. */
hf_status hf_add_tasks_bulk(hf_graph* g, int64_t n, const float* arr0, hf_task* first_out);

/* Edge a -> b ("a precedes b", Section III-A "Add a Dependency Link") with delay 0, or with
 * the given finite delay. Duplicate edges are allowed (each counts). Cycles are reported by
 * hf_finalize / hf_run. */
hf_status hf_precede(hf_graph* g, hf_task a, hf_task b);
hf_status hf_precede_w(hf_graph* g, hf_task a, hf_task b, float delay);

/* m edges src[i] -> dst[i] (host arrays); delay NULL = all 0. All-or-nothing: on HF_EINVAL
 * no edge is added. */
hf_status hf_precede_bulk(hf_graph* g, int64_t m, const int32_t* src, const int32_t* dst, const float* delay);

/* Writes the graph in Graphviz DOT to the file at `path` (Section III-A's graph dump): one node
 * per task labelled "<id> <kind> ..." (maxplus arr0=..., saxpy n=..., pull/push <bytes> B,
 * host), one edge per dependency labelled with its delay. Host only; any time. */
hf_status hf_dump(const hf_graph* g, const char* path);

/* Device placement (Section III-C, Algorithm 1): kernel tasks are grouped with the pull tasks
 * whose buffers they use, and push tasks with the pull they read (union-find), so that a group
 * never spans devices; the groups are packed onto ndev devices by decreasing cost, each onto the
 * least-loaded device. cost: host float[n] per-task costs, or NULL for the heuristic
 * 300 ns + 30 ns per out-edge + payload bytes / 8 bytes per ns. dev_out: host int32[n], the
 * device of each task, -1 for host tasks. Host only. */
hf_status hf_place(const hf_graph* g, int32_t ndev, const float* cost, int32_t* dev_out);

/* Host-side preparation: successor (CSR) and level-sorted predecessor lists, in-degrees,
 * topological levels, cycle check. Optional: hf_run finalizes a changed graph itself. */
hf_status hf_finalize(hf_graph* g);

typedef struct {
    int64_t tasks, edges;
    int32_t levels;         /* 1 + longest hop count from a source; 0 before finalize */
    int32_t sources;
    int64_t kind_count[4];  /* indexed by hf_kind */
    int64_t payload_tasks;  /* tasks with a saxpy or copy payload */
    int32_t finalized;
    int32_t pad_;
} hf_graph_info_t;

hf_status hf_graph_info(const hf_graph* g, hf_graph_info_t* info);
/* level (longest hop count from a source) of every task, after finalize; host array of n. */
hf_status hf_get_levels(const hf_graph* g, int32_t* level_out);

/* --- execution (Section III-B) --------------------------------------------------------- */

/* Enqueues one execution of the graph on `stream` and returns (non-blocking). opts NULL =
 * defaults. Device-side failures are reported by hf_sync_status. Re-running a graph re-runs
 * every payload (saxpy updates y again). */
hf_status hf_run(hf_graph* g, void* stream, const hf_run_opts* opts);
/* One execution on new edge delays read from host memory, with every arrival copied back to
 * host memory: the same result as hf_set_delays(delay, host) + hf_run + hf_get_arrivals, but
 * non-blocking like hf_run. The paper has no counterpart; it serves callers that stream timing
 * views through the graph. delay: m floats in insertion order (as hf_set_delays), or NULL to
 * keep the current delays; arr_out: n floats, or NULL. Both must be page-locked host memory
 * (cudaHostAlloc / cudaHostRegister), else HF_EINVAL and nothing is enqueued. The device reads
 * delay directly (no staging copy) on `stream` before the run; leave it unchanged until the
 * run has ended. The arrivals are converted on `stream` after the run and copied to arr_out on
 * a stream of the library's own, so that `stream` goes on at once with the caller's next work
 * (the next view's delays and run overlap this copy): arr_out is complete when hf_sync_status
 * for this run returns (a synchronisation of `stream` alone does not cover the copy).
 * Non-finite delays: as hf_set_delays. */
hf_status hf_run_host(hf_graph* g, void* stream, const hf_run_opts* opts, const float* delay, float* arr_out);

/* Section III-B's run_n and run_until. hf_run_n enqueues n runs back to back on `stream` (the
 * plan is reused; payloads apply n times) and returns at once; hf_sync_status then reports the
 * first failure of the n runs. hf_run_until runs, waits and calls pred(ctx) on the calling
 * thread after each run until it returns nonzero or max_runs runs have completed (*runs_out:
 * runs done); a failed run ends the loop with its status. Batch forms below. */
hf_status hf_run_n(hf_graph* g, void* stream, const hf_run_opts* opts, int32_t n);
hf_status hf_run_until(hf_graph* g, void* stream, const hf_run_opts* opts, int32_t (*pred)(void* ctx), void* ctx,
                       int32_t max_runs, int32_t* runs_out);

/* Waits for the graph's last run and returns its device status (HF_OK, HF_ETIMEDOUT, ...). */
hf_status hf_sync_status(hf_graph* g);

/* Arrival times of the last run (n floats). on_device != 0: `out` is a device pointer and the
 * copy is enqueued on the run's stream; else `out` is host memory and the call blocks. */
hf_status hf_get_arrivals(hf_graph* g, float* out, int on_device);

/* validate runs: per-task start and finish tickets (host int64[n]; from one global counter,
 * so finish[u] < start[v] for every edge u -> v) and execution counts (host int32[n]). */
hf_status hf_get_stamps(hf_graph* g, int64_t* start, int64_t* finish, int32_t* exec_count);

/* instrument runs: per-task %globaltimer start/end in ns (host int64[n]). */
hf_status hf_get_task_times(hf_graph* g, int64_t* t_start_ns, int64_t* t_end_ns);

/* time_kernel runs: device time (ms) of the executor's main work in the last run -- the
 * persistent kernel, or the whole level-synchronous CUDA graph -- from CUDA events on the
 * run's stream (the reset kernel before a persistent launch is not included). Blocks until
 * the run has finished. */
hf_status hf_kernel_ms(hf_graph* g, float* ms);

/* Replaces every edge delay of the graph's device plan (a new timing view of the same
 * circuit): delay[e] is the new delay of the e-th edge in the order edges were added
 * (hf_precede*), m floats, all finite (checked on the device: a non-finite delay is stored
 * anyway and makes every later hf_sync_status return HF_EINVAL until delays are set again).
 * on_device != 0: `delay` is a device pointer; else host memory: page-locked memory is read by
 * the device directly (leave it unchanged until `stream` has passed this point), other host
 * memory through a staging copy. Enqueued on `stream`; later runs on any
 * stream see the new delays once that stream has reached this point. The graph's own edge
 * list keeps the delays it was built with (they return if the plan is ever rebuilt, e.g.
 * after a mutation). Finalizes and uploads the graph first if needed. */
hf_status hf_set_delays(hf_graph* g, const float* delay, int on_device, void* stream);

/* --- batches: many independent graphs in one launch ------------------------------------- */

hf_status hf_batch_create(hf_batch** out);
hf_status hf_batch_destroy(hf_batch* b);
/* Appends a graph (finalizing it if needed); *index_out gets its position. The graph must not
 * be mutated while it belongs to a batch (HF_ESTATE); destroy the batch first. */
hf_status hf_batch_add(hf_batch* b, hf_graph* g, int32_t* index_out);
hf_status hf_batch_run(hf_batch* b, void* stream, const hf_run_opts* opts);
/* As hf_run_host for a batch: delay holds every graph's edge delays concatenated in batch order
 * (as hf_batch_set_delays), arr_out receives every graph's arrivals concatenated in batch order
 * (as hf_batch_get_arrivals with index -1); arr_out is complete when hf_batch_sync_status for
 * this run returns. */
hf_status hf_batch_run_host(hf_batch* b, void* stream, const hf_run_opts* opts, const float* delay, float* arr_out);
hf_status hf_batch_sync_status(hf_batch* b);
hf_status hf_batch_run_n(hf_batch* b, void* stream, const hf_run_opts* opts, int32_t n);
/* Sharding of a batch over ndev devices (one process per GPU, each running its own share):
 * graphs packed by decreasing heuristic cost (the sum of hf_place's per-task heuristic), each onto
 * the least-loaded device. dev_of_graph: host int32[graphs]; load_out: host double[ndev] or NULL.
 * Host only. */
hf_status hf_batch_partition(const hf_batch* b, int32_t ndev, int32_t* dev_of_graph, double* load_out);
hf_status hf_batch_run_until(hf_batch* b, void* stream, const hf_run_opts* opts, int32_t (*pred)(void* ctx),
                             void* ctx, int32_t max_runs, int32_t* runs_out);
/* Arrivals of graph `index` (its n floats), as hf_get_arrivals; index -1: every graph's
 * arrivals concatenated in batch order (sum of their task counts) in one copy. */
hf_status hf_batch_get_arrivals(hf_batch* b, int32_t index, float* out, int on_device);
hf_status hf_batch_get_task_times(hf_batch* b, int32_t index, int64_t* t_start_ns, int64_t* t_end_ns);
hf_status hf_batch_get_stamps(hf_batch* b, int32_t index, int64_t* start, int64_t* finish, int32_t* exec_count);
hf_status hf_batch_kernel_ms(hf_batch* b, float* ms);
/* Counters of the last persistent run with instrument bit 1 (host int64 out[n], n <= 16): warp
 * rounds with work, items processed, idle polls, successor releases, CAS attempts, ready tasks
 * kept in warp stacks, items pushed to / claims on / items popped from the global queue,
 * payload pieces run, SM cycles in rounds with work (4 counters: rounds, releases, CAS
 * sections, pushes), and with work stealing the items pushed to CTA rings and the items stolen
 * from another CTA's ring. Diagnostics only. */
hf_status hf_batch_get_stats(hf_batch* b, int64_t* out, int32_t n);
/* Per-graph %globaltimer start and end (ns; host arrays of the batch's graph count) of the last
 * team-executor run with instrument bit 0: when the graph's job started and when its last
 * level ended. */
hf_status hf_batch_get_graph_times(hf_batch* b, int64_t* start_ns, int64_t* end_ns);
/* Per-task costs (ns) recorded by the last team-executor run with instrument bit 2, into a host
 * array: for graph `index` its task count, for index -1 every graph's tasks concatenated in batch
 * order. A task's cost is what the team spent on it under the run's real load: for every task the
 * time of its thread's gather (predecessor keys in, arrival key stored), plus, for a payload
 * task, the summed times of the warps that ran its pieces. These are the costs the team planner
 * consumes, and the cost model's training target. */
hf_status hf_batch_get_task_costs(hf_batch* b, int32_t index, float* cost_ns);
/* Kernels the last run launched (executor kernels; copies and memsets not counted): one per
 * level for the level-synchronous executor, 2 for the persistent one (reset + executor), one
 * per team class for the team executor. */
hf_status hf_batch_last_launches(hf_batch* b, int32_t* n);
/* Team size (CTAs) each graph of the batch ran on in the last team-executor run, into a host
 * array of the batch's graph count: 1 for a single-CTA job, 2, 4, 8 or 16 for a thread-block
 * cluster, 0 for a graph without tasks. HF_ESTATE before the first team-executor run. */
hf_status hf_batch_team_plan(hf_batch* b, int32_t* team_size);
/* Whether each graph of the batch kept its arrival keys in its cluster's distributed shared
 * memory in the last team-executor run (1) or in global memory (0), into a host array of the
 * batch's graph count (see hf_run_opts::team_global_keys). HF_ESTATE before the first
 * team-executor run. */
hf_status hf_batch_team_keys(hf_batch* b, int32_t* shared);
/* How each graph of the batch ran in the last team-executor run, as bits into a host array of
 * the batch's graph count: 1 its keys lived in its cluster's distributed shared memory (as
 * hf_batch_team_keys); 2 its levels were software-pipelined (graphs of at least 32,768 tasks:
 * each thread reads its next level's task during the current level's gather); 4 its payload
 * tasks touch pairwise disjoint memory wherever one of them writes (checked on the host from
 * the payloads' address ranges: saxpy writes y and reads x and y, a copy writes its destination
 * and reads its source; a graph with host tasks never qualifies), so its cluster levels release
 * only the arrival keys. HF_ESTATE before the first team-executor run. */
hf_status hf_batch_team_flags(hf_batch* b, int32_t* flags);
/* As hf_set_delays for every graph of the batch: delay holds the graphs' edge delays
 * concatenated in batch order (sum of their edge counts). */
hf_status hf_batch_set_delays(hf_batch* b, const float* delay, int on_device, void* stream);

/* --- learned cost model ------------------------------------------------------------------
 * The paper's scheduler (Section III-C) orders ready tasks with a plain heuristic (FIFO work
 * stealing); it has no learned component. This library adds one, kept beside the heuristic:
 * an MLP 12 -> 64 -> 64 -> 1 (ReLU, BF16 weights and activations, FP32 accumulation and FP32
 * master weights) maps per-task features to a predicted log task cost (log ns that the team
 * executor spends on the task, as its cost recording measures it: hf_batch_get_task_costs).
 * Predicted costs plan the team executor (its payload cost per level, hence team sizes and job
 * order), give bottom-level weights b(v) = c(v) + max over successors b(s) (the remaining
 * critical path) that order the persistent executor's initial ready queue (its sources), and
 * give the predicted makespans that choose between the executors in HF_MODE_AUTO. Results
 * (arrivals, payload data) never depend on the model.
 *
 * Parameter vector (HF_COSTMODEL_PARAMS floats, row-major): W1[64][12], b1[64], W2[64][64],
 * b2[64], w3[64], b3. W1, W2, w3 are used rounded to BF16 (round to nearest even).
 * Feature vector per task (HF_FEATURES floats): one-hot max-plus / saxpy / pull / push,
 * log1p(fan-in), log1p(fan-out), level / levels, log1p(level), log1p(payload bytes),
 * log1p(tasks of its graph), log1p(edges of its graph), log1p(mean fan-out of successors). */

#define HF_COSTMODEL_PARAMS 5057
#define HF_FEATURES 12

typedef struct hf_costmodel hf_costmodel;

/* New model with He-uniform weights (limit sqrt(6/fan_in)) drawn from `seed`, zero biases. */
hf_status hf_costmodel_create(hf_costmodel** out, uint64_t seed);
hf_status hf_costmodel_destroy(hf_costmodel* cm);
/* Host arrays of HF_COSTMODEL_PARAMS floats (FP32 master weights); set also resets Adam. */
hf_status hf_costmodel_set_params(hf_costmodel* cm, const float* params);
hf_status hf_costmodel_get_params(hf_costmodel* cm, float* params);
hf_status hf_costmodel_save(hf_costmodel* cm, const char* path);  /* flat FP32 file */
hf_status hf_costmodel_load(hf_costmodel* cm, const char* path);

/* Device arrays: X[n][12] features, y[n] predictions (log ns). Enqueued on `stream`. */
hf_status hf_costmodel_forward(hf_costmodel* cm, const float* X, int64_t n, float* y, void* stream);
/* Gradient of mean((y - t)^2) over the n rows w.r.t. the parameter vector (device grad[P],
 * overwritten) and the loss (device float, overwritten). */
hf_status hf_costmodel_grad(hf_costmodel* cm, const float* X, const float* t, int64_t n, float* grad,
                            float* loss, void* stream);
/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8; bias-corrected) with device grad[P]. */
hf_status hf_costmodel_adam_step(hf_costmodel* cm, const float* grad, float lr, void* stream);
/* Mini-batch Adam training on device rows (X, t): `epochs` passes in an order shuffled by
 * `seed`, `batch` rows per step. *final_loss (host) = loss over all rows afterwards. Blocks. */
hf_status hf_costmodel_train(hf_costmodel* cm, const float* X, const float* t, int64_t n, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float* final_loss, void* stream);

/* Features of every task of the batch (graphs concatenated in batch order) into device
 * X[sum of tasks][12]; and of a single graph. */
hf_status hf_batch_features(hf_batch* b, float* X, void* stream);
hf_status hf_features(hf_graph* g, float* X, void* stream);

/* Attach a model to a batch (NULL detaches): HF_PRIO_LEARNED and HF_MODE_AUTO use it. The
 * model is borrowed; weights are read when priorities are (re)computed (first run with a
 * priority mode after attaching, or hf_batch_refresh_priorities). */
hf_status hf_batch_set_costmodel(hf_batch* b, hf_costmodel* cm);
hf_status hf_batch_refresh_priorities(hf_batch* b, void* stream);
/* Per-task predicted cost (ns) and bottom-level weight under `priority` (HEURISTIC or
 * LEARNED), device arrays of the batch's task count. */
hf_status hf_batch_task_costs(hf_batch* b, int32_t priority, float* cost, float* bottom, void* stream);
/* Bottom-level weights for caller-given per-task costs (device arrays of the batch's task
 * count): b(v) = c(v) + max over successors b(s) in FP32 (one rounded add per task), sinks
 * b = c. Enqueued on `stream`. */
hf_status hf_batch_bottom_levels(hf_batch* b, const float* cost, float* bottom, void* stream);

/* --- autotuning and executor choice ----------------------------------------------------- */

/* Times trial runs on this batch and writes the fastest options to *best (other fields from
 * `base`, NULL = defaults) and its time to *best_ms; each trial is one warm-up run, then three
 * blocks of three runs enqueued back to back (as a caller streaming runs issues them), timed
 * by CUDA events: the median block's time per run. base->mode HF_MODE_TEAM tunes the team
 * executor (coordinate descent over the planner's payload-cost scale from 1/4 to 16, the
 * cluster size for every graph, 0 = the cost model's plan, the payload piece size, and one launch
 * per team size or one folded launch); any other mode tunes the
 * persistent executor (CTA count, queue claim size, shared-memory stack depth, payload piece
 * size, payload warps, global queue or work stealing, copy warps; mode PERSISTENT in *best).
 * Results are cached per executor, priority source (base->priority) and size bucket (tasks,
 * edges per task, payload share, depth, batch or single graph), so a later call on a similar
 * batch returns without trials unless `force`. Runs the batch many times: payloads run each time (saxpy updates y). Blocks. */
hf_status hf_batch_autotune(hf_batch* b, void* stream, const hf_run_opts* base, int force, hf_run_opts* best,
                            float* best_ms);

/* Predicted makespans (ms) of the batch under each executor, from per-task costs of the given
 * priority source (HEURISTIC or LEARNED) and machine constants measured once per process on a
 * calibration chain (level-synchronous time per level, persistent time per hop, team time per
 * level for one CTA and for a cluster):
 *   level-sync  = levels * t_level (x 2.5 when the level data exceed half the L2) + sum over
 *                 levels of r_level * its in-edges over the SMs its CTAs occupy + sum over
 *                 levels of the largest saxpy- or host-task cost in it
 *   persistent  = critical path of costs + depth * t_hop + total cost / warps
 *   (both at least the copies' host-link time: each direction's bytes over its bandwidth, and
 *   all copy bytes over the bandwidth of both directions at once)
 *   team        = the team executor's planned makespan: per graph and cluster size k,
 *                 T(k) = sum over levels of t_lvl(k) * ceil(width / 256k) + r(k) * in-edges / k
 *                 + payload cost / 8k (t_lvl x 2.5 for levels too large to stage in shared
 *                 memory; r(k): hf_calibration's time per in-edge gathered on one SM),
 *                 the longest graphs on clusters, the rest on single CTAs (+inf with host tasks)
 * HF_MODE_AUTO runs the executor with the smallest prediction (LEARNED costs when a model is
 * attached, else HEURISTIC). */
hf_status hf_batch_predict(hf_batch* b, int32_t priority, void* stream, float* levelsync_ms, float* persistent_ms,
                           float* team_ms);
/* The machine constants behind the predictions, measured on first use in this process on the
 * current device: on the calibration chain (2,048 tasks, one per level) the level-synchronous
 * time per level, the persistent time per dependent hop, the team time per level on one CTA and
 * on a cluster (ns); the host link's bandwidth host to device, device to host, and both
 * directions at once (GB/s, the best of three 64 MiB copies between page-locked memory and the
 * device; both at once: the bytes of two concurrent copies over their common time); and, from a
 * wide calibration graph (512 levels of 256 tasks, 4 in-edges a task), the time per in-edge
 * gathered on one SM in a level (ns): level-synchronous, team on one CTA, team on a 4-CTA
 * cluster (a level's gather is bound by the SM's rate of scattered key loads). out[10].
 * Blocks the first time. */
hf_status hf_calibration(void* stream, float* out);

/* --- allocation-free entry point -------------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory: code that runs inside another framework's memory pool or under a fixed
 * memory budget, plug-ins whose host application forbids cudaMalloc, and loops where an
 * allocation, or the device-wide synchronisation cudaFree can bring, is not acceptable.
 *
 * hf_run_csr_noalloc computes the arrivals of one max-plus graph (the same result, bit for
 * bit, as hf_run on a graph of max-plus tasks with these edges) without any allocation: no
 * cudaMalloc, no cudaFree, no allocator hook, no graph object. Its scratch (12 bytes per task
 * plus 512 bytes) is a fixed device array inside the library, HF_NOALLOC_MAX_TASKS tasks
 * large (12 MiB), that every GPU where the library is loaded holds until the process exits.
 * Arguments (device pointers on the current device, all owned by the caller):
 *   n_tasks  tasks 0..n_tasks-1, 0 <= n_tasks <= HF_NOALLOC_MAX_TASKS (larger: HF_EINVAL);
 *   n_edges  edges, >= 0;
 *   row_ptr  int32[n_tasks + 1], CSR row starts: the successors of task v are
 *            succ[row_ptr[v] .. row_ptr[v+1]), row_ptr[0] = 0, row_ptr[n_tasks] = n_edges;
 *   succ     int32[n_edges] successor ids; delay float[n_edges] finite edge delays d(u, v);
 *   arr0     float[n_tasks] source arrivals, or NULL for +0: entry v is read only when task v
 *            has no predecessor, and must then be finite (other entries may hold anything);
 *   arr      float[n_tasks] output arrivals;
 *   spin_limit_ns  give up with HF_ETIMEDOUT after this long without progress (0 = 2 s);
 *   stream   cudaStream_t the work is enqueued on; the call then waits for that stream.
 * Errors: HF_EINVAL for sizes, NULL pointers or (found on the device) a malformed CSR, an
 * out-of-range successor, a non-finite delay or a non-finite arr0 of a source, with arr left
 * unwritten; HF_ETIMEDOUT when the edges form a cycle (arr partly written); HF_ECUDA for a
 * CUDA failure. The call returns only after `stream` has completed the work (it reads the
 * result status back from the device).
 * The first call on each device looks up the array's device address and sizes the grid
 * (with that device current); make that first call before any stream capture. Every call
 * on a device uses the same array: it clears what it reads before use, but two calls whose
 * work overlaps on the GPU (other streams, other host threads) race and corrupt each
 * other's results, so serialise them. */
#define HF_NOALLOC_MAX_TASKS 1048576
hf_status hf_run_csr_noalloc(int32_t n_tasks, int32_t n_edges, const int32_t* row_ptr, const int32_t* succ,
                             const float* delay, const float* arr0, float* arr, uint64_t spin_limit_ns,
                             void* stream);

/* --- memory and diagnostics ------------------------------------------------------------ */

/* Process-wide device allocator for library-owned buffers (NULL, NULL = cudaMalloc/cudaFree).
 * alloc(bytes, stream, ctx) returns a device pointer aligned to 256 bytes or NULL. */
typedef void* (*hf_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*hf_free_fn)(void* ptr, void* stream, void* ctx);
hf_status hf_set_allocator(hf_alloc_fn alloc, hf_free_fn free_fn, void* ctx);

const char* hf_status_string(hf_status s);
/* Message of the last failure on the calling thread ("" if none). */
const char* hf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HF_H */
