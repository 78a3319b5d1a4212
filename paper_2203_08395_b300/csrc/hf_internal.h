// hf_internal.h -- internal data structures of the task-graph executor (host builder,
// device plan, kernels). Not part of the C ABI; see include/hf.h for the public contract.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/hf.h"

namespace hf {

// ----------------------------------------------------------------------------- constants

// Order-preserving map from FP32 bits to uint32 (radix-sort key): negative values have all
// bits flipped, non-negative ones get the sign bit set; then unsigned comparison of keys
// equals the total order -inf < ... < -0 < +0 < ... < +inf on non-NaN floats.
constexpr uint32_t kKeyNegInf = 0x007FFFFFu;  // key(-inf)
constexpr uint32_t kKeyPosZero = 0x80000000u;  // key(+0)

// kPayHost: a host task (a_bits: its index in the plan's host-task list). The persistent
// executor's warp posts it to the host proxy and waits for it; the level-synchronous and team
// executors run host tasks their own way and skip the piece.
enum PayOp : uint32_t { kPaySaxpyF32 = 1, kPaySaxpyI32 = 2, kPayCopy = 3, kPayHost = 4 };

// One device payload record (saxpy or copy), 64 bytes. It also carries its task's id and row so
// that a warp holding only the payload index has everything it needs after one load.
struct DevPayload {
    void* dst;            // saxpy: y; copy: destination
    const void* src;      // saxpy: x; copy: source
    int64_t n;            // saxpy: elements; copy: bytes
    uint32_t op;          // PayOp
    uint32_t a_bits;      // saxpy scalar (float bits or int32)
    int32_t nchunks;      // pieces the payload is split into (>= 1)
    int32_t chunk_first;  // first piece-item index (multi-piece payloads), else -1
    int64_t chunk;        // piece size: elements (saxpy) or bytes (copy)
    int32_t task;         // the task carrying this payload
    int32_t row;          // its first out-edge
    int32_t deg;          // its out-degree
    int32_t pad_;
};

// Persistent-executor control block; hot counters on separate 128-byte lines.
struct alignas(128) Ctrl {
    int32_t head;
    int32_t pad0[31];
    int32_t tail;
    int32_t pad1[31];
    uint32_t done;
    int32_t pad2[31];
    int32_t status;
    int32_t abort;
    int32_t bad_input;  // set by hf_set_delays' kernel when a delay is not finite
    int32_t pad3[29];
    unsigned long long ticket;  // validation tickets
    int32_t pad4[30];
    int32_t phead;  // payload queue (warp-specialised runs)
    int32_t pad5[31];
    int32_t ptail;
    int32_t pad6[31];
    int32_t lhead0;  // copy queues (runs with copy warps): pull copies ...
    int32_t pad7[31];
    int32_t ltail0;
    int32_t pad8[31];
    int32_t lhead1;  // ... and push copies
    int32_t pad9[31];
    int32_t ltail1;
    int32_t pad10[31];
};

// Arguments of the persistent executor kernel (by value, < 4 KB).
struct PersistArgs {
    int32_t n_tasks;
    int32_t qcap;
    int32_t claim;
    int32_t local_keep;
    uint64_t spin_limit_ns;
    const int2* meta;        // n_tasks {first out-edge, out-degree}
    const int4* erec;        // out-edges, CSR order: {successor, delay bits, successor's first
                             // out-edge, successor's out-degree << 16 | in-degree (or marks)}
    const int32_t* pidx;     // n_tasks payload index or -1 (NULL: no payloads)
    const DevPayload* pay;
    const int32_t* chunk_pay;   // piece item -> payload index
    int32_t npieces;            // piece items (queue items n .. n+npieces-1; payload starts follow)
    int32_t ring_mask;          // work stealing: slots per CTA ring - 1 (a power of two minus one)
    unsigned long long* state;  // n_tasks {key << 32 | pending predecessors}
    uint32_t* key;              // n_tasks final arrival keys (output)
    int32_t* queue;             // qcap ready-queue slots (-1 = empty)
    int32_t* pqueue;            // pqcap payload-queue slots (used when pay_warps > 0)
    int32_t pqcap;
    int32_t pay_warps;          // warps per CTA that only run payload tasks (0: none)
    int32_t* chunks_left;       // per payload: pieces still running
    Ctrl* ctrl;
    int64_t* t_start;  // instrument: %globaltimer per task (NULL otherwise)
    int64_t* t_end;
    int64_t* tk_start;  // validate: tickets per task (NULL otherwise)
    int64_t* tk_end;
    int32_t* exec_count;
    unsigned long long* stats;  // instrument & 2: executor counters (kStat*), else NULL
    int32_t* post;              // host tasks: mapped mailbox (the i-th posted host task), else NULL
    const int32_t* hdone;       // mapped: host task k has run
    int32_t* post_ctr;          // device counter of posts
    // work stealing (NULL: the global queue alone): CTA c owns ring[c * (ring_mask + 1) ...],
    // cells {position + 1 << 32 | item} (0: never written), and ring_head[c * 32], the next
    // position to take; positions count from 0 in every run
    unsigned long long* ring;
    int32_t* ring_head;
    // copy warps (pdir NULL: none): per payload 0 (not a copy), 1 (pull: host to device) or 2
    // (push: device to host); copies of direction d + 1 go to queue lqueue_d, served by the
    // copy_warps warps of each CTA given to that direction
    const uint8_t* pdir;
    int32_t* lqueue0;
    int32_t* lqueue1;
    int32_t lqcap;
    int32_t copy_warps;
};

// Executor counters recorded by runs with instrument & 2 (hf_get_stats).
enum StatIdx {
    kStatRounds = 0,     // warp rounds that had work
    kStatItems,          // items processed (tasks and payload pieces)
    kStatIdle,           // idle polls
    kStatEdges,          // successor releases
    kStatCas,            // compare-and-swap attempts
    kStatPushLocal,      // ready tasks kept in a warp's stack
    kStatPushGlobal,     // items pushed to the global queue
    kStatClaims,         // claims on the global queue
    kStatPops,           // items taken from the global queue
    kStatPieces,         // payload pieces run
    kStatCycRound,       // SM cycles in rounds with work (from items in hand to round end)
    kStatCycRelease,     // ... of which releasing successors (pushes included)
    kStatCycCas,         // ... of which the compare-and-swap sections
    kStatCycPush,        // ... of which pushing ready tasks
    kStatRingPush,       // work stealing: items pushed to the CTA's own ring
    kStatSteals,         // work stealing: items taken from another CTA's ring
    kStatCount = 16
};

// Successors with more than this many predecessors are released with a max on the key half
// and a fenced decrement of the count half instead of one CAS on the packed state.
constexpr int32_t kNarrowIn = 64;

// Arguments of the reset kernel run before each persistent launch.
struct ResetArgs {
    int32_t n_tasks;
    int32_t qcap;
    int32_t n_seed;
    int32_t n_pay;
    int32_t stall_task;  // test hook: this task's counter starts one too high (-1: none)
    int32_t keep_status; // leave ctrl->status as the previous run left it
    int32_t n_pseed;     // payload seed items
    int32_t pqcap;
    int32_t split;       // payload seeds go to the payload queue (else to the main queue)
    const int32_t* indeg0;
    const uint32_t* key0;  // NULL: sources start at +0
    const int32_t* seeds;   // items of sources without payload
    const int32_t* pseeds;  // items of sources with a payload
    int32_t* pqueue;
    const DevPayload* pay;
    unsigned long long* state;
    int32_t* queue;
    int32_t* chunks_left;
    Ctrl* ctrl;
    int64_t* t_start;
    int64_t* t_end;
    int64_t* tk_start;
    int64_t* tk_end;
    int32_t* exec_count;
    unsigned long long* ring;  // work stealing: ring cells cleared (ring_cells of them), else NULL
    int64_t ring_cells;
    int32_t* ring_head;        // ring_heads counters cleared
    int32_t ring_heads;
    // payload seeds are pseeds[0, n_pseed) (no copy), then pull copies [n_pseed, + n_cseed0),
    // then push copies [.., + n_cseed1); with copy warps (link) the copies seed lqueue0/1
    int32_t n_cseed0, n_cseed1;
    int32_t link;
    int32_t lqcap;
    int32_t* lqueue0;
    int32_t* lqueue1;
};

// Team executor: a job is one graph, run by one CTA (solo job) or by the CTAs of one thread-block
// cluster (cluster job; jobs [0, ncjobs) of the list).
// TeamJob::flags: the graph's keys live in the team's shared memory (TeamArgs::key_cap); its
// levels are software-pipelined (each thread reads its next level's task while the current
// level's key loads are in flight: pays where the keys come from L2, not where they fit in L1)
constexpr int32_t kJobSharedKeys = 1;
constexpr int32_t kJobPipelined = 2;
// kJobPayloadLocal: no payload task of the graph touches memory another one writes (checked on
// the host from the payloads' address ranges; graphs with host tasks never qualify), so no task
// of the graph can observe another's payload data: a cluster level then releases only its
// arrival keys (an explicit cluster fence by the threads that stored them) and the level's
// cluster barrier need not wait for the payload stores to be acknowledged
constexpr int32_t kJobPayloadLocal = 4;
// graphs of at least this many tasks run pipelined (their keys outgrow an SM's L1)
constexpr int32_t kPipeMinTasks = 32768;

struct TeamJob {
    int32_t graph;
    int32_t flags;   // kJobSharedKeys | kJobPipelined
    int32_t seg0;    // first (graph, level) segment of the graph
    int32_t levels;  // levels of the graph
};

// One payload piece resolved for the team executor (built on the host per piece size, staged in
// shared memory with its level): pointers already offset to the piece, cnt in elements (saxpy)
// or bytes (copy), op 0 = none. 32 bytes.
struct alignas(16) TeamPiece {
    char* dst;
    const char* src;
    int32_t cnt;
    uint32_t a;
    uint32_t op;
    int32_t task;  // the task the piece belongs to (cost recording)
};

// Team-executor control words (zeroed before every run): solo-job counter, cluster-job counter.
constexpr int kTeamNext = 0;
constexpr int kTeamNextC = 32;
constexpr int kTeamWords = 64;

// Arguments of the team executor kernel.
struct TeamArgs {
    const int32_t* ls_node;  // merged level-sorted order (as the level-synchronous executor)
    const int32_t* ls_ptr;
    const int2* ls_in;
    const uint32_t* key0;
    uint32_t* key;
    const DevPayload* pay;
    const int2* items;       // payload work items {payload index, piece index}
    const int4* seg;         // (graph, level) segment -> {p0, p1, e0, e1}
    const int2* seg_items;   // (graph, level) segment -> payload items {i0, i1}
    const TeamJob* jobs;     // cluster jobs first, then solo jobs
    int32_t njobs;
    int32_t ncjobs;
    int32_t stage_n;         // stage buffer capacity: tasks and in-edges of a level
    int32_t stage_e;
    int32_t stage_p;         // ... and payload piece descriptors (0: none staged)
    int32_t key_cap;         // key table entries per CTA in shared memory (0: none; see TeamJob)
    const TeamPiece* pdesc;  // piece descriptors, in item order
    int32_t* team;           // control words (kTeam*)
    Ctrl* ctrl;              // status word (HF_ETIMEDOUT when a staged copy never lands)
    uint64_t spin_limit_ns;
    int64_t* g_start;        // instrument: %globaltimer per graph at job start / end (else NULL)
    int64_t* g_end;
    float* t_cost;           // instrument bit 2: per-task cost in ns (a task's gather; a payload task's
                             // pieces summed), else NULL
    const int2* seg_host;    // host tasks: (graph, level) segment -> range in host_order (NULL: none)
    const int32_t* host_order;
    int32_t* post;           // mapped host memory: the i-th posted host task
    const int32_t* hdone;    // mapped host memory: host task k has run
    int32_t* post_ctr;       // device counter of posts
    const int32_t* task_off; // first task id of each graph (ngraphs + 1)
};

// Arguments of one level kernel of the level-synchronous executor.
struct LevelArgs {
    const int32_t* ls_node;  // level-sorted position -> task id
    const int32_t* ls_ptr;   // level-sorted position -> first in-edge (n + 1)
    const int2* ls_in;       // in-edges {predecessor, delay bits}, level-sorted order
    const uint32_t* key0;    // NULL: sources start at +0
    uint32_t* key;
    const DevPayload* pay;
    const int2* items;       // payload work items {payload index, piece index}
    int32_t p0, p1;          // positions of this level
    int32_t i0, i1;          // payload items of this level
    int32_t nb_mp;           // blocks doing arrivals; the rest do payload items
    int32_t pad_;
};

// ----------------------------------------------------------------------------- host side

struct PayloadRec {
    int32_t kind = 0;  // hf_kind
    int32_t op = 0;    // hf_kernel_op for kernels
    // saxpy
    int64_t n = 0;
    float a_f = 0.f;
    int32_t a_i = 0;
    int32_t x_pull = -1, y_pull = -1;
    void* x_dev = nullptr;
    void* y_dev = nullptr;
    // pull / push
    const void* host_src = nullptr;
    void* host_dst = nullptr;
    size_t bytes = 0;
    int32_t src_pull = -1;
    const void* src_dev = nullptr;
    // host
    void (*fn)(void*) = nullptr;
    void* arg = nullptr;
};

// Finalized host form of one graph.
struct Final {
    int32_t n = 0;
    int64_t m = 0;
    int32_t levels = 0;
    int32_t nsrc = 0;
    std::vector<int32_t> row_ptr;   // n + 1 (successor CSR, edges in insertion order)
    std::vector<int2> succ;         // m
    std::vector<int32_t> indeg0;    // n
    std::vector<int32_t> level;     // n
    std::vector<int32_t> ls_node;   // n: tasks sorted by (level, id)
    std::vector<int32_t> level_ptr; // levels + 1
    std::vector<int32_t> ls_ptr;    // n + 1
    std::vector<int2> ls_in;        // m
    std::vector<int32_t> epos_csr;  // m: edge (insertion order) -> position in succ
    std::vector<int32_t> epos_ls;   // m: edge (insertion order) -> position in ls_in
};

struct Plan;  // device-resident form of one or more graphs (plan.cu)

}  // namespace hf

struct hf_graph {
    std::vector<uint8_t> kind;     // hf_kind
    std::vector<float> arr0;
    std::vector<int32_t> pay;      // payload index or -1
    std::vector<hf::PayloadRec> payloads;
    std::vector<int32_t> esrc, edst;
    std::vector<float> edly;
    bool dirty = true;
    bool any_arr0 = false;
    int in_batches = 0;
    hf::Final fin;
    hf::Plan* plan = nullptr;  // solo-run plan
};

struct hf_batch {
    std::vector<hf_graph*> graphs;
    hf::Plan* plan = nullptr;
    bool dirty = true;
    hf_costmodel* cm = nullptr;  // borrowed
};

namespace hf {

// error reporting (api.cpp)
hf_status fail(hf_status s, const std::string& msg);
hf_status cuda_fail(cudaError_t e, const char* what);

// device memory through the installed allocator (api.cpp)
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// plan.cu
hf_status plan_build(const std::vector<hf_graph*>& graphs, Plan** out);
void plan_destroy(Plan* p);
// keep_status: a later run of a sequence (hf_run_n) keeps the device status word of the runs
// before it, so the sequence reports its first failure
// io_dly (page-locked host memory, or NULL): the run first takes its edge delays from it (copied
// on the plan's input stream); io_arr (page-locked host memory, or NULL): every arrival is copied
// there after the run, on the plan's output stream (see hf_batch_run_host).
hf_status plan_run(Plan* p, cudaStream_t s, const hf_run_opts& o, bool keep_status = false,
                   const float* io_dly = nullptr, float* io_arr = nullptr);
hf_status plan_sync(Plan* p);
hf_status plan_busy(Plan* p);  // HF_ESTATE while a run is in flight
hf_status plan_get_arrivals(Plan* p, int32_t gi, float* out, int on_device);
hf_status plan_get_times(Plan* p, int32_t gi, int64_t* a, int64_t* b);
hf_status plan_get_stamps(Plan* p, int32_t gi, int64_t* a, int64_t* b, int32_t* c);
hf_status plan_kernel_ms(Plan* p, float* ms);
hf_status plan_get_stats(Plan* p, int64_t* out, int32_t n);
hf_status plan_get_graph_times(Plan* p, int64_t* start, int64_t* end);
hf_status plan_last_launches(Plan* p, int32_t* n);
hf_status plan_get_task_costs(Plan* p, int32_t gi, float* out);
hf_status plan_team_plan(Plan* p, int32_t* team_size);
hf_status plan_team_keys(Plan* p, int32_t* shared);
hf_status plan_team_flags(Plan* p, int32_t* flags);
hf_status plan_set_delays(Plan* p, const float* delay, int on_device, cudaStream_t s);
hf_status plan_run_host(Plan* p, cudaStream_t s, const hf_run_opts& o, const float* delay, float* arr_out);
hf_status plan_features(Plan* p, float* X, cudaStream_t s);
hf_status plan_task_costs(Plan* p, int32_t priority, const hf_costmodel* cm, float* cost, float* bottom,
                          cudaStream_t s);
hf_status plan_refresh_priorities(Plan* p, const hf_costmodel* cm, cudaStream_t s);
void plan_set_costmodel(Plan* p, const hf_costmodel* cm);
hf_status plan_bottom_levels(Plan* p, const float* cost, float* bottom, cudaStream_t s);
hf_status plan_autotune(Plan* p, cudaStream_t s, const hf_run_opts& base, int force, hf_run_opts* best,
                        float* best_ms);
hf_status plan_calibration(cudaStream_t s, float* out);
hf_status plan_predict(Plan* p, int32_t priority, const hf_costmodel* cm, cudaStream_t s, float* ls_ms,
                       float* p_ms, float* t_ms);

// costmodel.cu
hf_status mlp_forward(const float* params, const float* X, int64_t n, float* y, cudaStream_t s);
const float* costmodel_params(const hf_costmodel* cm);

}  // namespace hf
