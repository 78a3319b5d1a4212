// plan.cu -- device-resident execution plans and the two executors' launch logic.
//
// A plan is one or more finalized graphs concatenated with task/edge offsets (a batch of
// independent DAGs runs in one persistent launch, or level by level with all graphs' level l
// merged into one kernel). It owns every device buffer the graphs need: successor CSR,
// level-sorted predecessor lists, payload table, pull buffers, arrival keys, in-degree
// counters, the ready queue and the control block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <queue>
#include <string>
#include <tuple>
#include <vector>

#include "hf_internal.h"
#include "kernels.cuh"
#include "team.cuh"

namespace hf {

struct HostTask {
    int32_t level;
    void (*fn)(void*);
    void* arg;
    int32_t graph;  // batch index of its graph
};

struct Plan {
    int32_t ngraphs = 0;
    std::vector<int32_t> task_off;  // ngraphs + 1
    int32_t n = 0;
    int64_t m = 0;
    int32_t levels = 0;
    int32_t npay = 0;
    bool any_key0 = false;
    std::vector<HostTask> host_tasks;

    // host copies needed when the piece size changes
    std::vector<DevPayload> hpay;   // payload table (task-ordered by creation)
    std::vector<int32_t> pay_task;  // payload -> task
    std::vector<int32_t> pay_level; // payload -> level
    std::vector<uint8_t> pay_local; // graph -> 1: no payload touches memory another payload writes
    std::vector<int32_t> hpidx;     // task -> payload or -1
    std::vector<uint8_t> hpdir;     // payload -> 0, or 1 for a pull copy, 2 for a push copy
    std::vector<int32_t> pay_succ_level;  // payload -> its task's successors' lowest level (-1: none)
    int32_t ncopy[2] = {0, 0};      // pull copies, push copies
    // the level-synchronous executor's copy nodes: one per pull / push task with bytes, run by
    // the copy engines, after the level before the task's and before its first successor's level
    struct CopyNode {
        void* dst;
        const void* src;
        size_t bytes;
        int32_t level;       // the task's level
        int32_t succ_level;  // its successors' lowest level (-1: none)
        bool pull;           // host to device (else device to host)
    };
    std::vector<CopyNode> copies;
    std::vector<int32_t> sources;   // task ids with no predecessor
    std::vector<int32_t> level_ptr; // merged level-sorted positions (levels + 1)
    // team executor
    std::vector<int4> h_seg;          // (graph, level) segment -> {p0, p1, e0, e1}
    std::vector<int32_t> seg_first;   // graph -> first segment (ngraphs + 1)
    std::vector<int32_t> glevels;     // graph -> levels
    std::vector<int32_t> team_k;      // graph -> team size of the current team plan (0: no levels)
    int4* d_seg = nullptr;
    int2* d_seg_items = nullptr;      // segment -> payload items {i0, i1} (per piece size)
    size_t cap_seg_items = 0;
    TeamJob* d_jobs = nullptr;
    size_t cap_jobs = 0;
    int32_t njobs = 0;
    struct TeamClass {
        int32_t k;       // cluster size of the class's launch (1: single CTAs)
        int32_t job0;    // its jobs in d_jobs
        int32_t njobs;
        int32_t ncjobs;  // of which cluster jobs (first; the rest are single-CTA jobs)
        int32_t grid;    // CTAs launched
        int32_t key_cap; // key table entries per CTA in shared memory (0: keys in global memory)
        int32_t csk;     // 1: every graph of the class keeps its keys there (the k_team<., ., true> kernel)
    };
    std::vector<TeamClass> tclass;    // one launch per class, chained (plan_run), run concurrently
    // the classes' stream (tstream[0]) at the device's highest stream priority: pending team
    // CTAs are dispatched before those of the plan's helper kernels (the next view's delay gather)
    cudaStream_t tstream[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t tev_fork = nullptr;
    cudaEvent_t tev_join[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t* d_team = nullptr;        // control words (job counters), kTeamWords per class
    int32_t stage_n = 4, stage_e = 2;  // stage buffer capacities (tasks, in-edges per level)
    int32_t stage_p = 0;               // ... piece descriptors per level (per piece size)
    TeamPiece* d_pdesc = nullptr;      // piece descriptors in item order (per piece size)
    size_t cap_pdesc = 0;
    // team executor's host tasks: a mailbox in mapped page-locked memory and a proxy thread
    int2* d_seg_host = nullptr;       // (graph, level) segment -> host-task range in host_order
    int32_t* d_host_order = nullptr;  // host-task indices grouped by segment
    int32_t* h_post = nullptr;        // mapped: the i-th posted host task (-1: not yet)
    int32_t* h_hdone = nullptr;       // mapped: 1 once host task k has run
    int32_t* d_post = nullptr;        // device views of the two
    int32_t* d_hdone = nullptr;
    int32_t* d_post_ctr = nullptr;    // posts so far (device counter)
    std::thread proxy;                // runs the host tasks of the current run
    // priority, team_size, CTAs, scale, fold, global keys the jobs were built for
    int32_t team_for[6] = {-1, -1, -1, -1, -2, -1};
    std::vector<int32_t> team_sk;  // per graph: 1 when its keys live in shared memory (last team plan)
    const hf_costmodel* team_cm = nullptr;

    // device buffers
    std::vector<void*> owned;
    int32_t* d_row_ptr = nullptr;
    int4* d_erec = nullptr;  // successor edge records (persistent executor)
    int2* d_meta = nullptr;  // {first out-edge, out-degree} per task
    unsigned long long* d_state = nullptr;
    int32_t* d_indeg0 = nullptr;
    uint32_t* d_key0 = nullptr;
    int32_t* d_pidx = nullptr;
    DevPayload* d_pay = nullptr;
    int32_t* d_ls_node = nullptr;
    int32_t* d_ls_ptr = nullptr;
    int2* d_ls_in = nullptr;
    uint32_t* d_key = nullptr;
    int32_t* d_chunks_left = nullptr;
    Ctrl* d_ctrl = nullptr;
    float* d_arr = nullptr;  // conversion buffer for on_device = 0 reads
    // piece-size dependent
    int64_t chunk_elems = -1;
    int32_t nitems = 0;               // total pieces of multi-piece payloads
    int32_t qcap = 0;
    int32_t nseed = 0;
    int32_t* d_chunk_task = nullptr;  // sized for nitems
    int32_t* d_seeds = nullptr;
    int32_t* d_pseeds = nullptr;  // items of sources with a payload: non-copies, pull copies, push copies
    int32_t ncseed[2] = {0, 0};   // ... of which pull copies, push copies
    uint8_t* d_pdir = nullptr;    // hpdir on the device (plans with copies)
    int32_t* d_lqueue[2] = {nullptr, nullptr};  // copy queues (persistent runs with copy warps)
    size_t cap_lqueue = 0;
    int32_t* d_pqueue = nullptr;  // payload queue (warp-specialised runs)
    int32_t npseed = 0, pqcap = 0;
    int32_t* d_queue = nullptr;
    int2* d_items = nullptr;          // level-sync payload items
    std::vector<int32_t> item_ptr;    // levels + 1
    size_t cap_chunk_task = 0, cap_seeds = 0, cap_queue = 0, cap_items = 0, cap_pseeds = 0, cap_pqueue = 0;
    // instrumentation
    int64_t* d_t_start = nullptr;
    int64_t* d_t_end = nullptr;
    int64_t* d_tk_start = nullptr;
    int64_t* d_tk_end = nullptr;
    int32_t* d_exec = nullptr;
    unsigned long long* d_stats = nullptr;  // executor counters (instrument & 2)
    unsigned long long* d_ring = nullptr;   // work stealing: per-CTA rings of ready tasks
    int32_t* d_ring_head = nullptr;         // their take positions (one 128-byte line per CTA)
    size_t cap_ring = 0, cap_ring_head = 0;
    int64_t* d_gtime = nullptr;             // team executor: per-graph start, then end (instrument & 1)
    float* d_tcost = nullptr;               // team executor: per-task cost in ns (instrument & 4)
    bool last_tcost = false;
    int32_t last_launches = 0;              // executor kernels of the last run
    bool last_gtimes = false;
    bool last_stats = false;
    bool last_instrument = false, last_validate = false;
    // level-sync CUDA graph
    cudaGraph_t lgraph = nullptr;
    cudaGraphExec_t lexec = nullptr;
    std::vector<LevelArgs> largs;
    // host-buffer runs: a second level-sorted in-edge buffer (and its level graph); the next
    // view's delays are gathered into it while a run reads d_ls_in, then the two swap
    int2* d_ls_in_alt = nullptr;
    cudaGraph_t lgraph_alt = nullptr;
    cudaGraphExec_t lexec_alt = nullptr;
    std::vector<LevelArgs> largs_alt;
    int lsb = 0;                      // which of the two buffers d_ls_in is (0: the original)
    cudaEvent_t ev_buf[2] = {nullptr, nullptr};  // after the last run that read buffer b
    bool buf_used[2] = {false, false};
    int32_t* d_bad2 = nullptr;        // per buffer: a gathered delay was not finite
    // runtime
    int num_sms = 0;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaEvent_t kev0 = nullptr, kev1 = nullptr;  // time_kernel runs
    bool last_timed = false;
    int32_t* d_epos_csr = nullptr;  // edge -> succ position (m)
    int32_t* d_epos_ls = nullptr;   // edge -> ls_in position (m)
    float* d_dly_stage = nullptr;   // host delays staged on the device (m)
    bool ran = false;
    int32_t* h_status = nullptr;  // page-locked mirror of ctrl->status
    // cost model inputs and outputs (built on first use)
    std::vector<int32_t> h_level;  // task -> level within its graph
    std::vector<uint8_t> h_cat;    // task -> 0 max-plus, 1 saxpy, 2 pull, 3 push, 4 host
    std::vector<float4> h_gstat;   // graph -> {tasks, edges, levels, 0}
    int32_t* d_level = nullptr;
    uint8_t* d_cat = nullptr;
    int32_t* d_toff = nullptr;
    // host-buffer runs (hf_run_host): the arrivals go to the host from d_arr on a stream of the
    // plan's own, overlapping the caller's next work; d_arr is reused only after that copy.
    // New delays come in by copy engine on another plan stream into d_hstage (waiting only until
    // the previous view's gather has read it), then a gather puts them in ls_in. The level-sync
    // and team executors alternate two staging buffers with the copies on a stream of their own
    // (hstream), so that the next view's copy starts as soon as the copy engine is free.
    cudaStream_t cstream = nullptr, istream = nullptr, hstream = nullptr;
    cudaEvent_t ev_conv = nullptr, ev_d2h = nullptr, ev_h2d = nullptr, ev_gather = nullptr;
    bool d2h_pending = false, gather_pending = false;
    float* d_hstage = nullptr;      // host-buffer delays on the device (m)
    float* d_hstage2 = nullptr;     // the second staging buffer (level-sync and team)
    cudaEvent_t ev_hcopy[2] = {nullptr, nullptr};  // staging buffer j: its copy landed
    cudaEvent_t ev_hread[2] = {nullptr, nullptr};  // staging buffer j: last read by a gather/scatter
    bool hread_pending[2] = {false, false};
    int hsb = 0;                    // staging buffer the next level-sync/team upload fills
    int32_t* d_ls_edge = nullptr;   // in-edge position -> edge in insertion order (m)
    bool erec_stale = false;        // erec's delays older than ls_in's (refreshed before a persistent run)
    float4* d_gstat = nullptr;
    float* d_prio = nullptr;       // bottom-level weight per task under seed_prio
    int32_t seed_prio = HF_PRIO_FIFO;  // priority the seed order was built for
    const hf_costmodel* cm = nullptr;  // borrowed from the batch
    int32_t auto_mode = -1;            // executor chosen by HF_MODE_AUTO (-1: not yet predicted)
    const hf_costmodel* auto_cm = nullptr;
    int32_t auto_ctas = 0;             // CTA count the persistent prediction assumed
};

hf_status plan_auto_mode(Plan* p, cudaStream_t s, int* mode);

static hf_status plan_set_chunk(Plan* p, int64_t chunk_elems, cudaStream_t s);
static hf_status plan_team_jobs(Plan* p, const hf_run_opts& o, cudaStream_t s);
// default payload-cost scale: a 512-element piece takes ~0.75 us for a warp alone and ~3 us when
// every SM streams (measured on this B300), so concurrent graphs see about 4x the unloaded cost
constexpr int kTeamScaleDefault = 4;
// Learned costs are recorded by the team executor under its real load (contention included), so
// the planner takes them as they are.
static int team_scale_default(int32_t prio) { return prio == HF_PRIO_LEARNED ? 1 : kTeamScaleDefault; }
// hf_run_opts::team_scale as a factor: s > 0 is s, s < 0 is 1 / -s, 0 is the default
static double team_scale_factor(int32_t s, int32_t prio) {
    if (s == 0) s = team_scale_default(prio);
    return s > 0 ? (double)s : 1.0 / (double)(-s);
}
static int team_capacity(const Plan* p, int k, size_t smem = 0, bool csk = false);
static const void* team_kernel(bool pay, bool rec, bool csk);
static size_t team_smem(const Plan* p);
static size_t team_class_smem(const Plan* p, int32_t key_cap);
static void team_smem_attr(const Plan* p, size_t need = 0);
static hf_status team_decide(Plan* p, int32_t prio, int32_t ctas_opt, double scale, cudaStream_t s,
                             std::vector<int>* k_out, std::vector<int32_t>* order_out, double* M_out, int fold_k = 0);
hf_status plan_prepare_priority(Plan* p, int32_t priority, const hf_costmodel* cm, cudaStream_t s);

void plan_set_costmodel(Plan* p, const hf_costmodel* cm) {
    p->cm = cm;
    if (p->seed_prio == HF_PRIO_LEARNED) p->seed_prio = -1;  // recompute with the new model
}

static void* palloc(Plan* p, size_t bytes, cudaStream_t s) {
    void* d = dev_alloc(bytes, s);
    if (d) p->owned.push_back(d);
    return d;
}

// slack: extra bytes after the data (the team executor's bulk copies round ends up to 16 bytes)
template <typename T>
static hf_status upload(Plan* p, T** dst, const T* src, size_t count, cudaStream_t s, const char* what,
                        size_t slack = 0) {
    *dst = (T*)palloc(p, std::max<size_t>(count * sizeof(T) + slack, 16), s);
    if (!*dst) return fail(HF_ENOMEM, std::string("device allocation failed: ") + what);
    if (count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return HF_OK;
}

static void free_owned(Plan* p, void* ptr) {
    if (!ptr) return;
    auto it = std::find(p->owned.begin(), p->owned.end(), ptr);
    if (it != p->owned.end()) p->owned.erase(it);
    dev_free(ptr, nullptr);
}

// Device-visible address of page-locked host memory (NULL if `ptr` is not page-locked or not
// mapped for the device): kernels reach pull sources and push targets through it.
static void* host_dev_ptr(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost) return nullptr;
    return at.devicePointer;
}

static uint32_t host_f2key(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

void plan_destroy(Plan* p) {
    if (!p) return;
    if (p->ran && p->done_ev) cudaEventSynchronize(p->done_ev);
    if (p->d2h_pending) cudaEventSynchronize(p->ev_d2h);
    if (p->gather_pending) cudaEventSynchronize(p->ev_h2d);
    if (p->proxy.joinable()) p->proxy.join();
    if (p->h_post) cudaFreeHost(p->h_post);
    if (p->h_hdone) cudaFreeHost(p->h_hdone);
    if (p->istream) cudaStreamSynchronize(p->istream);
    if (p->hstream) cudaStreamSynchronize(p->hstream);
    if (p->lexec) cudaGraphExecDestroy(p->lexec);
    if (p->lgraph) cudaGraphDestroy(p->lgraph);
    if (p->lexec_alt) cudaGraphExecDestroy(p->lexec_alt);
    if (p->lgraph_alt) cudaGraphDestroy(p->lgraph_alt);
    for (int i = 0; i < 2; ++i)
        if (p->ev_buf[i]) cudaEventDestroy(p->ev_buf[i]);
    for (void* d : p->owned) dev_free(d, nullptr);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    if (p->kev0) cudaEventDestroy(p->kev0);
    if (p->kev1) cudaEventDestroy(p->kev1);
    for (int i = 0; i < 5; ++i) {
        if (p->tstream[i]) cudaStreamDestroy(p->tstream[i]);
        if (p->tev_join[i]) cudaEventDestroy(p->tev_join[i]);
    }
    if (p->tev_fork) cudaEventDestroy(p->tev_fork);
    if (p->cstream) cudaStreamDestroy(p->cstream);
    if (p->istream) cudaStreamDestroy(p->istream);
    if (p->hstream) cudaStreamDestroy(p->hstream);
    for (int i = 0; i < 2; ++i) {
        if (p->ev_hcopy[i]) cudaEventDestroy(p->ev_hcopy[i]);
        if (p->ev_hread[i]) cudaEventDestroy(p->ev_hread[i]);
    }
    if (p->ev_conv) cudaEventDestroy(p->ev_conv);
    if (p->ev_d2h) cudaEventDestroy(p->ev_d2h);
    if (p->ev_h2d) cudaEventDestroy(p->ev_h2d);
    if (p->ev_gather) cudaEventDestroy(p->ev_gather);
    delete p;
}

hf_status plan_build(const std::vector<hf_graph*>& graphs, Plan** out) {
    *out = nullptr;
    Plan* p = new (std::nothrow) Plan();
    if (!p) return fail(HF_ENOMEM, "host allocation failed");
    cudaStream_t s = nullptr;
    hf_status st = HF_OK;
    auto bail = [&](hf_status e) {
        plan_destroy(p);
        return e;
    };
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaGetDevice"));
    ce = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaDeviceGetAttribute"));
    ce = cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaEventCreate"));
    ce = cudaEventCreate(&p->kev0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&p->kev1);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaEventCreate"));
    ce = cudaHostAlloc((void**)&p->h_status, 64, cudaHostAllocDefault);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaHostAlloc"));
    std::memset(p->h_status, 0, 64);

    p->ngraphs = (int32_t)graphs.size();
    p->task_off.assign((size_t)p->ngraphs + 1, 0);
    int64_t ntot = 0, mtot = 0;
    for (int i = 0; i < p->ngraphs; ++i) {
        const hf_graph* g = graphs[(size_t)i];
        if (g->dirty) return bail(fail(HF_ESTATE, "graph not finalized"));
        ntot += g->fin.n;
        mtot += g->fin.m;
        p->levels = std::max(p->levels, g->fin.levels);
        if (g->any_arr0) p->any_key0 = true;
        if (ntot > INT32_MAX - 1 || mtot > INT32_MAX) return bail(fail(HF_EINVAL, "batch too large for 32-bit ids"));
        p->task_off[(size_t)i + 1] = (int32_t)ntot;
    }
    p->n = (int32_t)ntot;
    p->m = mtot;
    const int32_t n = p->n;

    try {
        // successor CSR, in-degrees, sources, source arrival keys
        std::vector<int32_t> row_ptr((size_t)n + 1);
        std::vector<int2> succ((size_t)p->m);
        std::vector<int32_t> indeg0((size_t)n);
        std::vector<int32_t> epos_csr((size_t)p->m), epos_ls((size_t)p->m);
        std::vector<uint32_t> key0;
        if (p->any_key0) key0.resize((size_t)n);
        int64_t eoff = 0;
        for (int i = 0; i < p->ngraphs; ++i) {
            const hf_graph* g = graphs[(size_t)i];
            const Final& f = g->fin;
            const int32_t toff = p->task_off[(size_t)i];
            for (int32_t v = 0; v < f.n; ++v) {
                row_ptr[(size_t)toff + v] = (int32_t)(eoff + f.row_ptr[v]);
                indeg0[(size_t)toff + v] = f.indeg0[v];
                if (f.indeg0[v] == 0) p->sources.push_back(toff + v);
                if (p->any_key0) key0[(size_t)toff + v] = host_f2key(g->arr0[v]);
            }
            for (int64_t e = 0; e < f.m; ++e) {
                int2 x = f.succ[(size_t)e];
                x.x += toff;
                succ[(size_t)(eoff + e)] = x;
                epos_csr[(size_t)(eoff + e)] = (int32_t)(eoff + f.epos_csr[(size_t)e]);
            }
            eoff += f.m;
        }
        row_ptr[(size_t)n] = (int32_t)eoff;
        // edge records and per-task rows for the persistent executor
        std::vector<int4> erec((size_t)p->m);
        std::vector<int2> meta((size_t)n);
        for (int32_t v = 0; v < n; ++v) meta[(size_t)v] = make_int2(row_ptr[(size_t)v], row_ptr[(size_t)v + 1] - row_ptr[(size_t)v]);
        for (int64_t e = 0; e < p->m; ++e) {
            const int32_t w = succ[(size_t)e].x;
            const uint32_t len = (uint32_t)meta[(size_t)w].y;
            const uint32_t in = (uint32_t)indeg0[(size_t)w];
            const uint32_t lo = in <= (uint32_t)kNarrowIn ? in : kWideMark;
            const uint32_t hi = len < kLongMark ? len : kLongMark;
            erec[(size_t)e] = make_int4(w, succ[(size_t)e].y, meta[(size_t)w].x, (int)((hi << 16) | lo));
        }
        // merged level-sorted order: level l of graph 0, level l of graph 1, ...
        std::vector<int32_t> ls_node((size_t)n), ls_ptr((size_t)n + 1);
        std::vector<int2> ls_in((size_t)p->m);
        std::vector<int64_t> geoff((size_t)p->ngraphs + 1, 0);
        for (int i = 0; i < p->ngraphs; ++i) geoff[(size_t)i + 1] = geoff[(size_t)i] + graphs[(size_t)i]->fin.m;
        std::vector<int32_t> ls_where((size_t)p->m);  // graph-local ls position (offset by graph) -> merged
        p->level_ptr.assign((size_t)p->levels + 1, 0);
        // (graph, level) segments of the merged order for the team executor
        p->seg_first.assign((size_t)p->ngraphs + 1, 0);
        p->glevels.assign((size_t)p->ngraphs, 0);
        for (int i = 0; i < p->ngraphs; ++i) {
            p->glevels[(size_t)i] = graphs[(size_t)i]->fin.levels;
            p->seg_first[(size_t)i + 1] = p->seg_first[(size_t)i] + graphs[(size_t)i]->fin.levels;
        }
        p->h_seg.assign((size_t)p->seg_first[(size_t)p->ngraphs], make_int4(0, 0, 0, 0));
        {
            int64_t pos = 0, ein = 0;
            for (int32_t l = 0; l < p->levels; ++l) {
                p->level_ptr[(size_t)l] = (int32_t)pos;
                for (int i = 0; i < p->ngraphs; ++i) {
                    const Final& f = graphs[(size_t)i]->fin;
                    if (l >= f.levels) continue;
                    int4& sgm = p->h_seg[(size_t)(p->seg_first[(size_t)i] + l)];
                    sgm.x = (int32_t)pos;
                    sgm.z = (int32_t)ein;
                    const int32_t toff = p->task_off[(size_t)i];
                    for (int32_t q = f.level_ptr[(size_t)l]; q < f.level_ptr[(size_t)l + 1]; ++q) {
                        ls_node[(size_t)pos] = toff + f.ls_node[(size_t)q];
                        ls_ptr[(size_t)pos] = (int32_t)ein;
                        for (int32_t e = f.ls_ptr[(size_t)q]; e < f.ls_ptr[(size_t)q + 1]; ++e) {
                            int2 x = f.ls_in[(size_t)e];
                            x.x += toff;
                            ls_where[(size_t)(geoff[(size_t)i] + e)] = (int32_t)ein;
                            ls_in[(size_t)ein++] = x;
                        }
                        pos++;
                    }
                    sgm.y = (int32_t)pos;
                    sgm.w = (int32_t)ein;
                }
            }
            p->level_ptr[(size_t)p->levels] = (int32_t)pos;
            ls_ptr[(size_t)n] = (int32_t)ein;
            for (int i = 0; i < p->ngraphs; ++i) {
                const Final& f = graphs[(size_t)i]->fin;
                for (int64_t e = 0; e < f.m; ++e)
                    epos_ls[(size_t)(geoff[(size_t)i] + e)] = ls_where[(size_t)(geoff[(size_t)i] + f.epos_ls[(size_t)e])];
            }
        }
        // payloads: pull buffers first (saxpy and push tasks may reference them)
        p->hpidx.assign((size_t)n, -1);
        std::vector<std::vector<void*>> pull_buf((size_t)p->ngraphs);
        for (int i = 0; i < p->ngraphs; ++i) {
            const hf_graph* g = graphs[(size_t)i];
            pull_buf[(size_t)i].assign(g->payloads.size(), nullptr);
            for (size_t k = 0; k < g->payloads.size(); ++k) {
                const PayloadRec& r = g->payloads[k];
                if (r.kind != HF_PULL) continue;
                if (r.bytes && !host_dev_ptr(r.host_src))
                    return bail(fail(HF_EINVAL, "pull host buffer is not page-locked"));
                void* d = palloc(p, ((r.bytes + 15) / 16) * 16, s);
                if (!d) return bail(fail(HF_ENOMEM, "device allocation failed: pull buffer"));
                pull_buf[(size_t)i][k] = d;
            }
        }
        for (int i = 0; i < p->ngraphs; ++i) {
            const hf_graph* g = graphs[(size_t)i];
            const int32_t toff = p->task_off[(size_t)i];
            for (int32_t v = 0; v < g->fin.n; ++v) {
                const int32_t k = g->pay[(size_t)v];
                if (k < 0) continue;
                const PayloadRec& r = g->payloads[(size_t)k];
                DevPayload d;
                std::memset(&d, 0, sizeof(d));
                uint8_t dir = 0;  // 1: pull copy, 2: push copy
                d.nchunks = 1;
                d.chunk_first = -1;
                d.task = toff + v;
                d.row = row_ptr[(size_t)toff + v];
                d.deg = row_ptr[(size_t)toff + v + 1] - row_ptr[(size_t)toff + v];
                if (r.kind == HF_HOST) {  // the persistent executor's handle on it (one piece)
                    d.op = kPayHost;
                    d.n = 1;
                    d.a_bits = (uint32_t)p->host_tasks.size();
                    p->host_tasks.push_back(HostTask{g->fin.level[(size_t)v], r.fn, r.arg, i});
                } else if (r.kind == HF_KERNEL) {
                    d.op = r.op == HF_K_SAXPY_I32 ? kPaySaxpyI32 : kPaySaxpyF32;
                    d.n = r.n;
                    if (r.op == HF_K_SAXPY_I32) std::memcpy(&d.a_bits, &r.a_i, 4);
                    else std::memcpy(&d.a_bits, &r.a_f, 4);
                    d.dst = r.y_pull >= 0 ? pull_buf[(size_t)i][(size_t)g->pay[(size_t)r.y_pull]] : r.y_dev;
                    d.src = r.x_pull >= 0 ? pull_buf[(size_t)i][(size_t)g->pay[(size_t)r.x_pull]] : r.x_dev;
                } else if (r.kind == HF_PULL) {
                    d.op = kPayCopy;
                    d.n = (int64_t)r.bytes;
                    d.dst = pull_buf[(size_t)i][(size_t)k];
                    d.src = r.bytes ? host_dev_ptr(r.host_src) : nullptr;
                    dir = 1;
                    if (r.bytes) p->copies.push_back(Plan::CopyNode{d.dst, r.host_src, r.bytes, g->fin.level[(size_t)v], -1, true});
                } else {  // HF_PUSH
                    void* hd = r.bytes ? host_dev_ptr(r.host_dst) : nullptr;
                    if (r.bytes && !hd) return bail(fail(HF_EINVAL, "push host buffer is not page-locked"));
                    d.op = kPayCopy;
                    d.n = (int64_t)r.bytes;
                    d.dst = hd;
                    d.src = r.src_pull >= 0 ? pull_buf[(size_t)i][(size_t)g->pay[(size_t)r.src_pull]] : r.src_dev;
                    dir = 2;
                    if (r.bytes) p->copies.push_back(Plan::CopyNode{r.host_dst, d.src, r.bytes, g->fin.level[(size_t)v], -1, false});
                }
                int32_t sl = -1;  // the task's successors' lowest level
                {
                    const Final& f = g->fin;
                    for (int32_t e = f.row_ptr[(size_t)v]; e < f.row_ptr[(size_t)v + 1]; ++e) {
                        const int32_t w = f.succ[(size_t)e].x;
                        if (sl < 0 || f.level[(size_t)w] < sl) sl = f.level[(size_t)w];
                    }
                }
                if (dir && r.bytes) p->copies.back().succ_level = sl;
                p->pay_succ_level.push_back(sl);
                p->ncopy[0] += dir == 1;
                p->ncopy[1] += dir == 2;
                p->hpdir.push_back((uint8_t)dir);
                p->hpidx[(size_t)toff + v] = (int32_t)p->hpay.size();
                p->hpay.push_back(d);
                p->pay_task.push_back(toff + v);
                p->pay_level.push_back(g->fin.level[(size_t)v]);
            }
        }
        p->npay = (int32_t)p->hpay.size();
        // per graph: payload memory ranges pairwise disjoint wherever one of them is written
        // (saxpy writes y and reads x and y; a copy writes dst and reads src; a host task may
        // touch anything)
        p->pay_local.assign((size_t)p->ngraphs, 1);
        {
            struct Rng {
                uint64_t a, b;
                int32_t owner;
                bool write;
            };
            std::vector<std::vector<Rng>> per((size_t)p->ngraphs);
            for (int32_t q = 0; q < p->npay; ++q) {
                const int32_t t = p->pay_task[(size_t)q];
                const int32_t gi = (int32_t)(std::upper_bound(p->task_off.begin(), p->task_off.end(), t) -
                                             p->task_off.begin()) - 1;
                const DevPayload& d = p->hpay[(size_t)q];
                if (d.op == kPayHost) {
                    p->pay_local[(size_t)gi] = 0;
                    continue;
                }
                const uint64_t bytes = d.op == kPayCopy ? (uint64_t)d.n : 4ull * (uint64_t)d.n;
                if (bytes == 0) continue;
                per[(size_t)gi].push_back(Rng{(uint64_t)d.dst, (uint64_t)d.dst + bytes, q, true});
                if (d.src) per[(size_t)gi].push_back(Rng{(uint64_t)d.src, (uint64_t)d.src + bytes, q, false});
            }
            for (int32_t gi = 0; gi < p->ngraphs; ++gi) {
                std::vector<Rng>& r = per[(size_t)gi];
                std::vector<Rng> w;
                for (const Rng& x : r)
                    if (x.write) w.push_back(x);
                std::sort(w.begin(), w.end(), [](const Rng& x, const Rng& y) { return x.a < y.a; });
                // written ranges of different payloads must not overlap each other or any range
                // another payload reads: for each range, the written ranges starting before its
                // end, scanned back while they could still reach it (ends below the running
                // maximum are skipped by the check, not by the scan)
                std::vector<uint64_t> wmax(w.size());
                for (size_t i = 0; i < w.size(); ++i) wmax[i] = std::max<uint64_t>(i ? wmax[i - 1] : 0, w[i].b);
                for (size_t k = 0; k < r.size() && p->pay_local[(size_t)gi]; ++k) {
                    const Rng& x = r[k];
                    size_t hi = (size_t)(std::lower_bound(w.begin(), w.end(), x.b,
                                                          [](const Rng& y, uint64_t v) { return y.a < v; }) -
                                         w.begin());
                    while (hi > 0 && wmax[hi - 1] > x.a) {
                        const Rng& y = w[hi - 1];
                        if (y.b > x.a && y.owner != x.owner) {
                            p->pay_local[(size_t)gi] = 0;
                            break;
                        }
                        --hi;
                    }
                }
            }
        }
        // cost-model inputs kept on the host until first use
        p->h_level.resize((size_t)n);
        p->h_cat.resize((size_t)n);
        p->h_gstat.resize((size_t)p->ngraphs);
        for (int i = 0; i < p->ngraphs; ++i) {
            const hf_graph* g = graphs[(size_t)i];
            const int32_t toff = p->task_off[(size_t)i];
            for (int32_t v = 0; v < g->fin.n; ++v) {
                p->h_level[(size_t)toff + v] = g->fin.level[(size_t)v];
                const uint8_t k = g->kind[(size_t)v];
                uint8_t c = 4;
                if (k == HF_KERNEL) c = g->pay[(size_t)v] < 0 ? 0 : 1;
                else if (k == HF_PULL) c = 2;
                else if (k == HF_PUSH) c = 3;
                p->h_cat[(size_t)toff + v] = c;
            }
            p->h_gstat[(size_t)i] = make_float4((float)g->fin.n, (float)g->fin.m, (float)g->fin.levels, 0.f);
        }

        // uploads
        if ((st = upload(p, &p->d_row_ptr, row_ptr.data(), row_ptr.size(), s, "row_ptr")) != HF_OK) return bail(st);
        for (auto& r : erec) {  // successors with a payload: flag, and their payload index
            const int32_t k = p->hpidx[(size_t)r.x];
            if (k >= 0) {
                r.w = (int)((uint32_t)r.w | kPayBit);
                r.z = k;
            }
        }
        if ((st = upload(p, &p->d_erec, erec.data(), erec.size(), s, "erec")) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_meta, meta.data(), meta.size(), s, "meta")) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_indeg0, indeg0.data(), indeg0.size(), s, "indeg0")) != HF_OK) return bail(st);
        if (p->any_key0 && (st = upload(p, &p->d_key0, key0.data(), key0.size(), s, "key0")) != HF_OK) return bail(st);
        if (p->npay && (st = upload(p, &p->d_pidx, p->hpidx.data(), p->hpidx.size(), s, "pidx")) != HF_OK)
            return bail(st);
        if (p->ncopy[0] + p->ncopy[1] > 0 &&
            (st = upload(p, &p->d_pdir, p->hpdir.data(), p->hpdir.size(), s, "pdir")) != HF_OK)
            return bail(st);
        if ((st = upload(p, &p->d_ls_node, ls_node.data(), ls_node.size(), s, "ls_node", 64)) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_ls_ptr, ls_ptr.data(), ls_ptr.size(), s, "ls_ptr", 64)) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_ls_in, ls_in.data(), ls_in.size(), s, "ls_in", 64)) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_seg, p->h_seg.data(), p->h_seg.size(), s, "seg")) != HF_OK) return bail(st);
        // team stage buffers cover the widest level, up to 1,024 tasks and 2,048 in-edges (about
        // 25 KB per buffer); larger levels go through L2 instead
        for (const int4& sg : p->h_seg) {
            p->stage_n = std::max(p->stage_n, std::min(((sg.y - sg.x + 3) / 4) * 4, 1024));
            p->stage_e = std::max(p->stage_e, std::min(((sg.w - sg.z + 1) / 2) * 2, 2048));
        }
        if ((st = upload(p, &p->d_epos_csr, epos_csr.data(), epos_csr.size(), s, "epos")) != HF_OK) return bail(st);
        if ((st = upload(p, &p->d_epos_ls, epos_ls.data(), epos_ls.size(), s, "epos")) != HF_OK) return bail(st);
        p->d_pay = (DevPayload*)palloc(p, std::max<size_t>(sizeof(DevPayload) * (size_t)p->npay, 64), s);
        p->d_key = (uint32_t*)palloc(p, std::max<size_t>(4 * (size_t)n, 16), s);
        p->d_state = (unsigned long long*)palloc(p, std::max<size_t>(8 * (size_t)n, 16), s);
        p->d_chunks_left = (int32_t*)palloc(p, std::max<size_t>(4 * (size_t)p->npay, 16), s);
        p->d_ctrl = (Ctrl*)palloc(p, sizeof(Ctrl), s);
        if (!p->d_pay || !p->d_key || !p->d_state || !p->d_chunks_left || !p->d_ctrl)
            return bail(fail(HF_ENOMEM, "device allocation failed: runtime state"));
        ce = cudaMemsetAsync(p->d_ctrl, 0, sizeof(Ctrl), s);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemsetAsync"));
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "plan upload"));
    } catch (const std::bad_alloc&) {
        return bail(fail(HF_ENOMEM, "host allocation failed in plan build"));
    }
    *out = p;
    return HF_OK;
}

// Piece layout for a payload piece size: multi-piece payloads get consecutive piece-item
// numbers after the task ids; level-sync gets a per-level list of (payload, piece) items.
static hf_status plan_set_chunk(Plan* p, int64_t chunk_elems, cudaStream_t s) {
    if (chunk_elems == p->chunk_elems) return HF_OK;
    int64_t items = 0;
    std::vector<int32_t> chunk_task;
    std::vector<int32_t> seeds, pseeds;
    std::vector<int2> litems, seg_items, litems_ls;
    std::vector<TeamPiece> pdesc;  // team executor: litems resolved
    int32_t stage_p = 0, ncseed0 = 0, ncseed1 = 0, npseed_nc = 0;
    std::vector<int32_t> item_ptr((size_t)p->levels + 1, 0), item_ptr_ls;
    try {
        for (int32_t k = 0; k < p->npay; ++k) {
            DevPayload& d = p->hpay[(size_t)k];
            const int64_t piece = d.op == kPayCopy ? chunk_elems * 4 : chunk_elems;
            int64_t nc = (d.n + piece - 1) / piece;
            if (nc < 1) nc = 1;
            if (nc > INT32_MAX / 2) return fail(HF_EINVAL, "payload too large for the piece size");
            d.chunk = piece;
            d.nchunks = (int32_t)nc;
            d.chunk_first = -1;
            if (nc > 1) {
                d.chunk_first = (int32_t)items;
                for (int64_t c = 0; c < nc; ++c) chunk_task.push_back(k);  // piece item -> payload
                items += nc;
            }
            item_ptr[(size_t)p->pay_level[(size_t)k] + 1] += (int32_t)nc;
        }
        if ((int64_t)p->n + items + p->npay > INT32_MAX) return fail(HF_EINVAL, "too many payload pieces");
        for (int32_t l = 0; l < p->levels; ++l) item_ptr[(size_t)l + 1] += item_ptr[(size_t)l];
        litems.resize((size_t)item_ptr[(size_t)p->levels]);
        {
            std::vector<int32_t> fill(item_ptr.begin(), item_ptr.end() - 1);
            for (int32_t k = 0; k < p->npay; ++k) {
                const int32_t l = p->pay_level[(size_t)k];
                for (int32_t c = 0; c < p->hpay[(size_t)k].nchunks; ++c) litems[(size_t)fill[(size_t)l]++] = make_int2(k, c);
            }
        }
        // payload sources enter the queues as payload starts: non-copies first, then pull copies,
        // then push copies (each group in source order)
        std::vector<int32_t> cseeds[2];
        for (int32_t t : p->sources) {
            const int32_t k = p->hpidx.empty() ? -1 : p->hpidx[(size_t)t];
            if (k < 0) seeds.push_back(t);
            else if (p->hpdir[(size_t)k]) cseeds[p->hpdir[(size_t)k] - 1].push_back(p->n + (int32_t)items + k);
            else pseeds.push_back(p->n + (int32_t)items + k);
        }
        // pull copies in the order their successors' levels come (none: last), so that the copy
        // queue delivers first what the graph needs first and unblocks its pushes early
        {
            const int32_t base = p->n + (int32_t)items;
            auto need = [&](int32_t it) {
                const int32_t sl = p->pay_succ_level[(size_t)(it - base)];
                return sl < 0 ? INT32_MAX : sl;
            };
            std::stable_sort(cseeds[0].begin(), cseeds[0].end(), [&](int32_t x, int32_t y) { return need(x) < need(y); });
        }
        ncseed0 = (int32_t)cseeds[0].size();
        ncseed1 = (int32_t)cseeds[1].size();
        npseed_nc = (int32_t)pseeds.size();
        pseeds.insert(pseeds.end(), cseeds[0].begin(), cseeds[0].end());
        pseeds.insert(pseeds.end(), cseeds[1].begin(), cseeds[1].end());
        // the level-synchronous executor's items: the same without copies (its copy nodes)
        item_ptr_ls.assign((size_t)p->levels + 1, 0);
        for (int32_t l = 0; l < p->levels; ++l) {
            for (int32_t q = item_ptr[(size_t)l]; q < item_ptr[(size_t)l + 1]; ++q)
                if (!p->hpdir[(size_t)litems[(size_t)q].x]) litems_ls.push_back(litems[(size_t)q]);
            item_ptr_ls[(size_t)l + 1] = (int32_t)litems_ls.size();
        }
        // team executor: each (graph, level) segment's run of items (payloads are numbered
        // graph by graph, so a level's items are grouped by graph in batch order)
        const size_t nseg = p->h_seg.size();
        seg_items.assign(nseg, make_int2(0, 0));
        std::vector<int32_t> seg_cnt(nseg, 0);
        for (int32_t k = 0; k < p->npay; ++k) {
            const int32_t g = (int32_t)(std::upper_bound(p->task_off.begin(), p->task_off.end(), p->pay_task[(size_t)k]) -
                                        p->task_off.begin()) - 1;
            seg_cnt[(size_t)(p->seg_first[(size_t)g] + p->pay_level[(size_t)k])] += p->hpay[(size_t)k].nchunks;
        }
        for (int32_t l = 0; l < p->levels; ++l) {
            int32_t off = item_ptr[(size_t)l];
            for (int32_t g = 0; g < p->ngraphs; ++g) {
                if (l >= p->glevels[(size_t)g]) continue;
                const size_t sidx = (size_t)(p->seg_first[(size_t)g] + l);
                seg_items[sidx] = make_int2(off, off + seg_cnt[sidx]);
                off += seg_cnt[sidx];
                // stage buffers hold a level's descriptors up to 256 of them (8 KB)
                stage_p = std::max(stage_p, std::min(seg_cnt[sidx], 256));
            }
        }
        pdesc.resize(litems.size());
        for (size_t q = 0; q < litems.size(); ++q) {
            const DevPayload& d = p->hpay[(size_t)litems[q].x];
            const int64_t b0 = (int64_t)litems[q].y * d.chunk;
            const int64_t b1 = std::min(b0 + d.chunk, d.n);
            const int64_t sc = d.op == kPayCopy ? 1 : 4;
            TeamPiece& t = pdesc[q];
            t.dst = (char*)d.dst + sc * b0;
            t.src = (const char*)d.src + sc * b0;
            t.cnt = (int32_t)std::max<int64_t>(b1 - b0, 0);
            t.a = d.a_bits;
            t.op = d.op;
            t.task = d.task;
        }
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    p->nitems = (int32_t)items;
    p->qcap = p->n + (int32_t)items + p->npay;  // tasks, pieces and payload starts
    p->nseed = (int32_t)seeds.size();
    p->npseed = npseed_nc;
    p->ncseed[0] = ncseed0;
    p->ncseed[1] = ncseed1;
    p->pqcap = p->npay + (int32_t)items;
    p->item_ptr = item_ptr_ls;
    p->stage_p = stage_p;
    auto grow = [&](void** ptr, size_t& cap, size_t bytes) -> bool {
        bytes = std::max<size_t>(bytes, 16);
        if (cap >= bytes) return true;
        free_owned(p, *ptr);
        *ptr = palloc(p, bytes, s);
        cap = *ptr ? bytes : 0;
        return *ptr != nullptr;
    };
    if (!grow((void**)&p->d_chunk_task, p->cap_chunk_task, 4 * chunk_task.size()) ||
        !grow((void**)&p->d_seeds, p->cap_seeds, 4 * seeds.size()) ||
        !grow((void**)&p->d_pseeds, p->cap_pseeds, 4 * pseeds.size()) ||
        !grow((void**)&p->d_pqueue, p->cap_pqueue, 4 * (size_t)p->pqcap) ||
        !grow((void**)&p->d_queue, p->cap_queue, 4 * (size_t)p->qcap) ||
        !grow((void**)&p->d_items, p->cap_items, 8 * litems_ls.size()) ||
        !grow((void**)&p->d_seg_items, p->cap_seg_items, 8 * seg_items.size()) ||
        !grow((void**)&p->d_pdesc, p->cap_pdesc, sizeof(TeamPiece) * pdesc.size()))
        return fail(HF_ENOMEM, "device allocation failed: queue");
    cudaError_t e = cudaSuccess;
    if (!chunk_task.empty()) e = cudaMemcpyAsync(p->d_chunk_task, chunk_task.data(), 4 * chunk_task.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !seeds.empty()) e = cudaMemcpyAsync(p->d_seeds, seeds.data(), 4 * seeds.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !pseeds.empty()) e = cudaMemcpyAsync(p->d_pseeds, pseeds.data(), 4 * pseeds.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !litems_ls.empty())
        e = cudaMemcpyAsync(p->d_items, litems_ls.data(), 8 * litems_ls.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !seg_items.empty())
        e = cudaMemcpyAsync(p->d_seg_items, seg_items.data(), 8 * seg_items.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !pdesc.empty())
        e = cudaMemcpyAsync(p->d_pdesc, pdesc.data(), sizeof(TeamPiece) * pdesc.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && p->npay) e = cudaMemcpyAsync(p->d_pay, p->hpay.data(), sizeof(DevPayload) * (size_t)p->npay, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors die at return
    if (e != cudaSuccess) return cuda_fail(e, "piece layout upload");
    for (cudaGraphExec_t* x : {&p->lexec, &p->lexec_alt})
        if (*x) {
            cudaGraphExecDestroy(*x);
            *x = nullptr;
        }
    for (cudaGraph_t* x : {&p->lgraph, &p->lgraph_alt})
        if (*x) {
            cudaGraphDestroy(*x);
            *x = nullptr;
        }
    p->chunk_elems = chunk_elems;
    return HF_OK;
}

static hf_status ensure_instr(Plan* p, bool instrument, bool validate, cudaStream_t s) {
    const size_t nb = std::max<size_t>(8 * (size_t)p->n, 16);
    if (instrument && !p->d_t_start) {
        p->d_t_start = (int64_t*)palloc(p, nb, s);
        p->d_t_end = (int64_t*)palloc(p, nb, s);
        if (!p->d_t_start || !p->d_t_end) return fail(HF_ENOMEM, "device allocation failed: timers");
    }
    if (validate && !p->d_exec) {
        p->d_tk_start = (int64_t*)palloc(p, nb, s);
        p->d_tk_end = (int64_t*)palloc(p, nb, s);
        p->d_exec = (int32_t*)palloc(p, std::max<size_t>(4 * (size_t)p->n, 16), s);
        if (!p->d_tk_start || !p->d_tk_end || !p->d_exec) return fail(HF_ENOMEM, "device allocation failed: tickets");
    }
    return HF_OK;
}

// Level-synchronous executor: one kernel node per level (arrivals + payload pieces of that
// level), one host node per host task and one copy node per pull or push task, in a CUDA graph.
// Levels follow each other. A host task's node runs after the level before its own; a copy's
// node (run by the copy engines, the paper's pull and push as asynchronous copies, Section
// III-A) also starts after the level before its task's and must finish before the level of
// its task's first successor, so copies overlap the levels in between and one another, pulls
// and pushes using the two directions of the host link at once.
static hf_status build_level_graph(Plan* p) {
    cudaError_t e = cudaGraphCreate(&p->lgraph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    p->largs.assign((size_t)p->levels, LevelArgs());
    std::vector<cudaGraphNode_t> prev, cur, extra;
    bool prev_kernel_only = false;  // the previous level is one kernel node (no host node)
    std::vector<std::vector<const HostTask*>> host_at((size_t)p->levels);
    for (const HostTask& h : p->host_tasks) host_at[(size_t)h.level].push_back(&h);
    std::vector<std::vector<const Plan::CopyNode*>> copy_at((size_t)p->levels);
    for (const Plan::CopyNode& c : p->copies) copy_at[(size_t)c.level].push_back(&c);
    std::vector<std::vector<cudaGraphNode_t>> copies_before((size_t)p->levels);  // copy nodes a level waits for
    // pulls (host to device) of a level run in kPullChains chains, each in the order their
    // successors' levels come, so that the link delivers first what the levels need first (the
    // copy engine keeps no order among independent nodes); pushes wait only for their levels
    constexpr int kPullChains = 4;
    cudaGraphNode_t chain_tail[kPullChains] = {};
    int chain_next = 0;
    const bool pay = p->npay > 0;
    for (int32_t l = 0; l < p->levels; ++l) {
        cur.clear();
        std::vector<const Plan::CopyNode*>& cl = copy_at[(size_t)l];
        std::stable_sort(cl.begin(), cl.end(), [](const Plan::CopyNode* x, const Plan::CopyNode* y) {
            const bool px = x->pull, py = y->pull;
            if (px != py) return px;  // pulls first
            const int32_t a = x->succ_level < 0 ? INT32_MAX : x->succ_level;
            const int32_t b = y->succ_level < 0 ? INT32_MAX : y->succ_level;
            return a < b;
        });
        // copy nodes of this level's copy tasks: after the previous level, before their
        // successors' level
        for (const Plan::CopyNode* c : cl) {
            std::vector<cudaGraphNode_t> cdeps(prev);
            cudaGraphNode_t* tail = c->pull ? &chain_tail[chain_next] : nullptr;
            if (tail && *tail) cdeps.push_back(*tail);
            cudaGraphNode_t node;
            e = cudaGraphAddMemcpyNode1D(&node, p->lgraph, cdeps.data(), cdeps.size(), c->dst, c->src, c->bytes,
                                         cudaMemcpyDefault);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddMemcpyNode1D (copy task)");
            if (tail) {
                *tail = node;
                chain_next = (chain_next + 1) % kPullChains;
            }
            if (c->succ_level > l) copies_before[(size_t)c->succ_level].push_back(node);
        }
        extra = copies_before[(size_t)l];
        std::vector<cudaGraphNode_t> deps(prev);
        deps.insert(deps.end(), extra.begin(), extra.end());
        LevelArgs& a = p->largs[(size_t)l];
        a.ls_node = p->d_ls_node;
        a.ls_ptr = p->d_ls_ptr;
        a.ls_in = p->d_ls_in;
        a.key0 = p->d_key0;
        a.key = p->d_key;
        a.pay = p->d_pay;
        a.items = p->d_items;
        a.p0 = p->level_ptr[(size_t)l];
        a.p1 = p->level_ptr[(size_t)l + 1];
        a.i0 = p->item_ptr[(size_t)l];
        a.i1 = p->item_ptr[(size_t)l + 1];
        a.nb_mp = (a.p1 - a.p0 + 255) / 256;
        const int items = a.i1 - a.i0;
        const int nb_pay = items ? std::min((items + 7) / 8, p->num_sms * 8) : 0;
        const int grid = a.nb_mp + nb_pay;
        if (grid > 0) {
            // a level after a level of one kernel node (and nothing else to wait for) depends on it
            // programmatically: it launches while that kernel runs and waits inside
            // (griddepcontrol.wait) for its results
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeKernel;
            np.kernel.func = pay ? (void*)k_level<true> : (void*)k_level<false>;
            np.kernel.gridDim = dim3((unsigned)grid);
            np.kernel.blockDim = dim3(256);
            void* args[1] = {&a};
            np.kernel.kernelParams = args;
            cudaGraphEdgeData ed = {};
            ed.from_port = cudaGraphKernelNodePortProgrammatic;
            ed.type = cudaGraphDependencyTypeProgrammatic;
            const bool pdl = prev_kernel_only && prev.size() == 1 && extra.empty();
            cudaGraphNode_t node;
            e = cudaGraphAddNode(&node, p->lgraph, deps.data(), pdl ? &ed : nullptr, deps.size(), &np);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddNode (level kernel)");
            cur.push_back(node);
        }
        for (const HostTask* h : host_at[(size_t)l]) {
            cudaHostNodeParams hp;
            hp.fn = h->fn;
            hp.userData = h->arg;
            cudaGraphNode_t node;
            e = cudaGraphAddHostNode(&node, p->lgraph, deps.data(), deps.size(), &hp);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddHostNode");
            cur.push_back(node);
        }
        if (!cur.empty()) {
            prev_kernel_only = grid > 0 && host_at[(size_t)l].empty();
            prev.swap(cur);
        } else if (!extra.empty()) {  // a level without nodes still passes its copies on
            prev.insert(prev.end(), extra.begin(), extra.end());
            prev_kernel_only = false;
        }
    }
    e = cudaGraphInstantiate(&p->lexec, p->lgraph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return HF_OK;
}

hf_status plan_busy(Plan* p) {
    if (!p || !p->ran) return HF_OK;
    cudaError_t e = cudaEventQuery(p->done_ev);
    if (e == cudaSuccess && p->d2h_pending) e = cudaEventQuery(p->ev_d2h);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return HF_ESTATE;
    }
    return HF_OK;
}

// Team executor, host tasks: per-segment lists of host-task indices on the device and the
// mailbox in mapped page-locked memory (built once); before every run the previous run must be
// over (its kernel may still wait on a done flag) and the mailbox is cleared.
static hf_status team_host_setup(Plan* p, cudaStream_t s) {
    const size_t nh = p->host_tasks.size();
    if (!p->h_post) {
        std::vector<int2> seg_host(p->h_seg.size(), make_int2(0, 0));
        std::vector<int32_t> order(nh);
        std::vector<int32_t> cnt(p->h_seg.size() + 1, 0);
        for (size_t k = 0; k < nh; ++k) {
            const HostTask& h = p->host_tasks[k];
            cnt[(size_t)(p->seg_first[(size_t)h.graph] + h.level) + 1] += 1;
        }
        for (size_t q = 0; q < p->h_seg.size(); ++q) cnt[q + 1] += cnt[q];
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (size_t k = 0; k < nh; ++k) {
            const HostTask& h = p->host_tasks[k];
            const size_t q = (size_t)(p->seg_first[(size_t)h.graph] + h.level);
            order[(size_t)fill[q]++] = (int32_t)k;
        }
        for (size_t q = 0; q < p->h_seg.size(); ++q) seg_host[q] = make_int2(cnt[q], cnt[q + 1]);
        hf_status st;
        if ((st = upload(p, &p->d_seg_host, seg_host.data(), seg_host.size(), s, "host segments")) != HF_OK) return st;
        if ((st = upload(p, &p->d_host_order, order.data(), order.size(), s, "host order")) != HF_OK) return st;
        p->d_post_ctr = (int32_t*)palloc(p, 16, s);
        if (!p->d_post_ctr) return fail(HF_ENOMEM, "device allocation failed: host mailbox");
        cudaError_t e = cudaHostAlloc((void**)&p->h_post, sizeof(int32_t) * nh, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->h_hdone, sizeof(int32_t) * nh, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&p->d_post, p->h_post, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&p->d_hdone, p->h_hdone, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "host mailbox");
    }
    if (p->ran) {
        cudaError_t e = cudaEventSynchronize(p->done_ev);
        if (e != cudaSuccess) return cuda_fail(e, "previous run");
    }
    if (p->proxy.joinable()) p->proxy.join();
    for (size_t k = 0; k < nh; ++k) {
        __atomic_store_n(&p->h_post[k], -1, __ATOMIC_RELAXED);
        __atomic_store_n(&p->h_hdone[k], 0, __ATOMIC_RELAXED);
    }
    std::atomic_thread_fence(std::memory_order_seq_cst);
    return HF_OK;
}

// Host proxy of a team run: runs the host tasks in the order the device posts them and raises
// each one's done flag. Gives up after limit_ns without a new post (the run ended early).
static void team_host_proxy(Plan* p, uint64_t limit_ns) {
    const size_t nh = p->host_tasks.size();
    auto last = std::chrono::steady_clock::now();
    for (size_t i = 0; i < nh; ++i) {
        int32_t k;
        while ((k = __atomic_load_n(&p->h_post[i], __ATOMIC_ACQUIRE)) < 0) {
            if ((uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - last)
                    .count() > limit_ns)
                return;
            std::this_thread::yield();
        }
        const HostTask& h = p->host_tasks[(size_t)k];
        if (h.fn) h.fn(h.arg);
        __atomic_store_n(&p->h_hdone[k], 1, __ATOMIC_RELEASE);
        last = std::chrono::steady_clock::now();
    }
}

// New delays for the level-sorted in-edges only, as a gather: in-edge j takes delay[edge[j]]
// (edge[j]: its edge in insertion order), so the writes are sequential; non-finite flagged as in
// k_set_delays.
__global__ void k_gather_delays(const float* __restrict__ delay, const int32_t* __restrict__ edge, int2* ls_in,
                                int64_t m, int32_t* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool nonfinite = false;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int b = __float_as_int(__ldg(delay + __ldg(edge + j)));
        nonfinite |= (b & 0x7f800000) == 0x7f800000;
        reinterpret_cast<int*>(ls_in)[2 * j + 1] = b;
    }
    if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

// The successor edge records' delays brought up to date from the level-sorted in-edges.
__global__ void k_erec_delays(const int32_t* __restrict__ pos_csr, const int32_t* __restrict__ pos_ls, int4* erec,
                              const int2* __restrict__ ls_in, int64_t m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        reinterpret_cast<int*>(erec)[4 * (int64_t)__ldg(pos_csr + i) + 1] =
            reinterpret_cast<const int*>(ls_in)[2 * (int64_t)__ldg(pos_ls + i) + 1];
}

// edge[pos_ls[e]] = e: the inverse of the edge -> in-edge position map.
__global__ void k_invert_pos(const int32_t* __restrict__ pos_ls, int32_t* __restrict__ edge, int64_t m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) edge[__ldg(pos_ls + i)] = (int32_t)i;
}

// New delays for the level-synchronous or team run about to be enqueued on s: copied by the
// copy engine into one of two staging buffers on the plan's copy stream (waiting only for the
// gather that last read that staging buffer), then gathered on the plan's input stream into the
// in-edge buffer the run before it did not use (waiting only for the last run that read that
// buffer), so that copy and gather overlap the runs before; s waits for the gather, then the
// buffers (and level graphs) swap.
static hf_status delays_double_buffered(Plan* p, cudaStream_t s, const float* host) {
    cudaError_t e = cudaSuccess;
    const int grid = (int)std::min<int64_t>((p->m + 255) / 256, (int64_t)p->num_sms * 16);
    if (!p->d_ls_in_alt) {
        p->d_hstage = p->d_hstage ? p->d_hstage : (float*)palloc(p, 4 * (size_t)p->m, s);
        p->d_hstage2 = (float*)palloc(p, 4 * (size_t)p->m, s);
        p->d_ls_edge = p->d_ls_edge ? p->d_ls_edge : (int32_t*)palloc(p, 4 * (size_t)p->m, s);
        p->d_ls_in_alt = (int2*)palloc(p, 8 * (size_t)p->m + 64, s);
        p->d_bad2 = (int32_t*)palloc(p, 16, s);
        if (!p->d_hstage || !p->d_hstage2 || !p->d_ls_edge || !p->d_ls_in_alt || !p->d_bad2)
            return fail(HF_ENOMEM, "device allocation failed: delay buffers");
        k_invert_pos<<<grid, 256, 0, s>>>(p->d_epos_ls, p->d_ls_edge, p->m);
        // the second buffer starts as a copy (predecessor ids and delays)
        if ((e = cudaMemcpyAsync(p->d_ls_in_alt, p->d_ls_in, 8 * (size_t)p->m, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
            (e = cudaEventRecord(p->ev_gather, s)) != cudaSuccess ||  // nothing on istream overtakes this
            (e = cudaStreamWaitEvent(p->istream, p->ev_gather, 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p->hstream, p->ev_gather, 0)) != cudaSuccess)  // nor on hstream
            return cuda_fail(e, "delay buffers");
    }
    if (p->ran && p->last_stream != s && (e = cudaStreamWaitEvent(s, p->done_ev, 0)) != cudaSuccess)
        return cuda_fail(e, "delay upload");
    const int nb = 1 - p->lsb;        // the buffer the coming run reads
    int2* other = p->d_ls_in_alt;     // (d_ls_in_alt always names the buffer that is not d_ls_in)
    // staging buffer j is free once the last gather or scatter that read it is done; the copy
    // runs on hstream, the gather on istream once the copy has landed and once the run that
    // last read in-edge buffer nb is done
    const int j = p->hsb;
    float* stage = j ? p->d_hstage2 : p->d_hstage;
    if ((p->hread_pending[j] && (e = cudaStreamWaitEvent(p->hstream, p->ev_hread[j], 0)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(stage, host, 4 * (size_t)p->m, cudaMemcpyHostToDevice, p->hstream)) != cudaSuccess ||
        (e = cudaEventRecord(p->ev_hcopy[j], p->hstream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->istream, p->ev_hcopy[j], 0)) != cudaSuccess ||
        (p->buf_used[nb] && (e = cudaStreamWaitEvent(p->istream, p->ev_buf[nb], 0)) != cudaSuccess) ||
        (e = cudaMemsetAsync(p->d_bad2 + nb, 0, sizeof(int32_t), p->istream)) != cudaSuccess)
        return cuda_fail(e, "delay upload");
    k_gather_delays<<<grid, 256, 0, p->istream>>>(stage, p->d_ls_edge, other, p->m, p->d_bad2 + nb);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(p->ev_hread[j], p->istream)) != cudaSuccess)
        return cuda_fail(e, "delay gather");
    p->hread_pending[j] = true;
    p->hsb = j ^ 1;
    if ((e = cudaEventRecord(p->ev_gather, p->istream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, p->ev_gather, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&p->d_ctrl->bad_input, p->d_bad2 + nb, sizeof(int32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "delay gather");
    std::swap(p->d_ls_in, p->d_ls_in_alt);
    std::swap(p->lgraph, p->lgraph_alt);
    std::swap(p->lexec, p->lexec_alt);
    std::swap(p->largs, p->largs_alt);
    p->lsb = nb;
    p->erec_stale = true;
    p->gather_pending = true;
    return HF_OK;
}

// New delays for the run about to be enqueued on s, from page-locked host memory. Level-sync
// and team runs: delays_double_buffered. Persistent runs: copied by the copy engine on the
// plan's input stream, which waits only until the previous view's gather or scatter has read
// the staging buffer (so the copy overlaps the previous run), then scattered on s into both
// edge layouts.
static hf_status delays_from_host(Plan* p, cudaStream_t s, const float* host, int mode) {
    cudaError_t e = cudaSuccess;
    if (!p->istream) {
        e = cudaStreamCreateWithFlags(&p->istream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->hstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_h2d, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_gather, cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->ev_buf[i], cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->ev_hcopy[i], cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->ev_hread[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "delay upload stream");
    }
    if (mode != HF_MODE_PERSISTENT) return delays_double_buffered(p, s, host);
    const int grid = (int)std::min<int64_t>((p->m + 255) / 256, (int64_t)p->num_sms * 16);
    if (!p->d_hstage) {
        p->d_hstage = (float*)palloc(p, 4 * (size_t)p->m, s);
        p->d_ls_edge = (int32_t*)palloc(p, 4 * (size_t)p->m, s);
        if (!p->d_hstage || !p->d_ls_edge) return fail(HF_ENOMEM, "device allocation failed: delay staging");
        k_invert_pos<<<grid, 256, 0, s>>>(p->d_epos_ls, p->d_ls_edge, p->m);
        // the first upload must not overtake the allocations on s
        if ((e = cudaEventRecord(p->ev_gather, s)) != cudaSuccess) return cuda_fail(e, "delay upload");
        p->gather_pending = true;
    }
    if (p->ran && p->last_stream != s && (e = cudaStreamWaitEvent(s, p->done_ev, 0)) != cudaSuccess)
        return cuda_fail(e, "delay upload");
    if ((p->gather_pending && (e = cudaStreamWaitEvent(p->istream, p->ev_gather, 0)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(p->d_hstage, host, 4 * (size_t)p->m, cudaMemcpyHostToDevice, p->istream)) != cudaSuccess ||
        (e = cudaEventRecord(p->ev_h2d, p->istream)) != cudaSuccess || (e = cudaStreamWaitEvent(s, p->ev_h2d, 0)) != cudaSuccess ||
        (e = cudaMemsetAsync(&p->d_ctrl->bad_input, 0, sizeof(int32_t), s)) != cudaSuccess)
        return cuda_fail(e, "delay upload");
    k_set_delays<<<grid, 256, 0, s>>>(p->d_hstage, p->d_epos_csr, p->d_epos_ls, p->d_erec, p->d_ls_in, p->m,
                                      &p->d_ctrl->bad_input);
    p->erec_stale = false;
    if ((e = cudaEventRecord(p->ev_gather, s)) != cudaSuccess ||
        (e = cudaEventRecord(p->ev_hread[0], s)) != cudaSuccess)  // d_hstage is staging buffer 0
        return cuda_fail(e, "delay upload");
    p->gather_pending = true;
    p->hread_pending[0] = true;
    return HF_OK;
}

// Arrivals of the run just enqueued on s to page-locked host memory: converted into d_arr on s,
// copied out on the plan's copy stream, so that s goes on with the caller's next work (a new
// delay upload, the next run) while the copy runs. The next use of d_arr waits for the copy.
static hf_status arrivals_to_host(Plan* p, cudaStream_t s, float* host) {
    cudaError_t e = cudaSuccess;
    if (!p->cstream) {
        e = cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_conv, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_d2h, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "copy stream");
    }
    if (!p->d_arr) {
        p->d_arr = (float*)palloc(p, std::max<size_t>(4 * (size_t)p->n, 16), s);
        if (!p->d_arr) return fail(HF_ENOMEM, "device allocation failed");
    }
    if (p->d2h_pending && (e = cudaStreamWaitEvent(s, p->ev_d2h, 0)) != cudaSuccess) return cuda_fail(e, "arrival copy");
    const int grid = (int)std::min<int64_t>(((int64_t)p->n + 255) / 256, (int64_t)p->num_sms * 16);
    k_keys_to_f32<<<grid, 256, 0, s>>>(p->d_key, p->d_arr, p->n);
    if ((e = cudaEventRecord(p->ev_conv, s)) != cudaSuccess || (e = cudaStreamWaitEvent(p->cstream, p->ev_conv, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(host, p->d_arr, 4 * (size_t)p->n, cudaMemcpyDeviceToHost, p->cstream)) != cudaSuccess ||
        (e = cudaEventRecord(p->ev_d2h, p->cstream)) != cudaSuccess)
        return cuda_fail(e, "arrival copy");
    p->d2h_pending = true;
    return HF_OK;
}

hf_status plan_run(Plan* p, cudaStream_t s, const hf_run_opts& o, bool keep_status, const float* io_dly,
                   float* io_arr) {
    int mode = o.mode;
    if (mode == HF_MODE_AUTO) {
        if (!p->host_tasks.empty()) {
            mode = HF_MODE_LEVELSYNC;
        } else {
            hf_status st = plan_auto_mode(p, s, &mode);
            if (st != HF_OK) return st;
        }
    }
    if (mode != HF_MODE_LEVELSYNC && mode != HF_MODE_PERSISTENT && mode != HF_MODE_TEAM)
        return fail(HF_EINVAL, "unknown mode");
    if (o.priority < HF_PRIO_FIFO || o.priority > HF_PRIO_LEARNED) return fail(HF_EINVAL, "unknown priority");
    if (o.priority == HF_PRIO_LEARNED && !p->cm) return fail(HF_ESTATE, "HF_PRIO_LEARNED needs a cost model (hf_batch_set_costmodel)");
    hf_status st = HF_OK;
    if (mode == HF_MODE_PERSISTENT && (st = plan_prepare_priority(p, o.priority, p->cm, s)) != HF_OK) return st;
    // default piece: 512 elements for level-sync (a level's payloads spread over many warps),
    // 16,384 for the persistent executor (fewer queue items); in AUTO mode the caller's piece
    // size applies to the persistent executor only
    const bool own_chunk = o.chunk_elems > 0 && !(o.mode == HF_MODE_AUTO && mode == HF_MODE_LEVELSYNC);
    int64_t chunk = own_chunk ? o.chunk_elems : (mode == HF_MODE_PERSISTENT ? 16384 : 512);
    chunk = ((chunk + 31) / 32) * 32;
    st = plan_set_chunk(p, chunk, s);
    if (st != HF_OK) return st;
    const bool instr = (o.instrument & 1) != 0, valid = o.validate != 0;
    if ((st = ensure_instr(p, instr, valid, s)) != HF_OK) return st;
    // host buffers: new delays from page-locked host memory before the run
    if (io_dly && p->m > 0 && (st = delays_from_host(p, s, io_dly, mode)) != HF_OK) return st;
    if (mode == HF_MODE_PERSISTENT && p->erec_stale && p->m > 0) {
        const int grid = (int)std::min<int64_t>((p->m + 255) / 256, (int64_t)p->num_sms * 16);
        k_erec_delays<<<grid, 256, 0, s>>>(p->d_epos_csr, p->d_epos_ls, p->d_erec, p->d_ls_in, p->m);
        p->erec_stale = false;
    }
    cudaError_t e = keep_status ? cudaSuccess : cudaMemsetAsync(&p->d_ctrl->status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (p->n > 0) {
        if (mode == HF_MODE_LEVELSYNC) {
            if (instr || valid) return fail(HF_ENOTSUP, "instrument/validate runs need the persistent executor");
            if (!p->lexec && (st = build_level_graph(p)) != HF_OK) return st;
            if (o.time_kernel) cudaEventRecord(p->kev0, s);
            e = cudaGraphLaunch(p->lexec, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            if (o.time_kernel) cudaEventRecord(p->kev1, s);
        } else if (mode == HF_MODE_TEAM) {
            if (valid) return fail(HF_ENOTSUP, "validate runs need the persistent executor");
            if ((st = plan_team_jobs(p, o, s)) != HF_OK) return st;
            TeamArgs a;
            std::memset(&a, 0, sizeof(a));
            a.ls_node = p->d_ls_node;
            a.ls_ptr = p->d_ls_ptr;
            a.ls_in = p->d_ls_in;
            a.key0 = p->d_key0;
            a.key = p->d_key;
            a.pay = p->d_pay;
            a.items = p->d_items;
            a.seg = p->d_seg;
            a.seg_items = p->d_seg_items;
            a.ctrl = p->d_ctrl;
            a.spin_limit_ns = o.spin_limit_ns ? o.spin_limit_ns : 2000000000ull;
            a.stage_n = p->stage_n;
            a.stage_e = p->stage_e;
            a.stage_p = p->npay ? p->stage_p : 0;
            a.pdesc = p->d_pdesc;
            team_smem_attr(p);
            if (!p->host_tasks.empty()) {
                if ((st = team_host_setup(p, s)) != HF_OK) return st;
                a.seg_host = p->d_seg_host;
                a.host_order = p->d_host_order;
                a.post = p->d_post;
                a.hdone = p->d_hdone;
                a.post_ctr = p->d_post_ctr;
                e = cudaMemsetAsync(p->d_post_ctr, 0, sizeof(int32_t), s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            }
            if (instr) {
                if (!p->d_gtime) {
                    p->d_gtime = (int64_t*)palloc(p, sizeof(int64_t) * 2 * std::max<size_t>((size_t)p->ngraphs, 1), s);
                    if (!p->d_gtime) return fail(HF_ENOMEM, "device allocation failed: graph timers");
                }
                a.g_start = p->d_gtime;
                a.g_end = p->d_gtime + p->ngraphs;
            }
            p->last_gtimes = instr;
            // instrument bit 2: per-task costs (ns), accumulated from zero
            const bool rec = (o.instrument & 4) != 0;
            if (rec) {
                if (!p->d_tcost) {
                    p->d_tcost = (float*)palloc(p, sizeof(float) * std::max<size_t>((size_t)p->n, 4), s);
                    if (!p->d_tcost) return fail(HF_ENOMEM, "device allocation failed: task costs");
                }
                e = cudaMemsetAsync(p->d_tcost, 0, sizeof(float) * (size_t)p->n, s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
                a.t_cost = p->d_tcost;
            }
            p->last_tcost = rec;
            e = cudaMemsetAsync(p->d_team, 0, sizeof(int32_t) * (size_t)kTeamWords * p->tclass.size(), s);
            // a failed team raises ctrl->abort so that no new job starts; every run starts clear
            if (e == cudaSuccess) e = cudaMemsetAsync(&p->d_ctrl->abort, 0, sizeof(int32_t), s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            if (o.time_kernel) cudaEventRecord(p->kev0, s);
            // one launch per team class, in decreasing cluster size, on the plan's high-priority
            // stream (forked from the caller's stream and joined back into it), each after the
            // first a programmatic dependent of the one before: a class is launched once every CTA
            // of the previous class has started, so the clusters, which need whole groups of free
            // SMs, are placed before smaller teams and single CTAs fill the GPU, and the classes
            // then run concurrently; every kernel waits for its predecessor only at its end, so the
            // last one's completion covers them all
            const size_t nc = p->tclass.size();
            if ((e = cudaEventRecord(p->tev_fork, s)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(p->tstream[0], p->tev_fork, 0)) != cudaSuccess)
                return cuda_fail(e, "team fork");
            for (size_t i = 0; i < nc; ++i) {
                const Plan::TeamClass& c = p->tclass[i];
                TeamArgs ai = a;
                ai.jobs = p->d_jobs + c.job0;
                ai.njobs = c.njobs;
                ai.ncjobs = c.ncjobs;
                ai.team = p->d_team + (size_t)kTeamWords * i;
                ai.key_cap = c.key_cap;
                ai.task_off = p->d_toff;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)c.grid);
                cfg.blockDim = dim3(kTeamBlock);
                cfg.dynamicSmemBytes = team_class_smem(p, c.key_cap);
                team_smem_attr(p, cfg.dynamicSmemBytes);
                cfg.stream = p->tstream[0];
                cudaLaunchAttribute at[2];
                unsigned na = 0;
                if (c.k > 1) {
                    at[na].id = cudaLaunchAttributeClusterDimension;
                    at[na].val.clusterDim.x = (unsigned)c.k;
                    at[na].val.clusterDim.y = 1;
                    at[na].val.clusterDim.z = 1;
                    ++na;
                }
                if (i > 0) {
                    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    at[na].val.programmaticStreamSerializationAllowed = 1;
                    ++na;
                }
                cfg.attrs = at;
                cfg.numAttrs = na;
                void* kargs[] = {&ai};
                e = cudaLaunchKernelExC(&cfg, team_kernel(p->npay != 0, rec, c.csk != 0), kargs);
                if (e != cudaSuccess) return cuda_fail(e, "k_team launch");
            }
            if ((e = cudaEventRecord(p->tev_join[0], p->tstream[0])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, p->tev_join[0], 0)) != cudaSuccess)
                return cuda_fail(e, "team join");
            if (o.time_kernel) cudaEventRecord(p->kev1, s);
            if (!p->host_tasks.empty()) {
                const uint64_t limit = o.spin_limit_ns ? o.spin_limit_ns : 2000000000ull;
                p->proxy = std::thread(team_host_proxy, p, limit);
            }
        } else {
            ResetArgs r;
            r.n_tasks = p->n;
            r.qcap = p->qcap;
            r.n_seed = p->nseed;
            r.n_pay = p->npay;
            r.indeg0 = p->d_indeg0;
            r.key0 = p->d_key0;
            r.seeds = p->d_seeds;
            r.pseeds = p->d_pseeds;
            r.n_pseed = p->npseed;
            r.pqcap = p->pqcap;
            r.pqueue = p->d_pqueue;
            const int pay_warps = p->npay ? std::min(std::max(o.payload_warps, 0), kWarpsPerCta - 1) : 0;
            r.split = pay_warps > 0 ? 1 : 0;
            // copy warps: as many per direction, at least one warp left for the main queue
            const bool has_copies = p->ncopy[0] + p->ncopy[1] > 0;
            const int copy_warps =
                has_copies ? std::min(std::max(o.copy_warps, 0), (kWarpsPerCta - 1 - pay_warps) / 2) : 0;
            r.link = copy_warps > 0 ? 1 : 0;
            r.n_cseed0 = p->ncseed[0];
            r.n_cseed1 = p->ncseed[1];
            r.lqcap = p->pqcap;
            r.lqueue0 = r.lqueue1 = nullptr;
            if (copy_warps > 0) {
                const size_t need = 4 * (size_t)std::max(p->pqcap, 4);
                if (p->cap_lqueue < need) {
                    for (int d = 0; d < 2; ++d) {
                        free_owned(p, p->d_lqueue[d]);
                        p->d_lqueue[d] = (int32_t*)palloc(p, need, s);
                    }
                    p->cap_lqueue = (p->d_lqueue[0] && p->d_lqueue[1]) ? need : 0;
                    if (!p->cap_lqueue) return fail(HF_ENOMEM, "device allocation failed: copy queues");
                }
                r.lqueue0 = p->d_lqueue[0];
                r.lqueue1 = p->d_lqueue[1];
            }
            r.pay = p->d_pay;
            r.state = p->d_state;
            r.queue = p->d_queue;
            r.chunks_left = p->d_chunks_left;
            r.ctrl = p->d_ctrl;
            r.t_start = instr ? p->d_t_start : nullptr;
            r.t_end = instr ? p->d_t_end : nullptr;
            r.tk_start = valid ? p->d_tk_start : nullptr;
            r.tk_end = valid ? p->d_tk_end : nullptr;
            r.exec_count = valid ? p->d_exec : nullptr;
            r.stall_task = (o.stall_task >= 0 && o.stall_task < p->n) ? o.stall_task : -1;
            r.keep_status = keep_status ? 1 : 0;
            int ctas = o.ctas;
            if (ctas <= 0) {  // two CTAs (16 warps) per SM, capped by occupancy: more idle warps
                              // only add polling traffic (the autotuner searches around this); with
                              // work stealing one per SM, as idle warps probe other CTAs' rings
                int occ = 0;
                if (p->npay) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<true>, kWarpsPerCta * 32, 0);
                else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<false>, kWarpsPerCta * 32, 0);
                ctas = p->num_sms * std::min(std::max(occ, 1), o.steal_ring > 0 ? 1 : 2);
            }
            // work stealing: a ring of ring_slots cells per CTA (a power of two, 64..16384)
            int32_t ring_slots = 0;
            r.ring = nullptr;
            r.ring_cells = 0;
            r.ring_head = nullptr;
            r.ring_heads = 0;
            if (o.steal_ring > 0) {
                ring_slots = 64;
                while (ring_slots < o.steal_ring && ring_slots < 16384) ring_slots *= 2;
                const size_t cells = (size_t)ctas * (size_t)ring_slots;
                const size_t heads = (size_t)ctas * 32;
                if (p->cap_ring < 8 * cells) {
                    free_owned(p, p->d_ring);
                    p->d_ring = (unsigned long long*)palloc(p, 8 * cells, s);
                    p->cap_ring = p->d_ring ? 8 * cells : 0;
                }
                if (p->cap_ring_head < 4 * heads) {
                    free_owned(p, p->d_ring_head);
                    p->d_ring_head = (int32_t*)palloc(p, 4 * heads, s);
                    p->cap_ring_head = p->d_ring_head ? 4 * heads : 0;
                }
                if (!p->d_ring || !p->d_ring_head) return fail(HF_ENOMEM, "device allocation failed: steal rings");
                r.ring = p->d_ring;
                r.ring_cells = (int64_t)cells;
                r.ring_head = p->d_ring_head;
                r.ring_heads = (int32_t)heads;
            }
            const int64_t work = std::max<int64_t>(std::max<int64_t>(p->n, p->qcap), r.ring_cells);
            const int rgrid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)p->num_sms * 16);
            k_reset<<<std::max(rgrid, 1), 256, 0, s>>>(r);
            PersistArgs a;
            std::memset(&a, 0, sizeof(a));
            a.n_tasks = p->n;
            a.qcap = p->qcap;
            a.claim = std::min(std::max(o.claim, 1), 32);
            a.local_keep = o.local_keep < 0 ? 16 : std::min(o.local_keep, kStackCap);
            a.spin_limit_ns = o.spin_limit_ns ? o.spin_limit_ns : 2000000000ull;
            a.meta = p->d_meta;
            a.erec = p->d_erec;
            a.pidx = p->npay ? p->d_pidx : nullptr;
            a.pay = p->d_pay;
            a.chunk_pay = p->d_chunk_task;  // piece item -> payload index
            a.npieces = p->nitems;
            a.key = p->d_key;
            a.state = p->d_state;
            a.queue = p->d_queue;
            a.pqueue = p->d_pqueue;
            a.pqcap = p->pqcap;
            a.pay_warps = pay_warps;
            a.chunks_left = p->d_chunks_left;
            a.ctrl = p->d_ctrl;
            a.t_start = r.t_start;
            a.t_end = r.t_end;
            a.tk_start = r.tk_start;
            a.tk_end = r.tk_end;
            a.exec_count = r.exec_count;
            a.ring = r.ring;
            a.ring_head = r.ring_head;
            a.ring_mask = ring_slots > 0 ? ring_slots - 1 : 0;
            a.pdir = copy_warps > 0 ? p->d_pdir : nullptr;
            a.lqueue0 = r.lqueue0;
            a.lqueue1 = r.lqueue1;
            a.lqcap = r.lqcap;
            a.copy_warps = copy_warps;
            a.stats = nullptr;
            if (o.instrument & 2) {
                if (!p->d_stats) {
                    p->d_stats = (unsigned long long*)palloc(p, sizeof(unsigned long long) * kStatCount, s);
                    if (!p->d_stats) return fail(HF_ENOMEM, "device allocation failed: stats");
                }
                e = cudaMemsetAsync(p->d_stats, 0, sizeof(unsigned long long) * kStatCount, s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
                a.stats = p->d_stats;
            }
            p->last_stats = a.stats != nullptr;
            if (!p->host_tasks.empty()) {  // host tasks: the team executor's mailbox and proxy thread
                if ((st = team_host_setup(p, s)) != HF_OK) return st;
                a.post = p->d_post;
                a.hdone = p->d_hdone;
                a.post_ctr = p->d_post_ctr;
                e = cudaMemsetAsync(p->d_post_ctr, 0, sizeof(int32_t), s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
            }
            if (o.time_kernel) cudaEventRecord(p->kev0, s);
            if (p->npay) k_persist<true><<<ctas, kWarpsPerCta * 32, 0, s>>>(a);
            else k_persist<false><<<ctas, kWarpsPerCta * 32, 0, s>>>(a);
            if (o.time_kernel) cudaEventRecord(p->kev1, s);
            if (!p->host_tasks.empty()) {
                const uint64_t limit = o.spin_limit_ns ? o.spin_limit_ns : 2000000000ull;
                p->proxy = std::thread(team_host_proxy, p, limit);
            }
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    }
    if (p->ev_buf[p->lsb] && p->n > 0) {  // host-buffer runs: this run's in-edge buffer is read until here
        e = cudaEventRecord(p->ev_buf[p->lsb], s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        p->buf_used[p->lsb] = true;
    }
    e = cudaMemcpyAsync(p->h_status, &p->d_ctrl->status, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    // arrivals to the host after the status copy: both are device-to-host copies, and the small
    // one, which the caller's stream waits for, must not queue behind the large one on the copy
    // engine (the synchronisation calls wait for the arrival copy separately)
    if (io_arr && p->n > 0 && (st = arrivals_to_host(p, s, io_arr)) != HF_OK) return st;
    e = cudaEventRecord(p->done_ev, s);  // after the conversion kernel, which reads the keys
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    p->last_stream = s;
    p->ran = true;
    p->last_timed = o.time_kernel && p->n > 0;
    p->last_launches = p->n == 0 ? 0
                       : mode == HF_MODE_LEVELSYNC ? p->levels
                       : mode == HF_MODE_PERSISTENT ? 2
                                                     : (int32_t)p->tclass.size();
    p->last_instrument = instr && mode == HF_MODE_PERSISTENT;
    p->last_validate = valid && mode == HF_MODE_PERSISTENT;
    return HF_OK;
}

hf_status plan_run_host(Plan* p, cudaStream_t s, const hf_run_opts& o, const float* delay, float* arr_out) {
    if (delay && p->m > 0 && !host_dev_ptr(delay)) return fail(HF_EINVAL, "delay is not page-locked host memory");
    if (arr_out && p->n > 0 && !host_dev_ptr(arr_out)) return fail(HF_EINVAL, "arr_out is not page-locked host memory");
    return plan_run(p, s, o, false, p->m > 0 ? delay : nullptr, p->n > 0 ? arr_out : nullptr);
}

hf_status plan_sync(Plan* p) {
    if (!p->ran) return fail(HF_ESTATE, "not run");
    cudaError_t e = cudaEventSynchronize(p->done_ev);
    if (e == cudaSuccess && p->d2h_pending) e = cudaEventSynchronize(p->ev_d2h);  // arrivals to the host
    if (p->proxy.joinable()) p->proxy.join();
    if (e != cudaSuccess) return cuda_fail(e, "run");
    const int32_t s = p->h_status[0];
    if (p->h_status[2]) return fail(HF_EINVAL, "a delay given to hf_set_delays is not finite");
    if (s == HF_ETIMEDOUT) return fail(HF_ETIMEDOUT, "persistent executor made no progress within the spin limit");
    if (s != 0) return fail((hf_status)s, "device status " + std::to_string(s));
    return HF_OK;
}

hf_status plan_get_arrivals(Plan* p, int32_t gi, float* out, int on_device) {
    if (!p->ran) return fail(HF_ESTATE, "not run");
    const int32_t off = gi < 0 ? 0 : p->task_off[(size_t)gi];
    const int64_t cnt = gi < 0 ? p->n : p->task_off[(size_t)gi + 1] - off;
    if (cnt == 0) return HF_OK;
    if (!out) return fail(HF_EINVAL, "out is NULL");
    cudaStream_t s = p->last_stream;
    const int grid = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
    if (on_device) {
        k_keys_to_f32<<<grid, 256, 0, s>>>(p->d_key + off, out, cnt);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? HF_OK : cuda_fail(e, "key conversion");
    }
    if (!p->d_arr) {
        p->d_arr = (float*)palloc(p, std::max<size_t>(4 * (size_t)p->n, 16), s);
        if (!p->d_arr) return fail(HF_ENOMEM, "device allocation failed");
    }
    if (p->d2h_pending) cudaStreamWaitEvent(s, p->ev_d2h, 0);
    k_keys_to_f32<<<grid, 256, 0, s>>>(p->d_key + off, p->d_arr + off, cnt);
    cudaError_t e = cudaMemcpyAsync(out, p->d_arr + off, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "arrival copy");
}

hf_status plan_get_times(Plan* p, int32_t gi, int64_t* a, int64_t* b) {
    if (!p->ran || !p->last_instrument) return fail(HF_ESTATE, "last run was not instrumented");
    const int32_t off = p->task_off[(size_t)gi];
    const int64_t cnt = p->task_off[(size_t)gi + 1] - off;
    cudaStream_t s = p->last_stream;
    cudaError_t e = cudaSuccess;
    if (a && cnt) e = cudaMemcpyAsync(a, p->d_t_start + off, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b && cnt) e = cudaMemcpyAsync(b, p->d_t_end + off, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "timer copy");
}

hf_status plan_get_stamps(Plan* p, int32_t gi, int64_t* a, int64_t* b, int32_t* c) {
    if (!p->ran || !p->last_validate) return fail(HF_ESTATE, "last run was not a validate run");
    const int32_t off = p->task_off[(size_t)gi];
    const int64_t cnt = p->task_off[(size_t)gi + 1] - off;
    cudaStream_t s = p->last_stream;
    cudaError_t e = cudaSuccess;
    if (a && cnt) e = cudaMemcpyAsync(a, p->d_tk_start + off, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b && cnt) e = cudaMemcpyAsync(b, p->d_tk_end + off, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && c && cnt) e = cudaMemcpyAsync(c, p->d_exec + off, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "ticket copy");
}

hf_status plan_get_stats(Plan* p, int64_t* out, int32_t n) {
    if (!p->ran || !p->last_stats) return fail(HF_ESTATE, "last run did not record executor counters");
    unsigned long long h[kStatCount];
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(h, p->d_stats, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    for (int32_t i = 0; i < n && i < kStatCount; ++i) out[i] = (int64_t)h[i];
    return HF_OK;
}

hf_status plan_get_graph_times(Plan* p, int64_t* start, int64_t* end) {
    if (!p->ran || !p->last_gtimes) return fail(HF_ESTATE, "last run was not an instrumented team run");
    const size_t g = (size_t)p->ngraphs;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e == cudaSuccess && g) e = cudaMemcpy(start, p->d_gtime, 8 * g, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && g) e = cudaMemcpy(end, p->d_gtime + g, 8 * g, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "graph timer copy");
}

hf_status plan_get_task_costs(Plan* p, int32_t gi, float* out) {
    if (!p->ran || !p->last_tcost) return fail(HF_ESTATE, "last run was not a team run with instrument bit 2");
    const int32_t off = gi < 0 ? 0 : p->task_off[(size_t)gi];
    const int64_t cnt = gi < 0 ? p->n : p->task_off[(size_t)gi + 1] - off;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e == cudaSuccess && cnt) e = cudaMemcpy(out, p->d_tcost + off, sizeof(float) * (size_t)cnt, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "task cost copy");
}

hf_status plan_last_launches(Plan* p, int32_t* n) {
    if (!p->ran) return fail(HF_ESTATE, "not run");
    *n = p->last_launches;
    return HF_OK;
}

hf_status plan_team_plan(Plan* p, int32_t* team_size) {
    if (p->team_k.size() != (size_t)p->ngraphs) return fail(HF_ESTATE, "no team-executor run yet");
    std::memcpy(team_size, p->team_k.data(), sizeof(int32_t) * p->team_k.size());
    return HF_OK;
}

hf_status plan_team_keys(Plan* p, int32_t* shared) {
    if (p->team_sk.size() != (size_t)p->ngraphs) return fail(HF_ESTATE, "no team-executor run yet");
    std::memcpy(shared, p->team_sk.data(), sizeof(int32_t) * p->team_sk.size());
    return HF_OK;
}

hf_status plan_team_flags(Plan* p, int32_t* flags) {
    if (p->team_sk.size() != (size_t)p->ngraphs) return fail(HF_ESTATE, "no team-executor run yet");
    for (int32_t g = 0; g < p->ngraphs; ++g) {
        int32_t f = p->team_sk[(size_t)g] ? kJobSharedKeys : 0;
        if (p->task_off[(size_t)g + 1] - p->task_off[(size_t)g] >= kPipeMinTasks) f |= kJobPipelined;
        if (p->pay_local[(size_t)g]) f |= kJobPayloadLocal;
        flags[g] = f;
    }
    return HF_OK;
}

hf_status plan_kernel_ms(Plan* p, float* ms) {
    if (!p->ran || !p->last_timed) return fail(HF_ESTATE, "last run was not a time_kernel run");
    cudaError_t e = cudaEventSynchronize(p->kev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, p->kev0, p->kev1);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "cudaEventElapsedTime");
}

hf_status plan_set_delays(Plan* p, const float* delay, int on_device, cudaStream_t s) {
    if (p->m == 0) return HF_OK;
    if (!delay) return fail(HF_EINVAL, "delay is NULL");
    const float* src = delay;
    // page-locked host memory: the scatter kernel reads it over the host link directly (one
    // pass, no staging copy); other host memory goes through a staging copy
    const float* mapped = on_device ? nullptr : (const float*)host_dev_ptr(delay);
    if (mapped) {
        src = mapped;
    } else if (!on_device) {
        if (!p->d_dly_stage) {
            p->d_dly_stage = (float*)palloc(p, 4 * (size_t)p->m, s);
            if (!p->d_dly_stage) return fail(HF_ENOMEM, "device allocation failed: delay staging");
        }
        cudaError_t e = cudaMemcpyAsync(p->d_dly_stage, delay, 4 * (size_t)p->m, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "delay copy");
        src = p->d_dly_stage;
    }
    const int grid = (int)std::min<int64_t>((p->m + 255) / 256, (int64_t)p->num_sms * 16);
    cudaError_t e0 = cudaMemsetAsync(&p->d_ctrl->bad_input, 0, sizeof(int32_t), s);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaMemsetAsync");
    k_set_delays<<<grid, 256, 0, s>>>(src, p->d_epos_csr, p->d_epos_ls, p->d_erec, p->d_ls_in, p->m,
                                      &p->d_ctrl->bad_input);
    p->erec_stale = false;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "delay scatter");
}

// ------------------------------------------------------------------ cost model plumbing

// The 12 features of every task (layout in include/hf.h).
__global__ void k_features(int n, const int2* __restrict__ meta, const int4* __restrict__ erec,
                           const int32_t* __restrict__ indeg0, const int32_t* __restrict__ level,
                           const uint8_t* __restrict__ cat, const int32_t* __restrict__ pidx,
                           const DevPayload* __restrict__ pay, const int32_t* __restrict__ toff, int ng,
                           const float4* __restrict__ gstat, float* __restrict__ X) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int lo = 0, hi = ng;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (toff[mid] <= v) lo = mid;
            else hi = mid;
        }
        const float4 gs = gstat[lo];
        const int2 mt = meta[v];
        const int c = cat[v];
        const int lev = level[v];
        double bytes = 0.0;
        const int p = pidx ? pidx[v] : -1;
        if (p >= 0) bytes = pay[p].op == kPayCopy ? (double)pay[p].n : pay[p].op == kPayHost ? 0.0 : 12.0 * (double)pay[p].n;
        float msf = 0.f;
        if (mt.y > 0) {
            int64_t sum = 0;
            for (int e = mt.x; e < mt.x + mt.y; ++e) {
                const int4 r = erec[e];
                int len = (int)((uint32_t)r.w >> 16);
                if ((uint32_t)len == kLongMark) len = meta[r.x].y;
                sum += len;
            }
            msf = (float)((double)sum / (double)mt.y);
        }
        float* x = X + (int64_t)v * HF_FEATURES;
        x[0] = c == 0 ? 1.f : 0.f;
        x[1] = c == 1 ? 1.f : 0.f;
        x[2] = c == 2 ? 1.f : 0.f;
        x[3] = c == 3 ? 1.f : 0.f;
        x[4] = log1pf((float)indeg0[v]);
        x[5] = log1pf((float)mt.y);
        x[6] = (float)lev / gs.z;
        x[7] = log1pf((float)lev);
        x[8] = log1pf((float)bytes);
        x[9] = log1pf(gs.x);
        x[10] = log1pf(gs.y);
        x[11] = log1pf(msf);
    }
}

// Plain heuristic cost (ns of warp time), the fallback the learned model is judged against:
// a fixed cost per task, one atomic round trip per out-edge, payload bytes at the bandwidth
// one warp sustains (one 512-element saxpy block, 6 KB, per ~0.75 us round trip). Constants
// are first-principles estimates, not fitted.
constexpr float kHeurTask = 300.f, kHeurEdge = 30.f, kHeurBytesPerNs = 8.f;

__global__ void k_costs(int n, const float* __restrict__ X, const float* __restrict__ y, float* __restrict__ c) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (y) {
            c[v] = expf(fminf(fmaxf(y[v], 0.f), 30.f));
        } else {
            const float* x = X + (int64_t)v * HF_FEATURES;
            c[v] = kHeurTask + kHeurEdge * expm1f(x[5]) + expm1f(x[8]) / kHeurBytesPerNs;
        }
    }
}

// One level of the reverse pass: b(v) = c(v) + max over successors b(s), sinks b = c.
__global__ void k_bottom(int p0, int p1, const int32_t* __restrict__ ls_node, const int2* __restrict__ meta,
                         const int4* __restrict__ erec, const float* __restrict__ c, float* __restrict__ b) {
    const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int v = ls_node[p];
    const int2 mt = meta[v];
    if (mt.y == 0) {
        b[v] = c[v];
        return;
    }
    float mx = -INFINITY;
    for (int e = mt.x; e < mt.x + mt.y; ++e) mx = fmaxf(mx, __ldcg(b + erec[e].x));
    b[v] = __fadd_rn(mx, c[v]);
}

static hf_status ensure_cm_inputs(Plan* p, cudaStream_t s) {
    if (p->d_level) return HF_OK;
    hf_status st;
    if ((st = upload(p, &p->d_level, p->h_level.data(), p->h_level.size(), s, "level")) != HF_OK) return st;
    if ((st = upload(p, &p->d_cat, p->h_cat.data(), p->h_cat.size(), s, "cat")) != HF_OK) return st;
    if ((st = upload(p, &p->d_toff, p->task_off.data(), p->task_off.size(), s, "task offsets")) != HF_OK) return st;
    if ((st = upload(p, &p->d_gstat, p->h_gstat.data(), p->h_gstat.size(), s, "graph stats")) != HF_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);  // host vectors stay alive, but keep uploads ordered
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "cost model inputs");
}

hf_status plan_features(Plan* p, float* X, cudaStream_t s) {
    if (p->n == 0) return HF_OK;
    if (!X) return fail(HF_EINVAL, "X is NULL");
    hf_status st = ensure_cm_inputs(p, s);
    if (st != HF_OK) return st;
    // the payload table reaches the device with the first piece layout
    if (p->chunk_elems < 0 && (st = plan_set_chunk(p, 16384, s)) != HF_OK) return st;
    const int grid = std::min((p->n + 255) / 256, p->num_sms * 16);
    k_features<<<grid, 256, 0, s>>>(p->n, p->d_meta, p->d_erec, p->d_indeg0, p->d_level, p->d_cat,
                                    p->npay ? p->d_pidx : nullptr, p->d_pay, p->d_toff, p->ngraphs, p->d_gstat, X);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "k_features");
}

hf_status plan_bottom_levels(Plan* p, const float* cost, float* bottom, cudaStream_t s) {
    if (p->n == 0) return HF_OK;
    if (!cost || !bottom) return fail(HF_EINVAL, "NULL argument");
    for (int32_t l = p->levels - 1; l >= 0; --l) {
        const int p0 = p->level_ptr[(size_t)l], p1 = p->level_ptr[(size_t)l + 1];
        k_bottom<<<(p1 - p0 + 255) / 256, 256, 0, s>>>(p0, p1, p->d_ls_node, p->d_meta, p->d_erec, cost, bottom);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "k_bottom");
}

hf_status plan_task_costs(Plan* p, int32_t priority, const hf_costmodel* cm, float* cost, float* bottom,
                          cudaStream_t s) {
    if (p->n == 0) return HF_OK;
    if (priority != HF_PRIO_HEURISTIC && priority != HF_PRIO_LEARNED) return fail(HF_EINVAL, "priority must be HEURISTIC or LEARNED");
    if (priority == HF_PRIO_LEARNED && !cm) return fail(HF_ESTATE, "no cost model attached");
    if (!cost || !bottom) return fail(HF_EINVAL, "NULL output");
    hf_status st = HF_OK;
    float* X = (float*)dev_alloc(sizeof(float) * HF_FEATURES * (size_t)p->n, s);
    float* y = priority == HF_PRIO_LEARNED ? (float*)dev_alloc(sizeof(float) * (size_t)p->n, s) : nullptr;
    if (!X || (priority == HF_PRIO_LEARNED && !y)) {
        dev_free(X, s);
        dev_free(y, s);
        return fail(HF_ENOMEM, "device allocation failed: features");
    }
    st = plan_features(p, X, s);
    if (st == HF_OK && y) st = mlp_forward(costmodel_params(cm), X, p->n, y, s);
    if (st == HF_OK) {
        const int grid = std::min((p->n + 255) / 256, p->num_sms * 16);
        k_costs<<<grid, 256, 0, s>>>(p->n, X, y, cost);
        cudaError_t e = cudaGetLastError();
        st = e != cudaSuccess ? cuda_fail(e, "k_costs") : plan_bottom_levels(p, cost, bottom, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);  // before the temporaries are released
    dev_free(X, s);
    dev_free(y, s);
    if (st == HF_OK && e != cudaSuccess) st = cuda_fail(e, "cost kernels");
    return st;
}

// The persistent executor's ready-queue priority: its seed tasks (the sources) enter the
// queue by decreasing bottom-level weight (longest remaining predicted critical path first) for
// HEURISTIC / LEARNED runs; FIFO keeps id order. Later ready tasks keep release order: ranking
// them by bottom level when a warp's stack overflows (which of them stay in shared memory) was
// measured and made runs 15-55 % slower on the batch workloads.
hf_status plan_prepare_priority(Plan* p, int32_t priority, const hf_costmodel* cm, cudaStream_t s) {
    if (priority == p->seed_prio && (priority == HF_PRIO_FIFO || p->d_prio)) return HF_OK;
    if (priority == HF_PRIO_FIFO) {
        std::sort(p->sources.begin(), p->sources.end());
    } else {
        if (!p->d_prio) {
            p->d_prio = (float*)palloc(p, sizeof(float) * std::max<size_t>((size_t)p->n, 4), s);
            if (!p->d_prio) return fail(HF_ENOMEM, "device allocation failed: priorities");
        }
        float* cost = (float*)dev_alloc(sizeof(float) * std::max<size_t>((size_t)p->n, 4), s);
        if (!cost) return fail(HF_ENOMEM, "device allocation failed: costs");
        hf_status st = plan_task_costs(p, priority, cm, cost, p->d_prio, s);
        dev_free(cost, s);
        if (st != HF_OK) return st;
        std::vector<float> b((size_t)p->n);
        cudaError_t e = cudaMemcpy(b.data(), p->d_prio, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "priority download");
        std::sort(p->sources.begin(), p->sources.end());
        std::stable_sort(p->sources.begin(), p->sources.end(),
                         [&](int32_t x, int32_t y) { return b[(size_t)x] > b[(size_t)y]; });
    }
    p->seed_prio = priority;
    p->chunk_elems = -1;  // seeds are rebuilt with the next piece layout
    return HF_OK;
}

hf_status plan_refresh_priorities(Plan* p, const hf_costmodel* cm, cudaStream_t s) {
    const int32_t pr = p->seed_prio;
    p->seed_prio = -1;
    p->auto_mode = -1;
    return plan_prepare_priority(p, pr == -1 ? HF_PRIO_FIFO : pr, cm, s);
}

// ------------------------------------------------------------------ autotuning

// Time per run of back-to-back runs (as a caller streaming runs sees it): one warm-up run, then
// three blocks of `reps` runs enqueued without synchronisation, each timed by CUDA events on s;
// the median block's time per run.
static hf_status time_runs(Plan* p, cudaStream_t s, const hf_run_opts& o, int reps, float* ms) {
    hf_run_opts w = o;
    w.time_kernel = 0;
    hf_status st = plan_run(p, s, w);
    if (st == HF_OK) st = plan_sync(p);
    if (st != HF_OK) return st;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(HF_ECUDA, "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(HF_ECUDA, "cudaEventCreate");
    }
    std::vector<float> t;
    for (int blk = 0; blk < 3 && st == HF_OK; ++blk) {
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && st == HF_OK; ++i) st = plan_run(p, s, w);
        cudaEventRecord(e1, s);
        if (st == HF_OK) st = plan_sync(p);
        float x = 0.f;
        if (st == HF_OK && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess) t.push_back(x / (float)std::max(reps, 1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HF_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t.empty() ? 0.f : t[t.size() / 2];
    return HF_OK;
}

using TuneKey = std::tuple<int, int, int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<hf_run_opts, float>> g_tune_cache;

static TuneKey tune_key(const Plan* p) {
    const int logn = p->n > 0 ? (int)std::floor(std::log2((double)p->n)) : 0;
    const int epn = p->n > 0 ? (int)std::lround(10.0 * (double)p->m / (double)p->n) : 0;
    const int payq = p->n > 0 ? (int)std::lround(20.0 * (double)p->npay / (double)p->n) : 0;
    const int logd = p->levels > 0 ? (int)std::floor(std::log2((double)p->levels)) : 0;
    return TuneKey(logn, epn, payq, logd, p->ngraphs > 1 ? 1 : 0, 0);
}

// Team executor: coordinate descent over the planner's payload-cost scale (contention), the
// cluster size for every graph (0: the cost model's plan) and the payload piece size; each
// trial the median of 3 timed runs.
static hf_status autotune_team(Plan* p, cudaStream_t s, const hf_run_opts& base, hf_run_opts* best, float* best_ms) {
    hf_run_opts cur = base;
    cur.mode = HF_MODE_TEAM;
    cur.instrument = cur.validate = cur.time_kernel = 0;
    cur.stall_task = -1;
    cur.team_size = 0;
    cur.team_scale = team_scale_default(cur.priority);
    if (cur.chunk_elems <= 0) cur.chunk_elems = 512;
    float best_t = 0.f;
    hf_status st = time_runs(p, s, cur, 3, &best_t);
    if (st != HF_OK) return st;
    const std::vector<int> size_v{0, 1, 2, 4, 8, 16};
    const std::vector<int64_t> chunk_v{256, 512, 1024, 2048};
    const std::vector<int> scale_v{-4, -2, 1, 2, 4, 8, 16};  // (negative: 1/4, 1/2)
    const std::vector<int> fold_v{0, -1, 4, 8, 16};
    for (int round = 0; round < 2; ++round) {
        for (int dim = 0; dim < 4; ++dim) {  // planner scale, cluster size, piece size, one launch or one per size
            if (dim == 2 && p->npay == 0) continue;
            if ((dim == 0 || dim == 3) && (cur.team_size != 0 || cur.priority == HF_PRIO_FIFO)) continue;
            if (dim == 0 && p->npay == 0) continue;
            const size_t nv = dim == 0 ? scale_v.size() : dim == 1 ? size_v.size() : dim == 2 ? chunk_v.size()
                                                                                               : fold_v.size();
            for (size_t i = 0; i < nv; ++i) {
                hf_run_opts t = cur;
                if (dim == 0) t.team_scale = scale_v[i];
                else if (dim == 1) t.team_size = size_v[i];
                else if (dim == 2) t.chunk_elems = chunk_v[i];
                else t.team_fold = fold_v[i];
                if (t.team_size == cur.team_size && t.chunk_elems == cur.chunk_elems && t.team_scale == cur.team_scale &&
                    t.team_fold == cur.team_fold)
                    continue;
                float ms = 0.f;
                if ((st = time_runs(p, s, t, 3, &ms)) != HF_OK) return st;
                if (ms < best_t) {
                    best_t = ms;
                    cur = t;
                }
            }
        }
    }
    *best = cur;
    *best_ms = best_t;
    return HF_OK;
}

hf_status plan_autotune(Plan* p, cudaStream_t s, const hf_run_opts& base, int force, hf_run_opts* best,
                        float* best_ms) {
    const bool team = base.mode == HF_MODE_TEAM;
    TuneKey key = tune_key(p);
    std::get<4>(key) += team ? 2 : 0;
    std::get<5>(key) = base.priority;  // the tuned plan depends on the cost source
    if (!force) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = base;
            best->mode = team ? HF_MODE_TEAM : HF_MODE_PERSISTENT;
            best->ctas = it->second.first.ctas;
            best->claim = it->second.first.claim;
            best->local_keep = it->second.first.local_keep;
            best->chunk_elems = it->second.first.chunk_elems;
            best->payload_warps = it->second.first.payload_warps;
            best->team_size = it->second.first.team_size;
            best->team_scale = it->second.first.team_scale;
            best->steal_ring = it->second.first.steal_ring;
            best->copy_warps = it->second.first.copy_warps;
            best->team_fold = it->second.first.team_fold;
            *best_ms = it->second.second;
            return HF_OK;
        }
    }
    if (team) {
        hf_status st = autotune_team(p, s, base, best, best_ms);
        if (st != HF_OK) return st;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_pair(*best, *best_ms);
        return HF_OK;
    }
    hf_run_opts cur = base;
    cur.mode = HF_MODE_PERSISTENT;
    cur.instrument = cur.validate = cur.time_kernel = 0;
    cur.stall_task = -1;
    const int sms = p->num_sms;
    cur.ctas = 2 * sms;
    cur.claim = 8;
    cur.local_keep = 8;
    if (cur.chunk_elems <= 0) cur.chunk_elems = 16384;
    float best_t = 0.f;
    hf_status st = time_runs(p, s, cur, 3, &best_t);
    if (st != HF_OK) return st;
    const std::vector<int> ctas_v{sms / 2, sms, 2 * sms, 4 * sms};
    const std::vector<int> claim_v{1, 4, 16, 32};
    const std::vector<int> keep_v{4, 8, 12, 16};
    const std::vector<int64_t> chunk_v{1024, 4096, 16384};
    const std::vector<int> payw_v{0, 1, 2, 4};
    const std::vector<int> ring_v{0, 1024};  // global queue alone, or work stealing
    const std::vector<int> copyw_v{0, 1, 2};
    const bool has_copies = p->ncopy[0] + p->ncopy[1] > 0;
    for (int round = 0; round < 2; ++round) {
        for (int dim = 0; dim < 7; ++dim) {
            if ((dim == 3 || dim == 4) && p->npay == 0) continue;
            if (dim == 6 && !has_copies) continue;
            const size_t nv = dim == 0 ? ctas_v.size() : dim == 1 ? claim_v.size() : dim == 2 ? keep_v.size()
                              : dim == 3 ? chunk_v.size() : dim == 4 ? payw_v.size() : dim == 5 ? ring_v.size()
                              : copyw_v.size();
            for (size_t i = 0; i < nv; ++i) {
                hf_run_opts t = cur;
                if (dim == 0) t.ctas = ctas_v[i];
                else if (dim == 1) t.claim = claim_v[i];
                else if (dim == 2) t.local_keep = keep_v[i];
                else if (dim == 3) t.chunk_elems = chunk_v[i];
                else if (dim == 4) t.payload_warps = payw_v[i];
                else if (dim == 5) t.steal_ring = ring_v[i];
                else t.copy_warps = copyw_v[i];
                if (t.ctas == cur.ctas && t.claim == cur.claim && t.local_keep == cur.local_keep &&
                    t.chunk_elems == cur.chunk_elems && t.payload_warps == cur.payload_warps &&
                    t.steal_ring == cur.steal_ring && t.copy_warps == cur.copy_warps)
                    continue;
                float ms = 0.f;
                if ((st = time_runs(p, s, t, 3, &ms)) != HF_OK) return st;
                if (ms < best_t) {
                    best_t = ms;
                    cur = t;
                }
            }
        }
    }
    *best = cur;
    *best_ms = best_t;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_pair(cur, best_t);
    return HF_OK;
}

// ------------------------------------------------------------------ executor choice

// Machine constants for the makespan predictions, measured once per process on a chain of
// tasks: the level-synchronous executor's time per level, the persistent executor's time per
// dependent hop, and the team executor's time per level for a solo CTA and for a cluster.
static std::mutex g_cal_mu;
static bool g_cal_done = false;
static float g_t_level_ns = 0.f, g_t_hop_ns = 0.f, g_t_team_solo_ns = 0.f, g_t_team_cluster_ns = 0.f;
// Time per in-edge gathered on one SM in one level (ns): a level's gather is bound by the SM's
// rate of scattered key loads, so a wide level costs more than the chain's one-task level.
// Measured on a wide calibration graph (512 levels of 256 tasks, 4 in-edges each) against the
// chain: level-sync (one CTA per 256 tasks), team on one CTA, team on a 4-CTA cluster.
static float g_r_level_ns = 0.f, g_r_team_ns = 0.f, g_r_cluster_ns = 0.f;
// host link (GB/s): host to device, device to host, and both directions at once (bytes of both
// copies over their common time)
static float g_link_gbs[3] = {0.f, 0.f, 0.f};

// Bandwidth of the host link: the best of three 64 MiB copies between page-locked host memory
// and the device (copy engine) in each direction, then both directions at once on two streams
// (what pulls and pushes running together get), timed with CUDA events.
static hf_status measure_link(cudaStream_t s) {
    const size_t bytes = 64u << 20;
    void* h = nullptr;
    void* h2 = nullptr;
    void* d = dev_alloc(2 * bytes, s);
    if (!d) return fail(HF_ENOMEM, "device allocation failed: link calibration");
    cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&h2, bytes, cudaHostAllocDefault);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    cudaStream_t s2 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&e2);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    char* d2 = static_cast<char*>(d) + bytes;
    for (int dir = 0; dir < 3 && e == cudaSuccess; ++dir) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess && dir != 1) e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && dir == 1) e = cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && dir == 2) {  // the other direction at the same time on s2
                e = cudaStreamWaitEvent(s2, e0, 0);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h2, d2, bytes, cudaMemcpyDeviceToHost, s2);
                if (e == cudaSuccess) e = cudaEventRecord(e2, s2);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e2, 0);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;  // rep 0 warms up
        }
        if (e == cudaSuccess) g_link_gbs[dir] = (float)((double)(dir == 2 ? 2 : 1) * bytes / (best * 1e-3) / 1e9);
    }
    if (s2) cudaStreamDestroy(s2);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    if (h) cudaFreeHost(h);
    if (h2) cudaFreeHost(h2);
    dev_free(d, s);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "link calibration");
}

static hf_status calibrate(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_cal_mu);
    if (g_cal_done) return HF_OK;
    const int32_t n = 2048;
    hf_graph* g = nullptr;
    hf_status st = hf_graph_create(&g, n, n);
    if (st != HF_OK) return st;
    st = hf_add_tasks_bulk(g, n, nullptr, nullptr);
    for (int32_t i = 0; i + 1 < n && st == HF_OK; ++i) st = hf_precede_w(g, i, i + 1, 1.0f);
    if (st == HF_OK) st = hf_finalize(g);
    Plan* p = nullptr;
    if (st == HF_OK) {
        std::vector<hf_graph*> one{g};
        st = plan_build(one, &p);
    }
    float tl = 0.f, tp = 0.f, ts = 0.f, tc = 0.f;
    if (st == HF_OK) {
        hf_run_opts o;
        hf_run_opts_default(&o);
        o.mode = HF_MODE_LEVELSYNC;
        st = time_runs(p, s, o, 1, &tl);
        o.mode = HF_MODE_PERSISTENT;
        o.ctas = p->num_sms;
        if (st == HF_OK) st = time_runs(p, s, o, 1, &tp);
        hf_run_opts_default(&o);
        o.mode = HF_MODE_TEAM;
        o.team_size = 1;
        if (st == HF_OK) st = time_runs(p, s, o, 1, &ts);
        o.team_size = 2;
        if (st == HF_OK) st = time_runs(p, s, o, 1, &tc);
    }
    if (p) plan_destroy(p);
    hf_graph_destroy(g);
    // the wide graph: level l's task i has its first in-edge from level l - 1, three more from
    // anywhere earlier (a fixed hash), delays 1
    const int32_t W = 256, LW = 512, FW = 4;
    float tlw = 0.f, tsw = 0.f, tcw = 0.f;
    hf_graph* gw = nullptr;
    Plan* pw = nullptr;
    if (st == HF_OK) st = hf_graph_create(&gw, (int64_t)W * LW, (int64_t)W * LW * FW);
    if (st == HF_OK) st = hf_add_tasks_bulk(gw, (int64_t)W * LW, nullptr, nullptr);
    if (st == HF_OK) {
        std::vector<int32_t> es, ed;
        uint64_t h = 0x9e3779b97f4a7c15ull;
        for (int32_t l = 1; l < LW; ++l)
            for (int32_t i = 0; i < W; ++i)
                for (int32_t j = 0; j < FW; ++j) {
                    h ^= h >> 33;
                    h *= 0xff51afd7ed558ccdull;
                    h ^= h >> 29;
                    h += 0x632be59bd9b4e5f5ull;
                    es.push_back(j == 0 ? (l - 1) * W + (int32_t)(h % W) : (int32_t)(h % (uint64_t)(l * W)));
                    ed.push_back(l * W + i);
                }
        std::vector<float> dl(es.size(), 1.0f);
        st = hf_precede_bulk(gw, (int64_t)es.size(), es.data(), ed.data(), dl.data());
    }
    if (st == HF_OK) st = hf_finalize(gw);
    if (st == HF_OK) {
        std::vector<hf_graph*> one{gw};
        st = plan_build(one, &pw);
    }
    if (st == HF_OK) {
        hf_run_opts o;
        hf_run_opts_default(&o);
        o.mode = HF_MODE_LEVELSYNC;
        st = time_runs(pw, s, o, 1, &tlw);
        hf_run_opts_default(&o);
        o.mode = HF_MODE_TEAM;
        o.team_size = 1;
        if (st == HF_OK) st = time_runs(pw, s, o, 1, &tsw);
        o.team_size = 4;
        if (st == HF_OK) st = time_runs(pw, s, o, 1, &tcw);
    }
    if (pw) plan_destroy(pw);
    if (gw) hf_graph_destroy(gw);
    if (st == HF_OK) st = measure_link(s);
    if (st != HF_OK) return st;
    const float e_lvl = (float)(W * FW);
    g_r_level_ns = std::max(0.f, 1e6f * tlw / (float)LW - 1e6f * tl / (float)n) / e_lvl;
    g_r_team_ns = std::max(0.f, 1e6f * tsw / (float)LW - 1e6f * ts / (float)n) / e_lvl;
    g_r_cluster_ns = std::max(0.f, 1e6f * tcw / (float)LW - 1e6f * tc / (float)n) / (e_lvl / 4.f);
    g_t_level_ns = 1e6f * tl / (float)n;
    g_t_hop_ns = 1e6f * tp / (float)n;
    g_t_team_solo_ns = 1e6f * ts / (float)n;
    g_t_team_cluster_ns = 1e6f * tc / (float)n;
    g_cal_done = true;
    return HF_OK;
}

hf_status plan_calibration(cudaStream_t s, float* out) {
    hf_status st = calibrate(s);
    if (st != HF_OK) return st;
    out[0] = g_t_level_ns;
    out[1] = g_t_hop_ns;
    out[2] = g_t_team_solo_ns;
    out[3] = g_t_team_cluster_ns;
    out[4] = g_link_gbs[0];
    out[5] = g_link_gbs[1];
    out[6] = g_link_gbs[2];
    out[7] = g_r_level_ns;
    out[8] = g_r_team_ns;
    out[9] = g_r_cluster_ns;
    return HF_OK;
}

hf_status plan_predict(Plan* p, int32_t priority, const hf_costmodel* cm, cudaStream_t s, float* ls_ms, float* p_ms,
                       float* t_ms) {
    hf_status st = calibrate(s);
    if (st != HF_OK) return st;
    if (p->n == 0) {
        *ls_ms = *p_ms = *t_ms = 0.f;
        return HF_OK;
    }
    float* c = (float*)dev_alloc(sizeof(float) * (size_t)p->n, s);
    float* b = (float*)dev_alloc(sizeof(float) * (size_t)p->n, s);
    if (!c || !b) {
        dev_free(c, s);
        dev_free(b, s);
        return fail(HF_ENOMEM, "device allocation failed: prediction");
    }
    st = plan_task_costs(p, priority, cm, c, b, s);
    std::vector<float> hc, hb;
    if (st == HF_OK) {
        hc.resize((size_t)p->n);
        hb.resize((size_t)p->n);
        cudaError_t e = cudaMemcpy(hc.data(), c, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hb.data(), b, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "prediction download");
    }
    dev_free(c, s);
    dev_free(b, s);
    if (st != HF_OK) return st;
    double cp = 0.0, work = 0.0;
    // a level-synchronous level costs t_level plus its payload: its saxpy tasks split into
    // 512-element pieces spread over the level kernel's warps (at most 64 per SM), so the slowest
    // piece or the level's payload work over those warps, whichever is longer; a host task as a
    // whole (a max-plus task is one gather, part of t_level; copies run beside the levels on the
    // copy engines)
    std::vector<double> lmax((size_t)std::max(p->levels, 1), 0.0), lwork((size_t)std::max(p->levels, 1), 0.0);
    for (int32_t v = 0; v < p->n; ++v) {
        cp = std::max(cp, (double)hb[(size_t)v]);
        work += hc[(size_t)v];
        const uint8_t c = p->h_cat[(size_t)v];
        const size_t l = (size_t)p->h_level[(size_t)v];
        if (c == 1) {
            const double n = (double)std::max<int64_t>(p->hpay[(size_t)p->hpidx[(size_t)v]].n, 1);
            lmax[l] = std::max(lmax[l], (double)hc[(size_t)v] * std::min(1.0, 512.0 / n));
            lwork[l] += hc[(size_t)v];
        } else if (c == 4) {
            lmax[l] = std::max(lmax[l], (double)hc[(size_t)v]);
        }
    }
    const double ls_warps = 64.0 * (double)p->num_sms;
    for (size_t l = 0; l < lmax.size(); ++l) lmax[l] = std::max(lmax[l], lwork[l] / ls_warps);
    // the host link: every copy's bytes cross it, each direction at its measured bandwidth
    double link_bytes[2] = {0.0, 0.0};
    for (int32_t q = 0; q < p->npay; ++q)
        if (p->hpdir[(size_t)q]) link_bytes[p->hpdir[(size_t)q] - 1] += (double)p->hpay[(size_t)q].n;
    double link_ns = 0.0;
    for (int d = 0; d < 2; ++d)
        if (g_link_gbs[d] > 0.f) link_ns = std::max(link_ns, link_bytes[d] / (double)g_link_gbs[d]);
    if (g_link_gbs[2] > 0.f) link_ns = std::max(link_ns, (link_bytes[0] + link_bytes[1]) / (double)g_link_gbs[2]);
    double lsum = 0.0;
    for (double x : lmax) lsum += x;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<false>, kWarpsPerCta * 32, 0);
    const double warps = (double)p->num_sms * std::max(occ, 1) * kWarpsPerCta;
    // the calibration chain's levels come from L2; when the level-sorted arrays exceed half the
    // L2, every level's task list and in-edges come from DRAM first: three dependent DRAM round
    // trips per level instead of L2 ones (x2.5)
    int l2 = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const double ls_bytes = 8.0 * (double)p->m + 8.0 * (double)p->n;
    const double dram = ls_bytes > 0.5 * (double)l2 ? 2.5 : 1.0;
    // a merged level's gather: its in-edges over the SMs its CTAs (256 tasks each) occupy
    std::vector<double> lw((size_t)std::max(p->levels, 1), 0.0), le((size_t)std::max(p->levels, 1), 0.0);
    for (int32_t gi = 0; gi < p->ngraphs; ++gi)
        for (int32_t l = 0; l < p->glevels[(size_t)gi] && (size_t)l < lw.size(); ++l) {
            const int4& sg = p->h_seg[(size_t)(p->seg_first[(size_t)gi] + l)];
            lw[(size_t)l] += (double)(sg.y - sg.x);
            le[(size_t)l] += (double)(sg.w - sg.z);
        }
    double gather = 0.0;
    for (size_t l = 0; l < lw.size(); ++l)
        gather += le[l] / std::max(1.0, std::min(std::ceil(lw[l] / 256.0), (double)p->num_sms));
    *ls_ms = (float)(std::max((double)p->levels * dram * g_t_level_ns + g_r_level_ns * gather + lsum, link_ns) / 1e6);
    *p_ms = (float)(std::max(cp + (double)p->levels * g_t_hop_ns + work / warps, link_ns) / 1e6);
    // team executor: its own plan under the same cost source (host tasks: not available)
    *t_ms = INFINITY;
    if (p->host_tasks.empty()) {
        std::vector<int32_t> order;
        std::vector<int> k;
        double M = 0.0;
        const hf_costmodel* keep = p->cm;
        p->cm = cm;
        st = team_decide(p, priority, 0, (double)team_scale_default(priority), s, &k, &order, &M);
        p->cm = keep;
        if (st != HF_OK) return st;
        *t_ms = (float)(M / 1e6);
    }
    return HF_OK;
}

// Team executor: predicted time of graph g on a team of k CTAs (ns),
//   T_g(k) = sum over levels l of  t_lvl(k) * ceil(w_l / (256 k)) + r(k) * E_l / k + P_l / (8 k),
// w_l the level's task count, E_l its in-edges, P_l the summed predicted cost (warp-ns) of its
// payload tasks, t_lvl the measured time of a one-task level (CTA barrier for k = 1, cluster
// barrier else), r(k) the measured time per in-edge gathered on one SM.
constexpr int kTeamMaxCluster = 16;  // above 8 is a non-portable cluster size

static double team_time(const Plan* p, const std::vector<double>& pay_ns, int32_t g, int k, double scale = 1.0) {
    double t = 0.0;
    const double tl = k == 1 ? g_t_team_solo_ns : g_t_team_cluster_ns;
    const double re = k == 1 ? g_r_team_ns : g_r_cluster_ns;  // per in-edge gathered on one SM
    const int32_t s0 = p->seg_first[(size_t)g];
    for (int32_t l = 0; l < p->glevels[(size_t)g]; ++l) {
        const int4& sg = p->h_seg[(size_t)(s0 + l)];
        const int64_t w = sg.y - sg.x;
        // a level too large to stage reads its task list, row starts and in-edges from memory:
        // three dependent round trips instead of one
        const double stage = (w <= p->stage_n && sg.w - sg.z <= p->stage_e) ? 1.0 : 2.5;
        t += stage * tl * (double)((w + 256LL * k - 1) / (256LL * k)) + re * (double)(sg.w - sg.z) / k +
             scale * pay_ns[(size_t)(s0 + l)] / (8.0 * k);
    }
    return t;
}

// CTAs of cluster size k resident at once (k = 1: plain occupancy).
// the stage buffers (the kernel places its key table right after them: same sizes as TeamArgs)
static size_t team_smem(const Plan* p) {
    return kTeamBufs * team_stage_bytes(p->stage_n, p->stage_e, p->npay ? p->stage_p : 0);
}

// a class's dynamic shared memory: the stage buffers, then its key table (16-byte multiple)
static size_t team_class_smem(const Plan* p, int32_t key_cap) {
    return team_smem(p) + (((size_t)key_cap * 4 + 15) & ~(size_t)15);
}

// The team kernel's instantiations: payloads, cost recording, cluster class with shared keys.
static const void* team_kernel(bool pay, bool rec, bool csk) {
    if (csk) {
        if (rec) return pay ? (const void*)k_team<true, true, true> : (const void*)k_team<false, true, true>;
        return pay ? (const void*)k_team<true, false, true> : (const void*)k_team<false, false, true>;
    }
    if (rec) return pay ? (const void*)k_team<true, true> : (const void*)k_team<false, true>;
    return pay ? (const void*)k_team<true, false> : (const void*)k_team<false, false>;
}

static std::vector<const void*> team_kernels() {
    std::vector<const void*> v;
    for (int i = 0; i < 8; ++i) v.push_back(team_kernel(i & 1, (i >> 1) & 1, (i >> 2) & 1));
    return v;
}

static void team_smem_attr(const Plan* p, size_t need) {
    static std::mutex mu;
    static size_t set_to = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (need == 0) need = team_smem(p);
    if (need > set_to) {
        for (const void* f : team_kernels()) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        set_to = need;
    }
}

// smem: the class's dynamic shared memory (0: stage buffers only); csk: the class runs the
// kernel with every cluster job's keys in shared memory
static int team_capacity(const Plan* p, int k, size_t smem, bool csk) {
    const void* fn = team_kernel(p->npay != 0, false, csk);
    if (smem == 0) smem = team_smem(p);
    team_smem_attr(p, smem);
    if (k == 1) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTeamBlock, smem);
        return p->num_sms * std::max(occ, 1);
    }
    if (k > 8)
        for (const void* f : team_kernels()) cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)k);
    cfg.blockDim = dim3(kTeamBlock);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)k;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc * k;
}

// Team plan under a cost source: a team size k_g in {1, 2, 4, 8, 16} per graph (k > 1: a
// thread-block cluster, resident for the whole run). Predicted makespan
//   M = max( longest T_g(k_g),  sum of T_g(1) over single-CTA graphs / CTAs left to them ).
// Every graph starts on one CTA; the graph with the longest predicted time moves to the larger
// team (of those that fit) that lowers M most, while one does; the first time none does, the
// plan is final.
// `order` lists the graphs in decreasing predicted time. Planning multiplies the payload costs
// by `scale` (the slowdown of memory traffic when all graphs stream together); *M_out is the
// plan's makespan in unscaled costs, comparable with the other executors' predictions. FIFO:
// one CTA per graph in batch order, M = 0.
static hf_status team_decide(Plan* p, int32_t prio, int32_t ctas_opt, double scale, cudaStream_t s,
                             std::vector<int>* k_out, std::vector<int32_t>* order_out, double* M_out, int fold_k) {
    const int32_t G = p->ngraphs;
    std::vector<int32_t>& order = *order_out;
    std::vector<int>& k = *k_out;
    order.clear();
    k.assign((size_t)G, 1);
    for (int32_t g = 0; g < G; ++g)
        if (p->glevels[(size_t)g] > 0) order.push_back(g);
    *M_out = 0.0;
    if (prio == HF_PRIO_FIFO) return HF_OK;
    hf_status st = calibrate(s);
    if (st != HF_OK) return st;
    std::vector<double> pay_ns(p->h_seg.size(), 0.0);
    if (p->npay) {
        float* c = (float*)dev_alloc(sizeof(float) * (size_t)p->n, s);
        float* b = (float*)dev_alloc(sizeof(float) * (size_t)p->n, s);
        st = (!c || !b) ? fail(HF_ENOMEM, "device allocation failed: team costs")
                        : plan_task_costs(p, prio, p->cm, c, b, s);
        std::vector<float> hc;
        if (st == HF_OK) {
            hc.resize((size_t)p->n);
            cudaError_t e = cudaMemcpy(hc.data(), c, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "team cost download");
        }
        dev_free(c, s);
        dev_free(b, s);
        if (st != HF_OK) return st;
        for (int32_t q = 0; q < p->npay; ++q) {
            const int32_t t = p->pay_task[(size_t)q];
            const int32_t g = (int32_t)(std::upper_bound(p->task_off.begin(), p->task_off.end(), t) -
                                        p->task_off.begin()) - 1;
            pay_ns[(size_t)(p->seg_first[(size_t)g] + p->pay_level[(size_t)q])] += hc[(size_t)t];
        }
    }
    std::vector<double> T((size_t)G, 0.0);
    double work = 0.0;
    for (int32_t g : order) {
        T[(size_t)g] = team_time(p, pay_ns, g, 1, scale);
        work += T[(size_t)g];
    }
    int capk[17] = {0};
    for (int kk = 2; kk <= kTeamMaxCluster; kk *= 2)
        capk[kk] = ctas_opt > 0 || (fold_k > 0 && kk != fold_k) ? 0 : team_capacity(p, kk);
    // folded: one launch of fold_k-CTA clusters, whose CTAs also run the single-CTA graphs
    int cap1 = fold_k > 0 ? capk[fold_k] : team_capacity(p, 1);
    if (ctas_opt > 0) cap1 = std::min(cap1, ctas_opt);
    // predicted makespan: the longest team, or the single-CTA graphs' total over the CTAs left
    // to them (they queue when there are more of them than CTAs)
    int cl_ctas = 0, inclass[17] = {0};
    double solo_sum = work;
    int nsolo = (int)order.size();
    auto makespan = [&](double tmax, double ssum, int c1, int ns) {
        return std::max(tmax, ns > 0 ? ssum / (double)std::max(c1, 1) : 0.0);
    };
    using Item = std::pair<double, int32_t>;
    std::priority_queue<Item> heap;
    for (int32_t g : order) heap.push({T[(size_t)g], g});
    while (!heap.empty()) {
        const Item top = heap.top();
        const int32_t g = top.second;
        const int k0 = k[(size_t)g];
        heap.pop();
        const double next = heap.empty() ? 0.0 : heap.top().first;
        const int ns1 = nsolo - (k0 == 1 ? 1 : 0);
        const double ss1 = solo_sum - (k0 == 1 ? T[(size_t)g] : 0.0);
        const double m0 = makespan(top.first, solo_sum, cap1 - cl_ctas, nsolo);
        // every larger team that fits (a level's gather spreads over more SMs, but the first
        // doubling may not pay for the cluster barrier where a larger team does); the best one
        int k1 = 0, cl1 = 0;
        double t1 = 0.0, m1 = m0;
        for (int kk = fold_k > 0 ? (k0 == 1 ? fold_k : 2 * kTeamMaxCluster) : 2 * k0; kk <= kTeamMaxCluster;
             kk = fold_k > 0 ? 2 * kTeamMaxCluster : 2 * kk) {
            if ((inclass[kk] + 1) * kk > capk[kk]) continue;
            const int c = cl_ctas + kk - (k0 > 1 ? k0 : 0);
            if (c > cap1 - (ns1 > 0 ? 1 : 0)) continue;
            const double tk = team_time(p, pay_ns, g, kk, scale);
            const double mk = makespan(std::max(next, tk), ss1, cap1 - c, ns1);
            if (mk < m1) {
                k1 = kk;
                cl1 = c;
                t1 = tk;
                m1 = mk;
            }
        }
        if (k1 == 0) {  // no larger team of the longest graph shortens the makespan
            heap.push(top);
            break;
        }
        if (k0 > 1) inclass[k0] -= 1;
        inclass[k1] += 1;
        k[(size_t)g] = k1;
        T[(size_t)g] = t1;
        cl_ctas = cl1;
        nsolo = ns1;
        solo_sum = ss1;
        heap.push({t1, g});
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return T[(size_t)x] > T[(size_t)y]; });
    // the plan's makespan in unscaled costs (the units of the other executors' predictions)
    double tmax = 0.0, ssum = 0.0;
    for (int32_t g : order) {
        const double t = team_time(p, pay_ns, g, k[(size_t)g]);
        tmax = std::max(tmax, t);
        if (k[(size_t)g] == 1) ssum += t;
    }
    *M_out = makespan(tmax, ssum, cap1 - cl_ctas, nsolo);
    return HF_OK;
}

// Job lists for a run: one class per team size, each class one concurrent launch with every
// one of its graphs resident (k > 1: cluster jobs, one per cluster; k = 1: solo jobs, queued
// when there are more than CTAs). team_size k > 0: every graph in one class of min(k, 16).
static hf_status plan_team_jobs(Plan* p, const hf_run_opts& o, cudaStream_t s) {
    const int32_t prio = o.priority;
    const int32_t scale = o.team_scale != 0 ? o.team_scale : team_scale_default(prio);
    const int32_t fold = o.team_size > 0 ? 0 : o.team_fold;
    if (fold != 0 && fold != -1 && fold != 2 && fold != 4 && fold != 8 && fold != 16)
        return fail(HF_EINVAL, "team_fold must be 0, -1, 2, 4, 8 or 16");
    if (o.team_global_keys != 0 && o.team_global_keys != 1) return fail(HF_EINVAL, "team_global_keys must be 0 or 1");
    if (p->team_for[0] == prio && p->team_for[1] == o.team_size && p->team_for[2] == o.ctas &&
        p->team_for[3] == scale && p->team_for[4] == fold && p->team_for[5] == o.team_global_keys &&
        (prio != HF_PRIO_LEARNED || p->team_cm == p->cm))
        return HF_OK;
    std::vector<int32_t> order;
    std::vector<int> k;
    double M = 0.0;
    const int32_t dprio = o.team_size > 0 ? HF_PRIO_FIFO : prio;
    int fold_k = fold;
    hf_status st = HF_OK;
    if (fold == -1) {  // one launch: the cluster size whose plan has the smallest predicted makespan
        double best = INFINITY;
        for (int kk = 2; kk <= kTeamMaxCluster && st == HF_OK; kk *= 2) {
            std::vector<int32_t> o2;
            std::vector<int> k2;
            double m2 = 0.0;
            if (team_capacity(p, kk) < kk) continue;
            st = team_decide(p, dprio, o.ctas, team_scale_factor(scale, prio), s, &k2, &o2, &m2, kk);
            if (st == HF_OK && m2 < best) {
                best = m2;
                fold_k = kk;
                k.swap(k2);
                order.swap(o2);
                M = m2;
            }
        }
        if (st == HF_OK && fold_k < 0) fold_k = 0;  // no cluster fits: single CTAs
        if (st == HF_OK && fold_k == 0)
            st = team_decide(p, dprio, o.ctas, team_scale_factor(scale, prio), s, &k, &order, &M);
    } else {
        st = team_decide(p, dprio, o.ctas, team_scale_factor(scale, prio), s, &k, &order, &M, fold_k);
    }
    if (st != HF_OK) return st;
    if (o.team_size > 0)
        for (auto& x : k) x = std::min(o.team_size, kTeamMaxCluster);
    p->team_k.assign((size_t)p->ngraphs, 0);
    for (int32_t g : order) p->team_k[(size_t)g] = k[(size_t)g];
    std::vector<TeamJob> jobs;
    p->tclass.clear();
    int cap1 = team_capacity(p, 1);
    if (o.ctas > 0) cap1 = std::min(cap1, o.ctas);
    int nclustered = 0;
    for (int32_t g : order) nclustered += k[(size_t)g] > 1 ? 1 : 0;
    if (fold_k > 0 && nclustered > 0) {
        // one launch with cluster size fold_k: its cluster jobs first, then every single-CTA job
        Plan::TeamClass c{fold_k, 0, 0, 0, 0};
        for (int32_t g : order)
            if (k[(size_t)g] == fold_k) jobs.push_back(TeamJob{g, 0, p->seg_first[(size_t)g], p->glevels[(size_t)g]});
        c.ncjobs = (int32_t)jobs.size();
        for (int32_t g : order)
            if (k[(size_t)g] == 1) jobs.push_back(TeamJob{g, 0, p->seg_first[(size_t)g], p->glevels[(size_t)g]});
        c.njobs = (int32_t)jobs.size();
        const int capk = team_capacity(p, fold_k);
        if (capk < fold_k) return fail(HF_ENOTSUP, "no resident cluster of " + std::to_string(fold_k) + " CTAs");
        const int want = c.ncjobs * fold_k + (c.njobs - c.ncjobs);
        c.grid = std::min((want + fold_k - 1) / fold_k, capk / fold_k) * fold_k;
        p->tclass.push_back(c);
    } else {
        int used = 0;
        for (int kk = kTeamMaxCluster; kk >= 1; --kk) {
            Plan::TeamClass c{kk, (int32_t)jobs.size(), 0, 0, 0};
            for (int32_t g : order)
                if (k[(size_t)g] == kk) jobs.push_back(TeamJob{g, 0, p->seg_first[(size_t)g], p->glevels[(size_t)g]});
            c.njobs = (int32_t)jobs.size() - c.job0;
            if (c.njobs == 0) continue;
            c.ncjobs = kk > 1 ? c.njobs : 0;
            if (kk > 1) {
                const int capk = team_capacity(p, kk);
                if (capk < kk) return fail(HF_ENOTSUP, "no resident cluster of " + std::to_string(kk) + " CTAs");
                c.grid = std::min(c.njobs * kk, (capk / kk) * kk);
            } else {
                c.grid = std::max(1, std::min(c.njobs, std::max(cap1 - used, 1)));
            }
            used += c.grid;
            p->tclass.push_back(c);
        }
    }
    if (p->tclass.size() > 5) return fail(HF_ENOTSUP, "too many team classes");
    for (TeamJob& j : jobs) {
        if (p->task_off[(size_t)j.graph + 1] - p->task_off[(size_t)j.graph] >= kPipeMinTasks) j.flags |= kJobPipelined;
        if (p->pay_local[(size_t)j.graph]) j.flags |= kJobPayloadLocal;
    }
    // Keys in distributed shared memory (team.cuh), per cluster class of a power-of-two size, in
    // batches without payloads, the largest clusters first. A key table of `cap` entries per CTA
    // must leave every CTA of the class resident and the shared memory of all classes' CTAs
    // together within 90 % of the GPU's (the classes run concurrently). When the largest share of
    // the class's graphs (ceil(n_g / k)) fits, the class runs the kernel with shared keys only
    // (every graph); otherwise the largest share that fits, for the graphs whose share fits. Not
    // for single CTAs, not in folded launches, and not with payloads: on batch256_mixed the
    // payload kernel with shared keys (118 registers, two CTAs per SM) ran its 2-CTA class so
    // much slower that the step took 4.74 instead of 3.28-3.48 ms.
    bool any_sk = false;
    p->team_sk.assign((size_t)p->ngraphs, 0);
    for (Plan::TeamClass& c : p->tclass) c.key_cap = c.csk = 0;
    if (fold_k == 0 && p->npay == 0 && o.team_global_keys == 0) {
        int max_dyn = 0, sm_smem = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        size_t stat = 0;
        for (const void* f : team_kernels()) {
            cudaFuncAttributes fa = {};
            cudaFuncGetAttributes(&fa, f);
            stat = std::max(stat, fa.sharedSizeBytes);
        }
        const size_t dyn_cap = (size_t)std::max(max_dyn - (int)stat, 0);
        const size_t per_cta = stat + 1024;  // static shared memory + the CTA's reserve
        const double budget = 0.9 * (double)p->num_sms * (double)sm_smem;
        double used = 0.0;
        for (const Plan::TeamClass& c : p->tclass) used += (double)c.grid * (double)(team_smem(p) + per_cta);
        auto share_of = [&](const Plan::TeamClass& c, int32_t j) {
            const int32_t g = jobs[(size_t)j].graph;
            return (p->task_off[(size_t)g + 1] - p->task_off[(size_t)g] + c.k - 1) / c.k;
        };
        auto fits = [&](const Plan::TeamClass& c, int32_t cap, bool csk, double* grow) {
            const size_t smem = team_class_smem(p, cap);
            if (smem > dyn_cap) return false;
            *grow = (double)c.grid * (double)(smem - team_smem(p));
            return used + *grow <= budget && team_capacity(p, c.k, smem, csk) >= c.grid;
        };
        for (Plan::TeamClass& c : p->tclass) {
            if (c.k == 1 || (c.k & (c.k - 1)) || c.njobs == 0) continue;
            std::vector<int32_t> share;
            for (int32_t j = c.job0; j < c.job0 + c.njobs; ++j) share.push_back(share_of(c, j));
            std::sort(share.begin(), share.end(), std::greater<int32_t>());
            share.erase(std::unique(share.begin(), share.end()), share.end());
            double grow = 0.0;
            if (fits(c, share[0], true, &grow)) {
                c.key_cap = share[0];
                c.csk = 1;
                used += grow;
            } else {
                for (size_t q = 0; q < share.size(); ++q)
                    if (fits(c, share[q], false, &grow)) {
                        c.key_cap = share[q];
                        used += grow;
                        break;
                    }
            }
            for (int32_t j = c.job0; j < c.job0 + c.njobs; ++j) {
                if (c.key_cap > 0 && share_of(c, j) <= c.key_cap) jobs[(size_t)j].flags |= kJobSharedKeys;
                p->team_sk[(size_t)jobs[(size_t)j].graph] = jobs[(size_t)j].flags & kJobSharedKeys;
                any_sk |= (jobs[(size_t)j].flags & kJobSharedKeys) != 0;
            }
        }
    }
    if (any_sk && !p->d_toff) {
        hf_status su = upload(p, &p->d_toff, p->task_off.data(), p->task_off.size(), s, "task offsets");
        if (su != HF_OK) return su;
    }
    const size_t bytes = std::max<size_t>(sizeof(TeamJob) * jobs.size(), 16);
    if (p->cap_jobs < bytes) {
        free_owned(p, p->d_jobs);
        p->d_jobs = (TeamJob*)palloc(p, bytes, s);
        p->cap_jobs = p->d_jobs ? bytes : 0;
        if (!p->d_jobs) return fail(HF_ENOMEM, "device allocation failed: team jobs");
    }
    if (!p->d_team) {
        p->d_team = (int32_t*)palloc(p, sizeof(int32_t) * (size_t)kTeamWords * 5, s);
        if (!p->d_team) return fail(HF_ENOMEM, "device allocation failed: team control");
    }
    if (!p->tev_fork) {
        // the classes run on a stream at the device's highest priority, above the default priority
        // of the plan's helper streams (the next view's delay gather)
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->tev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->tstream[0], cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->tev_join[0], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "team streams");
    }
    cudaError_t e = cudaSuccess;
    if (!jobs.empty()) e = cudaMemcpyAsync(p->d_jobs, jobs.data(), sizeof(TeamJob) * jobs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "team job upload");
    p->njobs = (int32_t)jobs.size();
    p->team_for[0] = prio;
    p->team_for[1] = o.team_size;
    p->team_for[2] = o.ctas;
    p->team_for[3] = scale;
    p->team_for[4] = fold;
    p->team_for[5] = o.team_global_keys;
    p->team_cm = p->cm;
    return HF_OK;
}

hf_status plan_auto_mode(Plan* p, cudaStream_t s, int* mode) {
    if (p->auto_mode >= 0 && p->auto_cm == p->cm) {
        *mode = p->auto_mode;
        return HF_OK;
    }
    float ls = 0.f, pe = 0.f, tm = 0.f;
    hf_status st = plan_predict(p, p->cm ? HF_PRIO_LEARNED : HF_PRIO_HEURISTIC, p->cm, s, &ls, &pe, &tm);
    if (st != HF_OK) return st;
    p->auto_mode = pe <= ls ? HF_MODE_PERSISTENT : HF_MODE_LEVELSYNC;
    if (tm < std::min(ls, pe)) p->auto_mode = HF_MODE_TEAM;
    p->auto_cm = p->cm;
    *mode = p->auto_mode;
    return HF_OK;
}

}  // namespace hf
