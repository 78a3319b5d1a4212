// api.cpp -- C ABI entry points: graph construction (Section III-A of the paper: tasks of four
// kinds, explicit edges, acyclic graphs), host-side finalization (successor CSR, level-sorted
// predecessor lists, in-degrees, topological levels, cycle check), batches, the allocator hook
// and error reporting. Execution lives in plan.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "hf_internal.h"

namespace hf {

static thread_local std::string g_err;

hf_status fail(hf_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

hf_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return HF_ECUDA;
}

static std::mutex g_alloc_mu;
static hf_alloc_fn g_alloc = nullptr;
static hf_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    hf_alloc_fn a;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (a) return a(bytes, (void*)s, ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, cudaStream_t s) {
    if (!p) return;
    hf_free_fn f;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f) {
        f(p, (void*)s, ctx);
        return;
    }
    cudaFree(p);
}

// Kahn pass over the successor CSR: levels (longest hop count from a source) and cycle check.
static hf_status finalize_graph(hf_graph* g) {
    Final& f = g->fin;
    const int64_t n64 = (int64_t)g->kind.size();
    const int64_t m = (int64_t)g->esrc.size();
    if (n64 > INT32_MAX - 1) return fail(HF_EINVAL, "too many tasks (max 2^31-2)");
    if (m > INT32_MAX) return fail(HF_EINVAL, "too many edges (max 2^31-1)");
    const int32_t n = (int32_t)n64;
    f = Final();
    f.n = n;
    f.m = m;
    try {
        f.row_ptr.assign((size_t)n + 1, 0);
        f.indeg0.assign((size_t)n, 0);
        for (int64_t e = 0; e < m; ++e) {
            f.row_ptr[(size_t)g->esrc[e] + 1]++;
            f.indeg0[(size_t)g->edst[e]]++;
        }
        for (int32_t v = 0; v < n; ++v) f.row_ptr[v + 1] += f.row_ptr[v];
        f.succ.resize((size_t)m);
        f.epos_csr.resize((size_t)m);
        f.epos_ls.resize((size_t)m);
        {
            std::vector<int32_t> fill(f.row_ptr.begin(), f.row_ptr.end() - 1);
            for (int64_t e = 0; e < m; ++e) {
                int2 x;
                x.x = g->edst[e];
                float d = g->edly[e];
                std::memcpy(&x.y, &d, 4);
                const int32_t at = fill[g->esrc[e]]++;
                f.succ[(size_t)at] = x;
                f.epos_csr[(size_t)e] = at;
            }
        }
        // Kahn: levels and cycle detection
        f.level.assign((size_t)n, 0);
        std::vector<int32_t> pend(f.indeg0);
        std::vector<int32_t> q;
        q.reserve((size_t)n);
        for (int32_t v = 0; v < n; ++v)
            if (pend[v] == 0) q.push_back(v);
        f.nsrc = (int32_t)q.size();
        int32_t maxlev = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            const int32_t u = q[h];
            const int32_t lu = f.level[u];
            for (int32_t e = f.row_ptr[u]; e < f.row_ptr[u + 1]; ++e) {
                const int32_t v = f.succ[e].x;
                if (f.level[v] < lu + 1) f.level[v] = lu + 1;
                if (--pend[v] == 0) q.push_back(v);
            }
            if (lu > maxlev) maxlev = lu;
        }
        if ((int64_t)q.size() != n) {
            f = Final();
            return fail(HF_ECYCLE, "dependency edges form a cycle (" + std::to_string(n - (int64_t)q.size()) +
                                       " tasks never become ready)");
        }
        f.levels = n ? maxlev + 1 : 0;
        // tasks sorted by (level, id)
        f.level_ptr.assign((size_t)f.levels + 1, 0);
        for (int32_t v = 0; v < n; ++v) f.level_ptr[f.level[v] + 1]++;
        for (int32_t l = 0; l < f.levels; ++l) f.level_ptr[l + 1] += f.level_ptr[l];
        f.ls_node.resize((size_t)n);
        std::vector<int32_t> pos((size_t)n);
        {
            std::vector<int32_t> fill(f.level_ptr.begin(), f.level_ptr.end() - 1);
            for (int32_t v = 0; v < n; ++v) {
                const int32_t p = fill[f.level[v]]++;
                f.ls_node[p] = v;
                pos[v] = p;
            }
        }
        f.ls_ptr.assign((size_t)n + 1, 0);
        for (int32_t p = 0; p < n; ++p) f.ls_ptr[p + 1] = f.ls_ptr[p] + f.indeg0[f.ls_node[p]];
        f.ls_in.resize((size_t)m);
        {
            std::vector<int32_t> fill(f.ls_ptr.begin(), f.ls_ptr.end() - 1);
            for (int64_t e = 0; e < m; ++e) {
                int2 x;
                x.x = g->esrc[e];
                float d = g->edly[e];
                std::memcpy(&x.y, &d, 4);
                const int32_t at = fill[pos[g->edst[e]]]++;
                f.ls_in[(size_t)at] = x;
                f.epos_ls[(size_t)e] = at;
            }
        }
    } catch (const std::bad_alloc&) {
        f = Final();
        return fail(HF_ENOMEM, "host allocation failed in finalize");
    }
    g->dirty = false;
    return HF_OK;
}

static hf_status check_mutable(hf_graph* g) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (g->in_batches > 0) return fail(HF_ESTATE, "graph belongs to a batch; destroy the batch first");
    if (g->plan && plan_busy(g->plan) != HF_OK) return fail(HF_ESTATE, "a run of this graph is in flight");
    return HF_OK;
}

static bool valid_task(const hf_graph* g, int64_t t) { return t >= 0 && t < (int64_t)g->kind.size(); }

static bool is_pull(const hf_graph* g, int64_t t) { return valid_task(g, t) && g->kind[(size_t)t] == HF_PULL; }

static void mark_dirty(hf_graph* g) { g->dirty = true; }

}  // namespace hf

using namespace hf;

extern "C" {

void hf_run_opts_default(hf_run_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = HF_MODE_PERSISTENT;
    o->priority = HF_PRIO_FIFO;
    o->claim = 8;
    o->local_keep = -1;
    o->stall_task = -1;
}

const char* hf_status_string(hf_status s) {
    switch (s) {
        case HF_OK: return "HF_OK";
        case HF_EINVAL: return "HF_EINVAL: invalid argument";
        case HF_ENOMEM: return "HF_ENOMEM: out of memory";
        case HF_ECYCLE: return "HF_ECYCLE: dependency cycle";
        case HF_ESTATE: return "HF_ESTATE: invalid state for this call";
        case HF_ETIMEDOUT: return "HF_ETIMEDOUT: executor made no progress within the spin limit";
        case HF_EQUEUE: return "HF_EQUEUE: device queue overflow";
        case HF_ECUDA: return "HF_ECUDA: CUDA runtime error";
        case HF_ENOTSUP: return "HF_ENOTSUP: not supported";
    }
    return "unknown hf_status";
}

const char* hf_last_error(void) { return g_err.c_str(); }

hf_status hf_set_allocator(hf_alloc_fn a, hf_free_fn f, void* ctx) {
    if ((a == nullptr) != (f == nullptr)) return fail(HF_EINVAL, "allocator and free must both be set or both NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = a;
    g_free = f;
    g_alloc_ctx = ctx;
    return HF_OK;
}

hf_status hf_graph_create(hf_graph** out, int64_t reserve_tasks, int64_t reserve_edges) {
    if (!out) return fail(HF_EINVAL, "out is NULL");
    *out = nullptr;
    if (reserve_tasks < 0 || reserve_edges < 0) return fail(HF_EINVAL, "negative reservation");
    try {
        hf_graph* g = new hf_graph();
        g->kind.reserve((size_t)reserve_tasks);
        g->arr0.reserve((size_t)reserve_tasks);
        g->pay.reserve((size_t)reserve_tasks);
        g->esrc.reserve((size_t)reserve_edges);
        g->edst.reserve((size_t)reserve_edges);
        g->edly.reserve((size_t)reserve_edges);
        *out = g;
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    return HF_OK;
}

hf_status hf_graph_destroy(hf_graph* g) {
    if (!g) return HF_OK;
    if (g->in_batches > 0) return fail(HF_ESTATE, "graph belongs to a batch; destroy the batch first");
    if (g->plan) plan_destroy(g->plan);
    delete g;
    return HF_OK;
}

hf_status hf_add_task(hf_graph* g, hf_kind kind, const void* payload, size_t payload_bytes, hf_task* out) {
    hf_status st = check_mutable(g);
    if (st != HF_OK) return st;
    if (g->kind.size() >= (size_t)INT32_MAX - 1) return fail(HF_EINVAL, "too many tasks");
    PayloadRec rec;
    rec.kind = kind;
    float arr0 = 0.f;
    bool has_pay = false;
    switch (kind) {
        case HF_KERNEL: {
            if (!payload) break;
            if (payload_bytes < sizeof(int32_t)) return fail(HF_EINVAL, "kernel payload too small");
            int32_t op;
            std::memcpy(&op, payload, sizeof(op));
            if (op == HF_K_MAXPLUS) {
                if (payload_bytes < sizeof(hf_maxplus_payload)) return fail(HF_EINVAL, "max-plus payload too small");
                hf_maxplus_payload p;
                std::memcpy(&p, payload, sizeof(p));
                if (!std::isfinite(p.arr0)) return fail(HF_EINVAL, "arr0 must be finite");
                arr0 = p.arr0;
            } else if (op == HF_K_SAXPY_F32 || op == HF_K_SAXPY_I32) {
                if (payload_bytes < sizeof(hf_saxpy_payload)) return fail(HF_EINVAL, "saxpy payload too small");
                hf_saxpy_payload p;
                std::memcpy(&p, payload, sizeof(p));
                if (p.n < 0) return fail(HF_EINVAL, "saxpy n < 0");
                const int64_t need = p.n * 4;
                if (p.x_pull >= 0) {
                    if (!is_pull(g, p.x_pull)) return fail(HF_EINVAL, "x_pull is not a pull task");
                    if ((int64_t)g->payloads[(size_t)g->pay[(size_t)p.x_pull]].bytes < need)
                        return fail(HF_EINVAL, "x_pull buffer smaller than n elements");
                } else if (p.x_pull != -1) {
                    return fail(HF_EINVAL, "x_pull must be a pull task id or -1");
                } else if (p.n > 0 && (!p.x_dev || ((uintptr_t)p.x_dev & 3))) {
                    return fail(HF_EINVAL, "x_dev NULL or not 4-byte aligned");
                }
                if (p.y_pull >= 0) {
                    if (!is_pull(g, p.y_pull)) return fail(HF_EINVAL, "y_pull is not a pull task");
                    if ((int64_t)g->payloads[(size_t)g->pay[(size_t)p.y_pull]].bytes < need)
                        return fail(HF_EINVAL, "y_pull buffer smaller than n elements");
                } else if (p.y_pull != -1) {
                    return fail(HF_EINVAL, "y_pull must be a pull task id or -1");
                } else if (p.n > 0 && (!p.y_dev || ((uintptr_t)p.y_dev & 3))) {
                    return fail(HF_EINVAL, "y_dev NULL or not 4-byte aligned");
                }
                rec.op = op;
                rec.n = p.n;
                rec.a_f = p.a_f;
                rec.a_i = p.a_i;
                rec.x_pull = p.x_pull;
                rec.y_pull = p.y_pull;
                rec.x_dev = p.x_dev;
                rec.y_dev = p.y_dev;
                has_pay = true;
            } else {
                return fail(HF_EINVAL, "unknown kernel op");
            }
            break;
        }
        case HF_PULL: {
            if (!payload || payload_bytes < sizeof(hf_pull_payload)) return fail(HF_EINVAL, "pull payload missing");
            hf_pull_payload p;
            std::memcpy(&p, payload, sizeof(p));
            if (p.bytes > 0 && !p.host_ptr) return fail(HF_EINVAL, "pull host_ptr is NULL");
            rec.host_src = p.host_ptr;
            rec.bytes = p.bytes;
            has_pay = true;
            break;
        }
        case HF_PUSH: {
            if (!payload || payload_bytes < sizeof(hf_push_payload)) return fail(HF_EINVAL, "push payload missing");
            hf_push_payload p;
            std::memcpy(&p, payload, sizeof(p));
            if (p.bytes > 0 && !p.host_ptr) return fail(HF_EINVAL, "push host_ptr is NULL");
            if (p.src_pull >= 0) {
                if (!is_pull(g, p.src_pull)) return fail(HF_EINVAL, "src_pull is not a pull task");
                if (g->payloads[(size_t)g->pay[(size_t)p.src_pull]].bytes < p.bytes)
                    return fail(HF_EINVAL, "push larger than its pull's buffer");
            } else if (p.src_pull != -1) {
                return fail(HF_EINVAL, "src_pull must be a pull task id or -1");
            } else if (p.bytes > 0 && !p.src_dev) {
                return fail(HF_EINVAL, "push src_dev is NULL");
            }
            rec.src_pull = p.src_pull;
            rec.src_dev = p.src_dev;
            rec.host_dst = p.host_ptr;
            rec.bytes = p.bytes;
            has_pay = true;
            break;
        }
        case HF_HOST: {
            if (!payload || payload_bytes < sizeof(hf_host_payload)) return fail(HF_EINVAL, "host payload missing");
            hf_host_payload p;
            std::memcpy(&p, payload, sizeof(p));
            if (!p.fn) return fail(HF_EINVAL, "host fn is NULL");
            rec.fn = p.fn;
            rec.arg = p.arg;
            has_pay = true;
            break;
        }
        default:
            return fail(HF_EINVAL, "unknown task kind");
    }
    try {
        const int32_t id = (int32_t)g->kind.size();
        int32_t pidx = -1;
        if (has_pay) {
            pidx = (int32_t)g->payloads.size();
            g->payloads.push_back(rec);
        }
        g->kind.push_back((uint8_t)kind);
        g->arr0.push_back(arr0);
        g->pay.push_back(pidx);
        if (arr0 != 0.f || std::signbit(arr0)) g->any_arr0 = true;
        if (out) *out = id;
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    mark_dirty(g);
    return HF_OK;
}

hf_status hf_add_tasks_bulk(hf_graph* g, int64_t n, const float* arr0, hf_task* first_out) {
    hf_status st = check_mutable(g);
    if (st != HF_OK) return st;
    if (n < 0) return fail(HF_EINVAL, "n < 0");
    if ((int64_t)g->kind.size() + n > (int64_t)INT32_MAX - 1) return fail(HF_EINVAL, "too many tasks");
    if (arr0)
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(arr0[i])) return fail(HF_EINVAL, "arr0 must be finite");
    try {
        const int32_t first = (int32_t)g->kind.size();
        g->kind.resize(g->kind.size() + (size_t)n, (uint8_t)HF_KERNEL);
        g->pay.resize(g->pay.size() + (size_t)n, -1);
        if (arr0) {
            g->arr0.insert(g->arr0.end(), arr0, arr0 + n);
            for (int64_t i = 0; i < n && !g->any_arr0; ++i)
                if (arr0[i] != 0.f || std::signbit(arr0[i])) g->any_arr0 = true;
        } else {
            g->arr0.resize(g->arr0.size() + (size_t)n, 0.f);
        }
        if (first_out) *first_out = first;
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    mark_dirty(g);
    return HF_OK;
}

hf_status hf_precede_w(hf_graph* g, hf_task a, hf_task b, float delay) {
    hf_status st = check_mutable(g);
    if (st != HF_OK) return st;
    if (!valid_task(g, a) || !valid_task(g, b)) return fail(HF_EINVAL, "task id out of range");
    if (!std::isfinite(delay)) return fail(HF_EINVAL, "delay must be finite");
    if ((int64_t)g->esrc.size() >= (int64_t)INT32_MAX) return fail(HF_EINVAL, "too many edges");
    try {
        g->esrc.push_back(a);
        g->edst.push_back(b);
        g->edly.push_back(delay);
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    mark_dirty(g);
    return HF_OK;
}

hf_status hf_precede(hf_graph* g, hf_task a, hf_task b) { return hf_precede_w(g, a, b, 0.f); }

hf_status hf_precede_bulk(hf_graph* g, int64_t m, const int32_t* src, const int32_t* dst, const float* delay) {
    hf_status st = check_mutable(g);
    if (st != HF_OK) return st;
    if (m < 0 || (m > 0 && (!src || !dst))) return fail(HF_EINVAL, "bad edge arrays");
    if ((int64_t)g->esrc.size() + m > (int64_t)INT32_MAX) return fail(HF_EINVAL, "too many edges");
    const int64_t n = (int64_t)g->kind.size();
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n)
            return fail(HF_EINVAL, "edge " + std::to_string(i) + ": task id out of range");
        if (delay && !std::isfinite(delay[i])) return fail(HF_EINVAL, "edge " + std::to_string(i) + ": delay not finite");
    }
    try {
        g->esrc.insert(g->esrc.end(), src, src + m);
        g->edst.insert(g->edst.end(), dst, dst + m);
        if (delay) g->edly.insert(g->edly.end(), delay, delay + m);
        else g->edly.resize(g->edly.size() + (size_t)m, 0.f);
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    mark_dirty(g);
    return HF_OK;
}

hf_status hf_finalize(hf_graph* g) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (!g->dirty) return HF_OK;
    hf_status st = check_mutable(g);
    if (st != HF_OK) return st;
    return finalize_graph(g);
}

hf_status hf_graph_info(const hf_graph* g, hf_graph_info_t* info) {
    if (!g || !info) return fail(HF_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->tasks = (int64_t)g->kind.size();
    info->edges = (int64_t)g->esrc.size();
    for (uint8_t k : g->kind) info->kind_count[k & 3]++;
    for (const auto& p : g->payloads)
        if (p.kind != HF_HOST) info->payload_tasks++;
    info->finalized = g->dirty ? 0 : 1;
    if (!g->dirty) {
        info->levels = g->fin.levels;
        info->sources = g->fin.nsrc;
    }
    return HF_OK;
}

hf_status hf_get_levels(const hf_graph* g, int32_t* level_out) {
    if (!g || !level_out) return fail(HF_EINVAL, "NULL argument");
    if (g->dirty) return fail(HF_ESTATE, "graph not finalized");
    if (g->fin.n) std::memcpy(level_out, g->fin.level.data(), sizeof(int32_t) * (size_t)g->fin.n);
    return HF_OK;
}

// Graphviz text of the graph: one node per task labelled with its id and kind (saxpy: size;
// copies: bytes; max-plus: source arrival when it has one), one edge per dependency labelled
// with its delay (%.9g round-trips binary32).
hf_status hf_dump(const hf_graph* g, const char* path) {
    if (!g || !path) return fail(HF_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(HF_EINVAL, std::string("cannot open ") + path);
    std::fprintf(f, "digraph hf {\n  node [shape=box];\n");
    for (size_t v = 0; v < g->kind.size(); ++v) {
        const int k = g->kind[v];
        const int32_t pi = g->pay[v];
        const hf::PayloadRec* r = pi >= 0 ? &g->payloads[(size_t)pi] : nullptr;
        char label[96];
        if (k == HF_KERNEL && r && r->op != HF_K_MAXPLUS)
            std::snprintf(label, sizeof label, "%zu saxpy%s n=%lld", v, r->op == HF_K_SAXPY_I32 ? "_i32" : "",
                          (long long)r->n);
        else if (k == HF_KERNEL)
            std::snprintf(label, sizeof label, "%zu maxplus arr0=%.9g", v, g->arr0.empty() ? 0.0 : (double)g->arr0[v]);
        else if (k == HF_PULL && r)
            std::snprintf(label, sizeof label, "%zu pull %zu B", v, r->bytes);
        else if (k == HF_PUSH && r)
            std::snprintf(label, sizeof label, "%zu push %zu B", v, r->bytes);
        else
            std::snprintf(label, sizeof label, "%zu host", v);
        std::fprintf(f, "  t%zu [label=\"%s\"];\n", v, label);
    }
    for (size_t e = 0; e < g->esrc.size(); ++e)
        std::fprintf(f, "  t%d -> t%d [label=\"%.9g\"];\n", g->esrc[e], g->edst[e], (double)g->edly[e]);
    std::fprintf(f, "}\n");
    const bool ok = std::fclose(f) == 0;
    return ok ? HF_OK : fail(HF_EINVAL, std::string("write failed: ") + path);
}

// ----------------------------------------------------------------------- device placement

// Heuristic task cost on the host (the same formula as the device's heuristic cost model):
// 300 ns + 30 ns per out-edge + payload bytes at 8 bytes/ns (saxpy 12 bytes per element,
// copies their bytes twice).
static double host_heuristic_cost(const hf_graph* g, int32_t v, int32_t fanout) {
    double bytes = 0.0;
    const int32_t pi = g->pay[(size_t)v];
    if (pi >= 0) {
        const hf::PayloadRec& r = g->payloads[(size_t)pi];
        if (r.kind == HF_KERNEL && r.op != HF_K_MAXPLUS) bytes = 12.0 * (double)r.n;
        else if (r.kind == HF_PULL || r.kind == HF_PUSH) bytes = 2.0 * (double)r.bytes;
    }
    return 300.0 + 30.0 * fanout + bytes / 8.0;
}

static int32_t uf_find(std::vector<int32_t>& up, int32_t x) {
    while (up[(size_t)x] != x) {
        up[(size_t)x] = up[(size_t)up[(size_t)x]];
        x = up[(size_t)x];
    }
    return x;
}

// Greedy longest-processing-time packing: items in decreasing cost (ties: lower index first),
// each onto the least-loaded device (ties: lower device).
static void lpt_pack(const std::vector<double>& cost, int32_t ndev, std::vector<int32_t>* dev, std::vector<double>* load) {
    std::vector<int32_t> order(cost.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[(size_t)a] > cost[(size_t)b]; });
    load->assign((size_t)ndev, 0.0);
    dev->assign(cost.size(), 0);
    for (int32_t i : order) {
        int32_t best = 0;
        for (int32_t d = 1; d < ndev; ++d)
            if ((*load)[(size_t)d] < (*load)[(size_t)best]) best = d;
        (*dev)[(size_t)i] = best;
        (*load)[(size_t)best] += cost[(size_t)i];
    }
}

hf_status hf_place(const hf_graph* g, int32_t ndev, const float* cost, int32_t* dev_out) {
    if (!g || !dev_out) return fail(HF_EINVAL, "NULL argument");
    if (ndev < 1) return fail(HF_EINVAL, "ndev < 1");
    const int32_t n = (int32_t)g->kind.size();
    try {
        // groups: a kernel task with the pulls it reads or writes, a push with the pull it reads
        std::vector<int32_t> up((size_t)n);
        for (int32_t v = 0; v < n; ++v) up[(size_t)v] = v;
        auto unite = [&](int32_t a, int32_t b) {
            a = uf_find(up, a);
            b = uf_find(up, b);
            if (a != b) up[(size_t)std::max(a, b)] = std::min(a, b);
        };
        std::vector<int32_t> fanout((size_t)n, 0);
        for (int32_t u : g->esrc) fanout[(size_t)u] += 1;
        for (int32_t v = 0; v < n; ++v) {
            const int32_t pi = g->pay[(size_t)v];
            if (pi < 0) continue;
            const hf::PayloadRec& r = g->payloads[(size_t)pi];
            if (r.kind == HF_KERNEL && r.op != HF_K_MAXPLUS) {
                if (r.x_pull >= 0) unite(v, r.x_pull);
                if (r.y_pull >= 0) unite(v, r.y_pull);
            } else if (r.kind == HF_PUSH && r.src_pull >= 0) {
                unite(v, r.src_pull);
            }
        }
        // group costs, then LPT over the groups (host tasks stay on the CPU: -1)
        std::vector<int32_t> gid((size_t)n, -1), root_gid((size_t)n, -1);
        std::vector<double> gcost;
        for (int32_t v = 0; v < n; ++v) {
            if (g->kind[(size_t)v] == HF_HOST) continue;
            const int32_t r = uf_find(up, v);
            if (root_gid[(size_t)r] < 0) {
                root_gid[(size_t)r] = (int32_t)gcost.size();
                gcost.push_back(0.0);
            }
            gid[(size_t)v] = root_gid[(size_t)r];
            gcost[(size_t)gid[(size_t)v]] += cost ? (double)cost[v] : host_heuristic_cost(g, v, fanout[(size_t)v]);
        }
        std::vector<int32_t> gdev;
        std::vector<double> load;
        lpt_pack(gcost, ndev, &gdev, &load);
        for (int32_t v = 0; v < n; ++v) dev_out[v] = gid[(size_t)v] < 0 ? -1 : gdev[(size_t)gid[(size_t)v]];
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    return HF_OK;
}

static hf_status ensure_plan(hf_graph* g) {
    if (g->dirty) {
        if (g->in_batches > 0) return fail(HF_ESTATE, "graph belongs to a batch");
        hf_status st = finalize_graph(g);
        if (st != HF_OK) return st;
    }
    if (g->plan) return HF_OK;
    std::vector<hf_graph*> one{g};
    return plan_build(one, &g->plan);
}

hf_status hf_run(hf_graph* g, void* stream, const hf_run_opts* opts) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (g->dirty && g->plan) {
        if (plan_busy(g->plan) != HF_OK) return fail(HF_ESTATE, "a run of this graph is in flight");
        plan_destroy(g->plan);
        g->plan = nullptr;
    }
    hf_status st = ensure_plan(g);
    if (st != HF_OK) return st;
    hf_run_opts o;
    if (opts) o = *opts;
    else hf_run_opts_default(&o);
    return plan_run(g->plan, (cudaStream_t)stream, o);
}

hf_status hf_run_host(hf_graph* g, void* stream, const hf_run_opts* opts, const float* delay, float* arr_out) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (g->dirty && g->plan) {
        if (plan_busy(g->plan) != HF_OK) return fail(HF_ESTATE, "a run of this graph is in flight");
        plan_destroy(g->plan);
        g->plan = nullptr;
    }
    hf_status st = ensure_plan(g);
    if (st != HF_OK) return st;
    hf_run_opts o;
    if (opts) o = *opts;
    else hf_run_opts_default(&o);
    return plan_run_host(g->plan, (cudaStream_t)stream, o, delay, arr_out);
}

hf_status hf_run_n(hf_graph* g, void* stream, const hf_run_opts* opts, int32_t n) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (n < 0) return fail(HF_EINVAL, "n < 0");
    for (int32_t i = 0; i < n; ++i) {
        hf_status st = i == 0 ? hf_run(g, stream, opts) : HF_OK;
        if (i > 0) {
            hf_run_opts o;
            if (opts) o = *opts;
            else hf_run_opts_default(&o);
            st = plan_run(g->plan, (cudaStream_t)stream, o, true);
        }
        if (st != HF_OK) return st;
    }
    return HF_OK;
}

hf_status hf_run_until(hf_graph* g, void* stream, const hf_run_opts* opts, int32_t (*pred)(void* ctx), void* ctx,
                       int32_t max_runs, int32_t* runs_out) {
    if (!g || !pred) return fail(HF_EINVAL, "NULL argument");
    if (max_runs < 0) return fail(HF_EINVAL, "max_runs < 0");
    int32_t runs = 0;
    hf_status st = HF_OK;
    while (runs < max_runs) {
        if ((st = hf_run(g, stream, opts)) != HF_OK) break;
        if ((st = hf_sync_status(g)) != HF_OK) break;
        ++runs;
        if (pred(ctx)) break;
    }
    if (runs_out) *runs_out = runs;
    return st;
}

hf_status hf_sync_status(hf_graph* g) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (!g->plan) return fail(HF_ESTATE, "graph has not run");
    return plan_sync(g->plan);
}

hf_status hf_get_arrivals(hf_graph* g, float* out, int on_device) {
    if (!g || (!out && g->kind.size())) return fail(HF_EINVAL, "NULL argument");
    if (!g->plan) return fail(HF_ESTATE, "graph has not run");
    return plan_get_arrivals(g->plan, 0, out, on_device);
}

hf_status hf_get_stamps(hf_graph* g, int64_t* start, int64_t* finish, int32_t* exec_count) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (!g->plan) return fail(HF_ESTATE, "graph has not run");
    return plan_get_stamps(g->plan, 0, start, finish, exec_count);
}

hf_status hf_get_task_times(hf_graph* g, int64_t* a, int64_t* b) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (!g->plan) return fail(HF_ESTATE, "graph has not run");
    return plan_get_times(g->plan, 0, a, b);
}

hf_status hf_kernel_ms(hf_graph* g, float* ms) {
    if (!g || !ms) return fail(HF_EINVAL, "NULL argument");
    if (!g->plan) return fail(HF_ESTATE, "graph has not run");
    return plan_kernel_ms(g->plan, ms);
}

hf_status hf_set_delays(hf_graph* g, const float* delay, int on_device, void* stream) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (g->dirty && g->plan) {
        if (plan_busy(g->plan) != HF_OK) return fail(HF_ESTATE, "a run of this graph is in flight");
        plan_destroy(g->plan);
        g->plan = nullptr;
    }
    hf_status st = ensure_plan(g);
    if (st != HF_OK) return st;
    return plan_set_delays(g->plan, delay, on_device, (cudaStream_t)stream);
}

hf_status hf_batch_create(hf_batch** out) {
    if (!out) return fail(HF_EINVAL, "out is NULL");
    try {
        *out = new hf_batch();
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    return HF_OK;
}

hf_status hf_batch_destroy(hf_batch* b) {
    if (!b) return HF_OK;
    if (b->plan) plan_destroy(b->plan);
    for (hf_graph* g : b->graphs) g->in_batches--;
    delete b;
    return HF_OK;
}

hf_status hf_batch_add(hf_batch* b, hf_graph* g, int32_t* index_out) {
    if (!b || !g) return fail(HF_EINVAL, "NULL argument");
    if (b->plan && plan_busy(b->plan) != HF_OK) return fail(HF_ESTATE, "a run of this batch is in flight");
    if (g->dirty) {
        hf_status st = hf_finalize(g);
        if (st != HF_OK) return st;
    }
    try {
        b->graphs.push_back(g);
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    g->in_batches++;
    if (b->plan) {
        plan_destroy(b->plan);
        b->plan = nullptr;
    }
    if (index_out) *index_out = (int32_t)b->graphs.size() - 1;
    return HF_OK;
}

static hf_status ensure_batch_plan(hf_batch* b) {
    if (b->plan) return HF_OK;
    hf_status st = plan_build(b->graphs, &b->plan);
    if (st != HF_OK) return st;
    plan_set_costmodel(b->plan, b->cm);
    return HF_OK;
}

hf_status hf_batch_set_costmodel(hf_batch* b, hf_costmodel* cm) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (b->plan && plan_busy(b->plan) != HF_OK) return fail(HF_ESTATE, "a run of this batch is in flight");
    b->cm = cm;
    if (b->plan) plan_set_costmodel(b->plan, cm);
    return HF_OK;
}

hf_status hf_batch_refresh_priorities(hf_batch* b, void* stream) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    if (plan_busy(b->plan) != HF_OK) return fail(HF_ESTATE, "a run of this batch is in flight");
    return plan_refresh_priorities(b->plan, b->cm, (cudaStream_t)stream);
}

hf_status hf_batch_features(hf_batch* b, float* X, void* stream) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    return plan_features(b->plan, X, (cudaStream_t)stream);
}

hf_status hf_features(hf_graph* g, float* X, void* stream) {
    if (!g) return fail(HF_EINVAL, "graph is NULL");
    if (g->dirty && g->plan) {
        if (plan_busy(g->plan) != HF_OK) return fail(HF_ESTATE, "a run of this graph is in flight");
        plan_destroy(g->plan);
        g->plan = nullptr;
    }
    hf_status st = ensure_plan(g);
    if (st != HF_OK) return st;
    return plan_features(g->plan, X, (cudaStream_t)stream);
}

hf_status hf_batch_task_costs(hf_batch* b, int32_t priority, float* cost, float* bottom, void* stream) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    return plan_task_costs(b->plan, priority, b->cm, cost, bottom, (cudaStream_t)stream);
}

hf_status hf_batch_autotune(hf_batch* b, void* stream, const hf_run_opts* base, int force, hf_run_opts* best,
                            float* best_ms) {
    if (!b || !best || !best_ms) return fail(HF_EINVAL, "NULL argument");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    hf_run_opts o;
    if (base) o = *base;
    else hf_run_opts_default(&o);
    return plan_autotune(b->plan, (cudaStream_t)stream, o, force, best, best_ms);
}

hf_status hf_batch_predict(hf_batch* b, int32_t priority, void* stream, float* levelsync_ms, float* persistent_ms,
                           float* team_ms) {
    if (!b || !levelsync_ms || !persistent_ms || !team_ms) return fail(HF_EINVAL, "NULL argument");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    return plan_predict(b->plan, priority, b->cm, (cudaStream_t)stream, levelsync_ms, persistent_ms, team_ms);
}

hf_status hf_calibration(void* stream, float* out) {
    if (!out) return fail(HF_EINVAL, "NULL argument");
    return plan_calibration((cudaStream_t)stream, out);
}

hf_status hf_batch_bottom_levels(hf_batch* b, const float* cost, float* bottom, void* stream) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    return plan_bottom_levels(b->plan, cost, bottom, (cudaStream_t)stream);
}

hf_status hf_batch_run(hf_batch* b, void* stream, const hf_run_opts* opts) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    {
        hf_status st = ensure_batch_plan(b);
        if (st != HF_OK) return st;
    }
    hf_run_opts o;
    if (opts) o = *opts;
    else hf_run_opts_default(&o);
    return plan_run(b->plan, (cudaStream_t)stream, o);
}

hf_status hf_batch_run_host(hf_batch* b, void* stream, const hf_run_opts* opts, const float* delay, float* arr_out) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    hf_run_opts o;
    if (opts) o = *opts;
    else hf_run_opts_default(&o);
    return plan_run_host(b->plan, (cudaStream_t)stream, o, delay, arr_out);
}

hf_status hf_batch_run_n(hf_batch* b, void* stream, const hf_run_opts* opts, int32_t n) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (n < 0) return fail(HF_EINVAL, "n < 0");
    for (int32_t i = 0; i < n; ++i) {
        hf_status st = HF_OK;
        if (i == 0) {
            st = hf_batch_run(b, stream, opts);
        } else {
            hf_run_opts o;
            if (opts) o = *opts;
            else hf_run_opts_default(&o);
            st = plan_run(b->plan, (cudaStream_t)stream, o, true);
        }
        if (st != HF_OK) return st;
    }
    return HF_OK;
}

hf_status hf_batch_run_until(hf_batch* b, void* stream, const hf_run_opts* opts, int32_t (*pred)(void* ctx),
                             void* ctx, int32_t max_runs, int32_t* runs_out) {
    if (!b || !pred) return fail(HF_EINVAL, "NULL argument");
    if (max_runs < 0) return fail(HF_EINVAL, "max_runs < 0");
    int32_t runs = 0;
    hf_status st = HF_OK;
    while (runs < max_runs) {
        if ((st = hf_batch_run(b, stream, opts)) != HF_OK) break;
        if ((st = hf_batch_sync_status(b)) != HF_OK) break;
        ++runs;
        if (pred(ctx)) break;
    }
    if (runs_out) *runs_out = runs;
    return st;
}

hf_status hf_batch_partition(const hf_batch* b, int32_t ndev, int32_t* dev_of_graph, double* load_out) {
    if (!b || !dev_of_graph) return fail(HF_EINVAL, "NULL argument");
    if (ndev < 1) return fail(HF_EINVAL, "ndev < 1");
    try {
        std::vector<double> cost(b->graphs.size(), 0.0);
        for (size_t i = 0; i < b->graphs.size(); ++i) {
            const hf_graph* g = b->graphs[i];
            std::vector<int32_t> fanout(g->kind.size(), 0);
            for (int32_t u : g->esrc) fanout[(size_t)u] += 1;
            for (int32_t v = 0; v < (int32_t)g->kind.size(); ++v) cost[i] += host_heuristic_cost(g, v, fanout[(size_t)v]);
        }
        std::vector<int32_t> dev;
        std::vector<double> load;
        lpt_pack(cost, ndev, &dev, &load);
        for (size_t i = 0; i < dev.size(); ++i) dev_of_graph[i] = dev[i];
        if (load_out)
            for (int32_t d = 0; d < ndev; ++d) load_out[d] = load[(size_t)d];
    } catch (const std::bad_alloc&) {
        return fail(HF_ENOMEM, "host allocation failed");
    }
    return HF_OK;
}

hf_status hf_batch_sync_status(hf_batch* b) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_sync(b->plan);
}

hf_status hf_batch_get_arrivals(hf_batch* b, int32_t index, float* out, int on_device) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    if (index < -1 || index >= (int32_t)b->graphs.size()) return fail(HF_EINVAL, "graph index out of range");
    return plan_get_arrivals(b->plan, index, out, on_device);
}

hf_status hf_batch_get_task_times(hf_batch* b, int32_t index, int64_t* t0, int64_t* t1) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    if (index < 0 || index >= (int32_t)b->graphs.size()) return fail(HF_EINVAL, "graph index out of range");
    return plan_get_times(b->plan, index, t0, t1);
}

hf_status hf_batch_get_stats(hf_batch* b, int64_t* out, int32_t n) {
    if (!b || !out || n < 0) return fail(HF_EINVAL, "bad argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_get_stats(b->plan, out, n);
}

hf_status hf_batch_get_graph_times(hf_batch* b, int64_t* start, int64_t* end) {
    if (!b || !start || !end) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_get_graph_times(b->plan, start, end);
}

hf_status hf_batch_get_task_costs(hf_batch* b, int32_t index, float* cost_ns) {
    if (!b || !cost_ns) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    if (index < -1 || index >= (int32_t)b->graphs.size()) return fail(HF_EINVAL, "graph index out of range");
    return plan_get_task_costs(b->plan, index, cost_ns);
}

hf_status hf_batch_last_launches(hf_batch* b, int32_t* n) {
    if (!b || !n) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_last_launches(b->plan, n);
}

hf_status hf_batch_team_plan(hf_batch* b, int32_t* team_size) {
    if (!b || !team_size) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_team_plan(b->plan, team_size);
}

hf_status hf_batch_team_keys(hf_batch* b, int32_t* shared) {
    if (!b || !shared) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_team_keys(b->plan, shared);
}

hf_status hf_batch_team_flags(hf_batch* b, int32_t* flags) {
    if (!b || !flags) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_team_flags(b->plan, flags);
}

hf_status hf_batch_kernel_ms(hf_batch* b, float* ms) {
    if (!b || !ms) return fail(HF_EINVAL, "NULL argument");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    return plan_kernel_ms(b->plan, ms);
}

hf_status hf_batch_set_delays(hf_batch* b, const float* delay, int on_device, void* stream) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    hf_status st = ensure_batch_plan(b);
    if (st != HF_OK) return st;
    return plan_set_delays(b->plan, delay, on_device, (cudaStream_t)stream);
}

hf_status hf_batch_get_stamps(hf_batch* b, int32_t index, int64_t* s0, int64_t* s1, int32_t* c) {
    if (!b) return fail(HF_EINVAL, "batch is NULL");
    if (!b->plan) return fail(HF_ESTATE, "batch has not run");
    if (index < 0 || index >= (int32_t)b->graphs.size()) return fail(HF_EINVAL, "graph index out of range");
    return plan_get_stamps(b->plan, index, s0, s1, c);
}

}  // extern "C"
