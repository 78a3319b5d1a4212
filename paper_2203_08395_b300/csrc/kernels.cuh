// kernels.cuh -- device code of the task-graph executor (sm_103a).
//
// Two executors share the payload code:
//   * level-synchronous: one kernel per topological level (captured in a CUDA graph); each
//     thread pulls the arrival of one task from its level-sorted in-edges;
//   * persistent: one launch; every warp loops popping ready tasks (shared-memory stack
//     first, then pre-claimed global queue slots), runs their payload pieces, and releases
//     successors through atomic in-degree counters, pushing the ones that become ready. In
//     the work-stealing variant each CTA also owns a ring of ready tasks that its warps fill
//     and take from first, and idle warps steal from other CTAs' rings.
// Arrivals are kept as order-preserving uint32 keys so that the max over predecessors is
// an unsigned integer max (an atomicMax in the persistent executor).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hf_internal.h"

namespace hf {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 8;
constexpr int kStackCap = 16;  // per-warp shared-memory ready stack (double-buffered)
constexpr int kStage = 8;      // edge records staged in shared memory per stacked task

__device__ __forceinline__ uint32_t f2key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(int32_t* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_max(uint32_t* p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_dec_acq_rel(int32_t* p) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], -1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// asynchronous 16-byte global -> shared copy (completion: cp_async_wait_all by the issuer)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------ payload pieces (warp-wide)

// y[i] = fma(a, x[i], y[i]) for i in [0, cnt): one warp, 16-byte vector accesses when x and y
// share their alignment, streaming cache hints (each element is touched once). The unaligned
// head and the ragged tail are loaded together with the first 512-element block, so a piece of
// up to 512 elements costs one round trip; lanes past the end of a block load its last vector
// again and store nothing.
__device__ __forceinline__ void warp_saxpy_f32(float* __restrict__ y, const float* __restrict__ x, int64_t cnt,
                                               float a, int lane) {
    if ((((uintptr_t)y ^ (uintptr_t)x) & 15) == 0) {
        int64_t head = (int64_t)(((16 - ((uintptr_t)y & 15)) & 15) >> 2);
        if (head > cnt) head = cnt;
        float hx = 0.f, hy = 0.f, tx = 0.f, ty = 0.f;
        if (lane < head) {
            hx = __ldcg(x + lane);
            hy = __ldcg(y + lane);
        }
        float* yb = y + head;
        const float* xb = x + head;
        const int64_t body = cnt - head;
        const int64_t nv = body >> 2;
        const int64_t done = nv << 2;
        if (lane < body - done) {
            tx = __ldcg(xb + done + lane);
            ty = __ldcg(yb + done + lane);
        }
        float4* __restrict__ y4 = reinterpret_cast<float4*>(yb);
        const float4* __restrict__ x4 = reinterpret_cast<const float4*>(xb);
        for (int64_t k = lane; k - lane < nv; k += 128) {
            float4 xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = k + 32 * u < nv ? k + 32 * u : nv - 1;
                xv[u] = __ldcs(x4 + i);
                yv[u] = __ldcs(y4 + i);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                yv[u].x = __fmaf_rn(a, xv[u].x, yv[u].x);
                yv[u].y = __fmaf_rn(a, xv[u].y, yv[u].y);
                yv[u].z = __fmaf_rn(a, xv[u].z, yv[u].z);
                yv[u].w = __fmaf_rn(a, xv[u].w, yv[u].w);
                if (k + 32 * u < nv) __stcs(y4 + k + 32 * u, yv[u]);
            }
        }
        if (lane < head) y[lane] = __fmaf_rn(a, hx, hy);
        if (lane < body - done) yb[done + lane] = __fmaf_rn(a, tx, ty);
    } else {
        for (int64_t i = lane; i < cnt; i += 32) y[i] = __fmaf_rn(a, __ldcg(x + i), __ldcg(y + i));
    }
}

// int32 saxpy with two's-complement wrap-around (unsigned arithmetic), same access pattern
__device__ __forceinline__ void warp_saxpy_i32(int32_t* __restrict__ y, const int32_t* __restrict__ x, int64_t cnt,
                                               uint32_t a, int lane) {
    if ((((uintptr_t)y ^ (uintptr_t)x) & 15) == 0) {
        int64_t head = (int64_t)(((16 - ((uintptr_t)y & 15)) & 15) >> 2);
        if (head > cnt) head = cnt;
        uint32_t hx = 0, hy = 0, tx = 0, ty = 0;
        if (lane < head) {
            hx = (uint32_t)__ldcg(x + lane);
            hy = (uint32_t)__ldcg(y + lane);
        }
        int32_t* yb = y + head;
        const int32_t* xb = x + head;
        const int64_t body = cnt - head;
        const int64_t nv = body >> 2;
        const int64_t done = nv << 2;
        if (lane < body - done) {
            tx = (uint32_t)__ldcg(xb + done + lane);
            ty = (uint32_t)__ldcg(yb + done + lane);
        }
        int4* __restrict__ y4 = reinterpret_cast<int4*>(yb);
        const int4* __restrict__ x4 = reinterpret_cast<const int4*>(xb);
        for (int64_t k = lane; k - lane < nv; k += 128) {
            int4 xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = k + 32 * u < nv ? k + 32 * u : nv - 1;
                xv[u] = __ldcs(x4 + i);
                yv[u] = __ldcs(y4 + i);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                yv[u].x = (int32_t)(a * (uint32_t)xv[u].x + (uint32_t)yv[u].x);
                yv[u].y = (int32_t)(a * (uint32_t)xv[u].y + (uint32_t)yv[u].y);
                yv[u].z = (int32_t)(a * (uint32_t)xv[u].z + (uint32_t)yv[u].z);
                yv[u].w = (int32_t)(a * (uint32_t)xv[u].w + (uint32_t)yv[u].w);
                if (k + 32 * u < nv) __stcs(y4 + k + 32 * u, yv[u]);
            }
        }
        if (lane < head) y[lane] = (int32_t)(a * hx + hy);
        if (lane < body - done) yb[done + lane] = (int32_t)(a * tx + ty);
    } else {
        for (int64_t i = lane; i < cnt; i += 32) y[i] = (int32_t)(a * (uint32_t)__ldcg(x + i) + (uint32_t)__ldcg(y + i));
    }
}

// byte copy (either end may be page-locked host memory reached over the host link), same
// access pattern with 16-byte vectors
__device__ __forceinline__ void warp_copy(char* __restrict__ d, const char* __restrict__ s, int64_t cnt, int lane) {
    if ((((uintptr_t)d ^ (uintptr_t)s) & 15) == 0) {
        int64_t head = (int64_t)((16 - ((uintptr_t)d & 15)) & 15);
        if (head > cnt) head = cnt;
        char hc = 0, tc = 0;
        if (lane < head) hc = __ldcg(s + lane);
        char* db = d + head;
        const char* sb = s + head;
        const int64_t body = cnt - head;
        const int64_t nv = body >> 4;
        const int64_t done = nv << 4;
        if (lane < body - done) tc = __ldcg(sb + done + lane);
        uint4* __restrict__ d4 = reinterpret_cast<uint4*>(db);
        const uint4* __restrict__ s4 = reinterpret_cast<const uint4*>(sb);
        for (int64_t k = lane; k - lane < nv; k += 128) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcg(s4 + (k + 32 * u < nv ? k + 32 * u : nv - 1));
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k + 32 * u < nv) __stcg(d4 + k + 32 * u, v[u]);
        }
        if (lane < head) d[lane] = hc;
        if (lane < body - done) db[done + lane] = tc;
    } else {
        for (int64_t i = lane; i < cnt; i += 32) d[i] = __ldcg(s + i);
    }
}

__device__ __forceinline__ void run_piece(const DevPayload& P, int piece, int lane) {
    const int64_t b0 = (int64_t)piece * P.chunk;
    int64_t b1 = b0 + P.chunk;
    if (b1 > P.n) b1 = P.n;
    if (b1 <= b0) return;
    if (P.op == kPaySaxpyF32) {
        warp_saxpy_f32((float*)P.dst + b0, (const float*)P.src + b0, b1 - b0, __uint_as_float(P.a_bits), lane);
    } else if (P.op == kPaySaxpyI32) {
        warp_saxpy_i32((int32_t*)P.dst + b0, (const int32_t*)P.src + b0, b1 - b0, P.a_bits, lane);
    } else if (P.op == kPayCopy) {
        warp_copy((char*)P.dst + b0, (const char*)P.src + b0, b1 - b0, lane);
    }
}

__device__ __forceinline__ void st_release_sys(int32_t* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_sys(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Host task k through the mapped mailbox (one thread): the system-scope fence makes what this
// thread observed of upstream device work (push copies into host memory included) visible to
// the callback; the post is a release, the done flag an acquire that orders the callback's
// writes before the successors this warp releases. Bounded: after limit_ns the status becomes
// HF_ETIMEDOUT and `abort` (if given) is raised. Returns false on timeout.
__device__ __noinline__ bool host_task_roundtrip(int32_t* post, int32_t* post_ctr, const int32_t* hdone, int k,
                                                 uint64_t limit_ns, int32_t* status, int32_t* abort) {
    __threadfence_system();
    st_release_sys(post + atomicAdd(post_ctr, 1), k);
    const uint64_t t0 = gtimer();
    while (ld_acquire_sys(hdone + k) == 0) {
        if (gtimer() - t0 > limit_ns) {
            atomicCAS(status, 0, (int)HF_ETIMEDOUT);
            if (abort) atomicExch(abort, 1);
            return false;
        }
        __nanosleep(200);
    }
    return true;
}

// ------------------------------------------------------------------ level-synchronous kernel

// Arrivals of one topological level (pull form over level-sorted in-edges; no atomics) plus
// the payload pieces of that level's tasks. Blocks [0, nb_mp) do arrivals, one thread per
// task; the remaining blocks do payload pieces, one warp per piece.
template <bool PAY>
__global__ void __launch_bounds__(256) k_level(const LevelArgs a) {
    // programmatic dependent launch: the next level's kernel may be scheduled now; this one
    // reads the previous level's results only after griddepcontrol.wait, so it can load its
    // own task list and in-edges while the previous level finishes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if ((int)blockIdx.x < a.nb_mp) {
        const int p = a.p0 + (int)blockIdx.x * 256 + (int)threadIdx.x;
        if (p >= a.p1) return;
        const int v = __ldg(a.ls_node + p);
        const int e0 = __ldg(a.ls_ptr + p), e1 = __ldg(a.ls_ptr + p + 1);
        uint32_t best;
        if (e0 == e1) {
            best = a.key0 ? __ldg(a.key0 + v) : kKeyPosZero;
        } else {
            // batches of up to 8 in-edges: every key load of a batch is issued before the first
            // is used, so a task's gather costs one round trip
            best = 0u;
            for (int e = e0; e < e1; e += 8) {
                const int cnt = e1 - e < 8 ? e1 - e : 8;
                int2 ie[8];
                uint32_t kk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < cnt) ie[j] = __ldg(a.ls_in + e + j);
                if (e == e0) asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < cnt) kk[j] = __ldcg(a.key + ie[j].x);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < cnt) best = max(best, f2key(__fadd_rn(key2f(kk[j]), __int_as_float(ie[j].y))));
            }
        }
        a.key[v] = best;
        return;
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (PAY) {
        const int lane = threadIdx.x & 31;
        const int wg = ((int)blockIdx.x - a.nb_mp) * 8 + ((int)threadIdx.x >> 5);
        const int nw = ((int)gridDim.x - a.nb_mp) * 8;
        for (int it = a.i0 + wg; it < a.i1; it += nw) {
            const int2 w = __ldg(a.items + it);
            run_piece(a.pay[w.x], w.y, lane);
        }
    }
}

// ------------------------------------------------------------------ persistent executor
//
// Per-task state is one 64-bit word: arrival key (high 32 bits) and pending-predecessor count
// (low 32 bits). A finished predecessor u releases successor v with one compare-and-swap that
// raises the key to max(key, key(arr[u] + d(u,v))) and decrements the count together, so the
// predecessor that brings the count to zero learns v's final arrival from the CAS itself and
// no memory fence is needed for max-plus tasks (only payload tasks, whose data other tasks
// read, fence before releasing and after becoming ready). The successor edge record carries
// v's in-degree, so the first CAS is issued without reading v's state. Tasks with more than
// kNarrowIn predecessors use a 32-bit max on the key half, a fence and an atomic decrement on
// the count half instead, which avoids CAS retry storms on wide joins.

// Edge record word w: bits 0-6 successor's in-degree (kWideMark: wide join), bits 7-14 zero,
// bit 15 set when it has a payload, bits 16-31 its out-degree (kLongMark: look it up in meta).
constexpr uint32_t kWideMark = 0x7Fu;
constexpr uint32_t kLongMark = 0xFFFFu;
constexpr uint32_t kPayBit = 1u << 15;

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 residency. The per-task state words (8 bytes per task, one compare-and-swap per edge at a
// random task) must stay in L2 across the run, while the edge records stream past them once:
// the reset kernel stores the state words with an evict-last policy, the executor reads them
// with it, and reads edge records with an evict-first policy (and without L1 allocation).
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ int4 ld_stream_int4(const int4* p, uint64_t pol) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ void st_keep_u64(unsigned long long* p, unsigned long long v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_keep_u64(const unsigned long long* p, uint64_t pol) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int atom_dec_relaxed(int32_t* p) {
    int old;
    asm volatile("atom.relaxed.gpu.global.add.s32 %0, [%1], -1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__global__ void k_reset(const ResetArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t keep = l2_policy_last();
    for (int64_t i = tid; i < a.n_tasks; i += stride) {
        const int d = a.indeg0[i];
        const uint32_t k = d ? kKeyNegInf : (a.key0 ? a.key0[i] : kKeyPosZero);
        const uint32_t c = (uint32_t)d + (i == a.stall_task ? 1u : 0u);
        st_keep_u64(a.state + i, ((unsigned long long)k << 32) | c, keep);
        if (a.t_start) {
            a.t_start[i] = INT64_MAX;
            a.t_end[i] = 0;
        }
        if (a.exec_count) {
            a.exec_count[i] = 0;
            a.tk_start[i] = -1;
            a.tk_end[i] = -1;
        }
    }
    // sources without payload seed the main queue; sources with one (pseeds: non-copy payloads,
    // then pull copies, then push copies) seed the payload queue in warp-specialised runs, else
    // they follow in the main queue; with copy warps the copies seed their own queues instead
    const int64_t nc = (int64_t)a.n_cseed0 + a.n_cseed1;
    const int64_t npay_seed = a.link ? a.n_pseed : (int64_t)a.n_pseed + nc;
    const int64_t nmain = a.split ? a.n_seed : (int64_t)a.n_seed + npay_seed;
    for (int64_t i = tid; i < a.qcap; i += stride) {
        int v = -1;
        if (i < a.n_seed) v = a.seeds[i];
        else if (i < nmain) v = a.pseeds[i - a.n_seed];
        if (v >= 0 && v == a.stall_task) v = -2;  // never a task id: its slot is skipped
        a.queue[i] = v;
    }
    if (a.split)
        for (int64_t i = tid; i < a.pqcap; i += stride) {
            int v = i < npay_seed ? a.pseeds[i] : -1;
            if (v >= 0 && v == a.stall_task) v = -2;
            a.pqueue[i] = v;
        }
    if (a.link)
        for (int64_t i = tid; i < a.lqcap; i += stride) {
            int v0 = i < a.n_cseed0 ? a.pseeds[a.n_pseed + i] : -1;
            int v1 = i < a.n_cseed1 ? a.pseeds[a.n_pseed + a.n_cseed0 + i] : -1;
            if (v0 >= 0 && v0 == a.stall_task) v0 = -2;
            if (v1 >= 0 && v1 == a.stall_task) v1 = -2;
            a.lqueue0[i] = v0;
            a.lqueue1[i] = v1;
        }
    for (int64_t i = tid; i < a.n_pay; i += stride) a.chunks_left[i] = a.pay[i].nchunks;
    if (a.ring) {  // work stealing: empty rings, positions from 0
        for (int64_t i = tid; i < a.ring_cells; i += stride) a.ring[i] = 0ull;
        for (int64_t i = tid; i < a.ring_heads; i += stride) a.ring_head[i] = 0;
    }
    if (tid == 0) {
        a.ctrl->head = 0;
        a.ctrl->tail = (int32_t)nmain;
        a.ctrl->phead = 0;
        a.ctrl->ptail = a.split ? (int32_t)npay_seed : 0;
        a.ctrl->lhead0 = 0;
        a.ctrl->ltail0 = a.link ? a.n_cseed0 : 0;
        a.ctrl->lhead1 = 0;
        a.ctrl->ltail1 = a.link ? a.n_cseed1 : 0;
        a.ctrl->done = 0;
        if (!a.keep_status) a.ctrl->status = 0;
        a.ctrl->abort = 0;
        a.ctrl->ticket = 0;
    }
}

// Per-warp executor counters (reported when PersistArgs::stats is set); `cas` is per lane.
struct WStats {
    uint32_t rounds = 0, items = 0, idle = 0, edges = 0, cas = 0, local = 0, global = 0, claims = 0, pops = 0,
             pieces = 0, ring = 0, steals = 0;
    unsigned long long cyc_round = 0, cyc_release = 0, cyc_cas = 0, cyc_push = 0;
    bool on = false;  // cycle counts are taken only when counters are recorded
};

__device__ __forceinline__ long long clk(const WStats& ws) { return ws.on ? clock64() : 0; }

// Queue items: [0, n) a task without payload; [n, n + npieces) one piece of a multi-piece
// payload; [n + npieces, n + npieces + npay) the start of payload p (the warp that pops it
// pushes the payload's other pieces, if any, and runs the first).

// Appends each lane's `cnt` items (first_item, first_item+1, ... when multi, else first_item)
// to a global queue with one atomicAdd on its tail per warp, then publishes them.
__device__ __forceinline__ void push_items(const PersistArgs& a, int32_t* slots, int32_t cap, int32_t* tailp, int cnt,
                                           int first_item, bool multi, int lane, WStats& ws) {
    if (__ballot_sync(kFull, cnt > 0) == 0) return;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    int base = 0;
    ws.global += (uint32_t)total;
    if (lane == 0) base = atomicAdd(tailp, total);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base + total > (int64_t)cap) {  // cannot happen with a correct capacity
        if (lane == 0) {
            atomicExch(&a.ctrl->status, (int)HF_EQUEUE);
            atomicExch(&a.ctrl->abort, 1);
        }
        __syncwarp();
        return;
    }
    fence_acq_rel();  // release: the ready task's state (and inputs) before its queue slot
    const int start = base + incl - cnt;
    for (int k = 0; k < cnt; ++k) st_relaxed(slots + start + k, first_item + (multi ? k : 0));
    __syncwarp();
}

// ---- work stealing (Section III-C): per-CTA rings beside the global queue
// The warps of a CTA push the ready tasks that do not stay in their stacks (and the pieces of
// payloads they expand) to the CTA's own ring. A warp takes from its own ring first, then from
// the global queue (sources and ring overflow), and when both are empty steals from the ring of
// a randomly chosen other CTA. A ring is a bounded FIFO with one producer side and many
// consumers: its fill position lives in the owner's shared memory (only the owner's warps
// push), its take position in global memory (owner and thieves take with a compare-and-swap),
// and every cell carries the position it was written for, so a taker sees exactly which cells
// at the front are published and a cell left from an earlier lap never passes for a new one.

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// As push_items, to this CTA's ring: the leading items that fit go to the ring (a slot is free
// once the take position has passed the cell's previous lap), the rest to the global queue.
// rt[0]: the ring's fill position; rt[1]: a lower bound of its take position (shared memory).
__device__ __forceinline__ void ring_push(const PersistArgs& a, int* rt, int cnt, int first_item, bool multi,
                                          int lane, WStats& ws) {
    if (__ballot_sync(kFull, cnt > 0) == 0) return;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - cnt;
    const int cap = a.ring_mask + 1;
    int base = 0, fit = 0;
    if (lane == 0) {
        const int32_t* hp = a.ring_head + (size_t)blockIdx.x * 32;
        for (int tries = 0; tries < 64; ++tries) {  // contended only by this CTA's warps
            const int t = *(volatile int*)&rt[0];
            int h = *(volatile int*)&rt[1];
            if (t + total - h > cap) {  // the cached take position may be behind: reload it
                h = max(h, ld_relaxed(hp));
                atomicMax(&rt[1], h);
            }
            fit = min(total, max(h + cap - t, 0));
            if (fit == 0) break;
            if (atomicCAS(&rt[0], t, t + fit) == t) {
                base = t;
                break;
            }
            fit = 0;
        }
    }
    base = __shfl_sync(kFull, base, 0);
    fit = __shfl_sync(kFull, fit, 0);
    const int mine = min(cnt, max(fit - excl, 0));  // this lane's items that go to the ring
    if (fit > 0) {
        ws.ring += (uint32_t)fit;
        fence_acq_rel();  // release: the ready tasks' state (and inputs) before their cells
        unsigned long long* cells = a.ring + (size_t)blockIdx.x * cap;
        for (int k = 0; k < mine; ++k) {
            const int pos = base + excl + k;
            st_relaxed_u64(cells + (pos & a.ring_mask),
                           ((unsigned long long)(uint32_t)(pos + 1) << 32) | (uint32_t)(first_item + (multi ? k : 0)));
        }
    }
    push_items(a, a.queue, a.qcap, &a.ctrl->tail, cnt - mine, first_item + (multi ? mine : 0), multi, lane, ws);
}

// Takes up to `most` (<= 32) published items from the front of CTA c's ring into lanes
// 0..k-1 (`item`) and returns k: the published run at the front (half of it when stealing),
// 0 when the front is not published or another warp took it first. h: the take position the
// front is read at (the CAS fails if it moved); rt: the owner's shared positions, whose take
// hint follows the head (NULL when stealing).
__device__ __forceinline__ int ring_take_at(const PersistArgs& a, int c, int h, int most, bool half, int* rt,
                                            int lane, int& item) {
    int32_t* hp = a.ring_head + (size_t)c * 32;
    unsigned long long cell = 0;
    if (lane < most) cell = ld_relaxed_u64(a.ring + (size_t)c * (a.ring_mask + 1) + ((h + lane) & a.ring_mask));
    const unsigned pub = __ballot_sync(kFull, lane < most && (uint32_t)(cell >> 32) == (uint32_t)(h + lane + 1));
    int k = pub == kFull ? 32 : __ffs(~pub) - 1;
    if (half) k = (k + 1) >> 1;
    if (k == 0) return 0;
    int prev = 0;
    if (lane == 0) {
        prev = atomicCAS(hp, h, h + k);
        if (rt) atomicMax(&rt[1], prev == h ? h + k : prev);  // the owner's hint follows the head
    }
    if (__shfl_sync(kFull, prev, 0) != h) return 0;
    if (lane < k) item = (int)(uint32_t)cell;
    fence_acq_rel();  // acquire: what the pusher released with the cells
    return k;
}

// This CTA's own ring: empty when the shared fill position has not passed the shared hint of
// the take position (thieves only move the head further), so an idle check costs no global
// access; otherwise the front is read at the hint.
__device__ __forceinline__ int ring_take_own(const PersistArgs& a, int* rt, int most, int lane, int& item) {
    const int t = *(volatile int*)&rt[0];
    const int h = *(volatile int*)&rt[1];
    if (t <= h) return 0;
    return ring_take_at(a, (int)blockIdx.x, h, min(most, t - h), false, rt, lane, item);
}

// Another CTA's ring: its head first, then half of its published front.
__device__ __forceinline__ int ring_steal(const PersistArgs& a, int c, int most, int lane, int& item) {
    int h = 0;
    if (lane == 0) h = ld_relaxed(a.ring_head + (size_t)c * 32);
    h = __shfl_sync(kFull, h, 0);
    return ring_take_at(a, c, h, most, true, nullptr, lane, item);
}

// Pushes this warp's ready tasks (lane: r.x >= 0 with r = {task, key, first out-edge (payload
// index for payload tasks), out-degree | payload flag << 31}). Tasks go to the warp's stack
// while it has room (up to local_keep; the first lanes' tasks) -- plain tasks with their first
// kStage out-edges staged in shared memory for the next round -- except payload tasks in
// warp-specialised runs, which go to the payload queue, and copies in runs with copy warps,
// which go to their direction's queue; the rest go to the main queue (with work stealing: to
// the CTA's ring, rt). nstk / nedg: the stack buffer filled this round and its staging area.
template <bool PAY>
__device__ __forceinline__ void push_ready(const PersistArgs& a, int4 r, int4* nstk, int4* nedg, int& top,
                                           int* rt, int lane, WStats& ws) {
    const long long c_push = clk(ws);
    const int v = r.x;
    const bool haspay = PAY && v >= 0 && r.w < 0;
    // copies go to the copy queue of their direction when the run has copy warps (1: pull, 2: push)
    const int cls = (haspay && a.pdir) ? (int)__ldg(a.pdir + r.z) : 0;
    const bool topay = haspay && cls == 0 && a.pay_warps > 0;
    const bool single = v >= 0 && !topay && cls == 0;
    const unsigned sm = __ballot_sync(kFull, single);
    const int room = a.local_keep - top;
    const int rank = __popc(sm & lanemask_lt());
    bool go_global = v >= 0;
    if (single && rank < room) {
        const int slot = top + rank;
        nstk[slot] = r;
        const int len = min(r.w & 0x7fffffff, kStage);
        if (!haspay) {  // stage its first out-edges now; they are read next round
            for (int j = 0; j < len; ++j) cp_async16(nedg + slot * kStage + j, a.erec + r.z + j);
            cp_async_commit();
        }
        go_global = false;
    }
    top += min(__popc(sm), max(room, 0));
    ws.local += (uint32_t)min(__popc(sm), max(room, 0));
    const int item = haspay ? a.n_tasks + a.npieces + r.z : v;
    const int to_main = (go_global && !topay && cls == 0) ? 1 : 0;
    if (a.ring) ring_push(a, rt, to_main, item, false, lane, ws);
    else push_items(a, a.queue, a.qcap, &a.ctrl->tail, to_main, item, false, lane, ws);
    if (PAY && a.pay_warps > 0) push_items(a, a.pqueue, a.pqcap, &a.ctrl->ptail, topay ? 1 : 0, item, false, lane, ws);
    if (PAY && a.pdir) {
        push_items(a, a.lqueue0, a.lqcap, &a.ctrl->ltail0, cls == 1 ? 1 : 0, item, false, lane, ws);
        push_items(a, a.lqueue1, a.lqcap, &a.ctrl->ltail1, cls == 2 ? 1 : 0, item, false, lane, ws);
    }
    if (ws.on) ws.cyc_push += (unsigned long long)(clk(ws) - c_push);
}

// Releases successor v of a finished task: returns true when v becomes ready, with its final
// key in *kv. f16 is v's in-degree from the edge record (kWideMark for wide joins).
__device__ __forceinline__ bool release_succ(const PersistArgs& a, int v, uint32_t ck, uint32_t f16,
                                             uint32_t* kv, uint32_t& ncas) {
    unsigned long long* st = a.state + v;
    if (f16 != kWideMark) {
        unsigned long long expected = ((unsigned long long)kKeyNegInf << 32) | f16;
        unsigned long long desired;
        for (;;) {
            const uint32_t ek = (uint32_t)(expected >> 32);
            const uint32_t ec = (uint32_t)expected;
            desired = ((unsigned long long)max(ek, ck) << 32) | (unsigned long long)(ec - 1u);
            const unsigned long long prev = atomicCAS(st, expected, desired);
            ++ncas;
            if (prev == expected) break;
            expected = prev;
        }
        *kv = (uint32_t)(desired >> 32);
        return (uint32_t)desired == 0u;
    }
    uint32_t* khalf = reinterpret_cast<uint32_t*>(st) + 1;
    int32_t* chalf = reinterpret_cast<int32_t*>(st);
    red_max(khalf, ck);
    fence_acq_rel();
    if (atom_dec_relaxed(chalf) != 1) return false;
    fence_acq_rel();
    *kv = ld_relaxed_u(khalf);
    return true;
}

// Releases every successor of this warp's finishing tasks (lane: task `fin` >= 0 with arrival
// key kt, first out-edge rs, out-degree deg), flattened over the warp 32 edges at a time, and
// pushes the ones that become ready with their key, row (payload index) and payload flag.
// Memory order: the arrival travels inside the state word, so plain releases need no fence.
// Payload data is ordered by fences: a warp fences after running payload pieces (release) and
// before running pieces of a task that became ready (acquire); queue publication fences; and
// without warp specialisation a window that releases a payload task fences first, so that data
// written upstream by a payload task reaches it through plain tasks in between (each such warp
// acquires what it observed, then releases).
// staged: this lane's task came from the warp's stack with its out-edges staged in
// cedg[lane * kStage ...]; nstk / nedg receive the tasks that become ready.
template <bool PAY>
__device__ __forceinline__ void release_all(const PersistArgs& a, int fin, uint32_t kt, int rs, int deg, bool staged,
                                            const int4* cedg, int4* nstk, int4* nedg, int& top, int* rt, int lane,
                                            WStats& ws) {
    const long long c_rel = clk(ws);
    if (fin < 0) deg = 0;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - deg;
    ws.edges += (uint32_t)total;
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + lane;
        int owner = 0;
#pragma unroll
        for (int b = 16; b >= 1; b >>= 1) {
            const int probe = owner + b - 1;
            const int iv = __shfl_sync(kFull, incl, probe);
            if (iv <= e) owner += b;
        }
        const int o_rs = __shfl_sync(kFull, rs, owner);
        const int o_ex = __shfl_sync(kFull, excl, owner);
        const uint32_t o_k = __shfl_sync(kFull, kt, owner);
        const bool o_st = __shfl_sync(kFull, staged ? 1 : 0, owner) != 0;
        int4 rec = make_int4(-1, 0, 0, 0);
        if (e < total) {
            const int j = e - o_ex;  // the first kStage edges of a stacked task are staged
            rec = (o_st && j < kStage) ? cedg[owner * kStage + j] : ld_stream_int4(a.erec + o_rs + j, l2_policy_first());
            // warm what the successor needs next while its CAS is in flight
            if ((uint32_t)rec.w & kPayBit) prefetch_l2(a.pay + rec.z);
            else prefetch_l2(a.erec + rec.z);
        }
        const uint32_t w = (uint32_t)rec.w;
        // (warp-specialised runs publish payload tasks through a queue, which fences already)
        if (PAY && a.pay_warps == 0 && __ballot_sync(kFull, rec.x >= 0 && (w & kPayBit))) fence_acq_rel();
        const long long c_cas = clk(ws);
        int4 r = make_int4(-1, 0, 0, 0);
        if (rec.x >= 0) {
            const float cand = __fadd_rn(key2f(o_k), __int_as_float(rec.y));
            uint32_t kv;
            if (release_succ(a, rec.x, f2key(cand), w & kWideMark, &kv, ws.cas)) {
                int len = (int)(w >> 16);
                if ((uint32_t)len == kLongMark) len = __ldg(a.meta + rec.x).y;
                r = make_int4(rec.x, (int)kv, rec.z, len | ((w & kPayBit) ? (int)0x80000000u : 0));
            }
        }
        const bool any_ready = __ballot_sync(kFull, r.x >= 0) != 0;
        if (ws.on) ws.cyc_cas += (unsigned long long)(clk(ws) - c_cas);
        if (any_ready) push_ready<PAY>(a, r, nstk, nedg, top, rt, lane, ws);
    }
    if (ws.on) ws.cyc_release += (unsigned long long)(clk(ws) - c_rel);
}

template <bool PAY>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 2) k_persist(const PersistArgs a) {
    __shared__ int4 s_stack[kWarpsPerCta][2][kStackCap];
    __shared__ int4 s_edges[kWarpsPerCta][2][kStackCap * kStage];
    __shared__ int s_ring[2];  // work stealing: this CTA's ring fill position, a lower bound of its take position
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_ring[0] = 0;
        s_ring[1] = 0;
    }
    __syncthreads();
    int pb = 0;  // buffer holding the stacked tasks; a round pops all of it and fills the other
    int top = 0;
    int qbase = 0;
    unsigned pend = 0;
    uint32_t last_done = 0xffffffffu;
    uint64_t stall_t0 = 0;
    unsigned backoff = 32;
    const int n_tasks = a.n_tasks;
    const int start_base = n_tasks + a.npieces;  // payload-start items begin here
    // role: in warp-specialised runs the last pay_warps warps of each CTA take their work from
    // the payload queue (payload starts and pieces); with copy warps, the copy_warps warps before
    // them take pull copies and the copy_warps before those push copies, each from their own
    // queue; the others take from the main queue
    const int pw = PAY ? a.pay_warps : 0;
    const int cw = (PAY && a.pdir) ? a.copy_warps : 0;
    const int role = wid >= kWarpsPerCta - pw            ? 1
                     : wid >= kWarpsPerCta - pw - cw     ? 2
                     : wid >= kWarpsPerCta - pw - 2 * cw ? 3
                                                         : 0;
    int32_t* const qslots = role == 1 ? a.pqueue : role == 2 ? a.lqueue0 : role == 3 ? a.lqueue1 : a.queue;
    const int qcap = role == 1 ? a.pqcap : role >= 2 ? a.lqcap : a.qcap;
    int32_t* const qhead = role == 1   ? &a.ctrl->phead
                           : role == 2 ? &a.ctrl->lhead0
                           : role == 3 ? &a.ctrl->lhead1
                                       : &a.ctrl->head;
    int32_t* const qtail = role == 1   ? &a.ctrl->ptail
                           : role == 2 ? &a.ctrl->ltail0
                           : role == 3 ? &a.ctrl->ltail1
                                       : &a.ctrl->tail;
    const int nwarps = (int)gridDim.x * (role == 1 ? pw : role >= 2 ? cw : kWarpsPerCta - pw - 2 * cw);
    // work stealing: main-queue warps take from rings (the other roles keep their queues)
    const bool steal = a.ring != nullptr && role == 0;
    uint32_t rng = ((uint32_t)blockIdx.x * kWarpsPerCta + (uint32_t)wid) * 2654435761u + 0x9e3779b9u;  // victims
    uint32_t ndone = 0;  // completions not yet added to ctrl->done (warp-uniform)
    uint32_t iter = 0;
    WStats ws;
    ws.on = a.stats != nullptr;

    for (;;) {
        int item = -1;
        int4 loc = make_int4(-1, 0, 0, 0);
        const int cb = pb;  // staged edges of this round's stacked tasks stay in buffer cb
        if (top > 0) {
            cp_async_wait_all();
            __syncwarp();
            if (lane < top) {
                loc = s_stack[wid][cb][lane];
                item = loc.x;
            }
            top = 0;
            pb ^= 1;
            __syncwarp();
        } else {
            int took = 0;  // items taken from a ring (lanes 0..took-1)
            if (pend == 0 && steal) took = ring_take_own(a, s_ring, a.claim, lane, item);
            if (pend == 0 && took == 0) {
                // claim a fair share of the published backlog (at least 1, at most `claim`); with
                // work stealing only slots the tail covers, since the global queue then holds just
                // sources and ring overflow, and a slot past the tail may never be filled
                int b = qcap, k = 0;
                if (lane == 0) {
                    const int h = ld_relaxed(qhead);
                    const int t = ld_relaxed(qtail);
                    if (h < qcap) {
                        k = max(1, min((t - h) / nwarps, a.claim));
                        if (!steal) {
                            b = atomicAdd(qhead, k);
                        } else {
                            k = t > h ? min(k, t - h) : 0;
                            if (k > 0 && atomicCAS(qhead, h, h + k) == h) b = h;
                            else k = 0;
                        }
                        ws.claims++;
                    }
                }
                b = __shfl_sync(kFull, b, 0);
                k = __shfl_sync(kFull, k, 0);
                qbase = b;
                k = min(k, qcap - b);
                pend = k <= 0 ? 0u : (k >= 32 ? kFull : ((1u << k) - 1u));
                if (steal && pend == 0 && gridDim.x > 1) {  // both empty: try a random victim
                    rng ^= rng << 13;
                    rng ^= rng >> 17;
                    rng ^= rng << 5;
                    int c = (int)(rng % (gridDim.x - 1u));
                    if (c >= (int)blockIdx.x) ++c;
                    took = ring_steal(a, c, a.claim, lane, item);
                    ws.steals += (uint32_t)took;
                }
            }
            if (pend & (1u << lane)) {
                const int v = ld_relaxed(qslots + qbase + lane);
                if (v >= 0) item = v;
            }
            const unsigned hit = __ballot_sync(kFull, item >= 0);
            pend &= ~hit;
            ws.pops += (uint32_t)__popc(hit);
            if (hit) fence_acq_rel();  // acquire: what the pusher released with the slot
        }
        const unsigned got = __ballot_sync(kFull, item >= 0);
        if (got == 0) {
            if (ndone && lane == 0) atomicAdd(&a.ctrl->done, ndone);
            ndone = 0;
            int quit = 0;
            if (lane == 0) {
                const uint32_t d = ld_relaxed_u(&a.ctrl->done);
                if (d >= (uint32_t)n_tasks || ld_relaxed(&a.ctrl->abort)) {
                    quit = 1;
                } else {
                    const uint64_t now = gtimer();
                    if (d != last_done) {
                        last_done = d;
                        stall_t0 = now;
                    } else if (now - stall_t0 > a.spin_limit_ns) {
                        atomicCAS(&a.ctrl->status, 0, (int)HF_ETIMEDOUT);
                        atomicExch(&a.ctrl->abort, 1);
                        quit = 1;
                    }
                }
            }
            if (__shfl_sync(kFull, quit, 0)) break;
            ws.idle++;
            __nanosleep(backoff);
            backoff = min(backoff * 2u, 256u);
            continue;
        }
        backoff = 32;
        ws.rounds++;
        const long long c_round = clk(ws);
        ws.items += (uint32_t)__popc(got);

        // ---- resolve this round's items: a task (with key, row, payload flag), a payload start
        // (to expand) or a payload piece
        int t = -1, p = -1, piece = 0;
        uint32_t kt = 0;
        int rs = 0, deg = 0;
        bool haspay = false, staged = false, expand = false, key_known = false;
        if (item >= 0) {
            if (item < n_tasks) {
                t = item;
                if (loc.x >= 0) {  // from the warp's stack: key, row and flag came along
                    kt = (uint32_t)loc.y;
                    key_known = true;
                    deg = loc.w & 0x7fffffff;
                    haspay = PAY && loc.w < 0;
                    if (haspay) {
                        p = loc.z;
                        expand = true;
                    } else {
                        rs = loc.z;
                        staged = true;
                    }
                } else {  // a task without payload from the main queue
                    const int2 mt = __ldg(a.meta + t);
                    rs = mt.x;
                    deg = mt.y;
                    kt = (uint32_t)(ld_relaxed_keep_u64(a.state + t, l2_policy_last()) >> 32);
                    key_known = true;
                }
            } else if (PAY) {
                haspay = true;
                if (item < start_base) {  // one piece of a multi-piece payload
                    const int g = item - n_tasks;
                    p = __ldg(a.chunk_pay + g);
                    piece = g - a.pay[p].chunk_first;
                } else {  // a payload start
                    p = item - start_base;
                    expand = true;
                }
                t = a.pay[p].task;
            }
            if (a.t_start) {
                const int64_t now = (int64_t)gtimer();
                if (expand || !haspay) a.t_start[t] = now;
                else atomicMin((long long*)(a.t_start + t), (long long)now);
            }
            if (a.exec_count) {
                const long long tk = (long long)atomicAdd(&a.ctrl->ticket, 1ull);
                if (expand || !haspay) a.tk_start[t] = tk;
                else atomicCAS((unsigned long long*)(a.tk_start + t), ~0ull, (unsigned long long)tk);
            }
        }

        // ---- phase 1: tasks without payload finish now and release their successors
        int fin = (item >= 0 && !haspay) ? t : -1;
        if (fin >= 0) {
            if (a.exec_count) {  // finish ticket before any successor is released
                a.tk_end[fin] = (int64_t)atomicAdd(&a.ctrl->ticket, 1ull);
                atomicAdd(a.exec_count + fin, 1);
            }
            a.key[fin] = kt;
        }
        if (__ballot_sync(kFull, fin >= 0))
            release_all<PAY>(a, fin, kt, rs, deg, staged, s_edges[wid][cb], s_stack[wid][pb], s_edges[wid][pb], top,
                             s_ring, lane, ws);
        if (a.t_end && fin >= 0) a.t_end[fin] = (int64_t)gtimer();
        ndone += (uint32_t)__popc(__ballot_sync(kFull, fin >= 0));

        // ---- phase 2: payload pieces, then the payload tasks that completed release theirs
        if (PAY) {
            unsigned work = __ballot_sync(kFull, haspay);
            if (work) {
                // expansion: a payload start (or a stacked payload task) of several pieces puts
                // pieces 1.. on the queue this warp serves and runs piece 0 here
                int nc = 1, cf = 0;
                if (haspay) {
                    nc = a.pay[p].nchunks;
                    cf = a.pay[p].chunk_first;
                }
                if (steal) ring_push(a, s_ring, (expand && nc > 1) ? nc - 1 : 0, n_tasks + cf + 1, true, lane, ws);
                else push_items(a, qslots, qcap, qtail, (expand && nc > 1) ? nc - 1 : 0, n_tasks + cf + 1, true, lane, ws);
                ws.pieces += (uint32_t)__popc(work);
                fence_acq_rel();  // acquire: inputs written by upstream payload tasks
                while (work) {
                    const int src = __ffs(work) - 1;
                    work &= work - 1;
                    const int pp = __shfl_sync(kFull, p, src);
                    const int pc = __shfl_sync(kFull, piece, src);
                    if (a.pay[pp].op == kPayHost) {  // a host task: this warp waits for the proxy
                        if (lane == 0 && a.post)
                            host_task_roundtrip(a.post, a.post_ctr, a.hdone, (int)a.pay[pp].a_bits, a.spin_limit_ns,
                                                &a.ctrl->status, &a.ctrl->abort);
                        __syncwarp();
                    } else {
                        run_piece(a.pay[pp], pc, lane);
                    }
                }
                fence_acq_rel();  // release: every lane's payload writes before any release below
                __syncwarp();
                int fin2 = -1;
                if (haspay) {
                    if (nc == 1) fin2 = t;
                    else if (atom_dec_acq_rel(a.chunks_left + p) == 1) fin2 = t;
                }
                if (fin2 >= 0) {
                    rs = a.pay[p].row;
                    deg = a.pay[p].deg;
                    if (!key_known) kt = (uint32_t)(ld_relaxed_keep_u64(a.state + t, l2_policy_last()) >> 32);
                    if (a.exec_count) {
                        a.tk_end[fin2] = (int64_t)atomicAdd(&a.ctrl->ticket, 1ull);
                        atomicAdd(a.exec_count + fin2, 1);
                    }
                    a.key[fin2] = kt;
                }
                if (__ballot_sync(kFull, fin2 >= 0))
                    release_all<PAY>(a, fin2, kt, rs, deg, false, s_edges[wid][cb], s_stack[wid][pb],
                                     s_edges[wid][pb], top, s_ring, lane, ws);
                if (a.t_end && fin2 >= 0) a.t_end[fin2] = (int64_t)gtimer();
                ndone += (uint32_t)__popc(__ballot_sync(kFull, fin2 >= 0));
            }
        }

        if (ws.on) ws.cyc_round += (unsigned long long)(clk(ws) - c_round);
        // completions reach ctrl->done in batches: when the warp goes idle, and every 32 rounds
        // so that the stall timer of idle warps sees progress made by long-busy warps
        if ((++iter & 31u) == 0 && ndone) {
            if (lane == 0) atomicAdd(&a.ctrl->done, ndone);
            ndone = 0;
        }
    }
    if (a.stats) {
        uint32_t cas = ws.cas;
        for (int o = 16; o > 0; o >>= 1) cas += __shfl_xor_sync(kFull, cas, o);
        if (lane == 0) {
            atomicAdd(a.stats + kStatRounds, (unsigned long long)ws.rounds);
            atomicAdd(a.stats + kStatItems, (unsigned long long)ws.items);
            atomicAdd(a.stats + kStatIdle, (unsigned long long)ws.idle);
            atomicAdd(a.stats + kStatEdges, (unsigned long long)ws.edges);
            atomicAdd(a.stats + kStatCas, (unsigned long long)cas);
            atomicAdd(a.stats + kStatPushLocal, (unsigned long long)ws.local);
            atomicAdd(a.stats + kStatPushGlobal, (unsigned long long)ws.global);
            atomicAdd(a.stats + kStatClaims, (unsigned long long)ws.claims);
            atomicAdd(a.stats + kStatPops, (unsigned long long)ws.pops);
            atomicAdd(a.stats + kStatPieces, (unsigned long long)ws.pieces);
            atomicAdd(a.stats + kStatCycRound, ws.cyc_round);
            atomicAdd(a.stats + kStatCycRelease, ws.cyc_release);
            atomicAdd(a.stats + kStatCycCas, ws.cyc_cas);
            atomicAdd(a.stats + kStatCycPush, ws.cyc_push);
            atomicAdd(a.stats + kStatRingPush, (unsigned long long)ws.ring);
            atomicAdd(a.stats + kStatSteals, (unsigned long long)ws.steals);
        }
    }
}

// New edge delays: delay[e] (edges in insertion order) into both edge layouts.
// A delay that is not finite is stored all the same and flagged in *bad (reported as
// HF_EINVAL by the next synchronisation).
__global__ void k_set_delays(const float* __restrict__ delay, const int32_t* __restrict__ pos_csr,
                             const int32_t* __restrict__ pos_ls, int4* erec, int2* ls_in, int64_t m,
                             int32_t* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool nonfinite = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int b = __float_as_int(__ldcs(delay + i));  // device or page-locked host memory, read once
        nonfinite |= (b & 0x7f800000) == 0x7f800000;
        reinterpret_cast<int*>(erec)[4 * (int64_t)__ldg(pos_csr + i) + 1] = b;
        reinterpret_cast<int*>(ls_in)[2 * (int64_t)__ldg(pos_ls + i) + 1] = b;
    }
    if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

__global__ void k_keys_to_f32(const uint32_t* __restrict__ key, float* __restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = key2f(key[i]);
}

}  // namespace hf
