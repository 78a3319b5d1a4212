// team.cuh -- the team executor for batches of independent graphs (sm_103a).
//
// One persistent launch runs a batch. Each graph is one job, run level by level in the pull
// form of the level-synchronous executor with a barrier between levels instead of a kernel
// boundary. A solo job belongs to one CTA and ends each level with a CTA barrier; a cluster job
// belongs to the CTAs of one thread-block cluster, which split each level among themselves and
// end it with the hardware cluster barrier. Independent graphs never wait for one another, so
// a batch costs its longest graph's chain of levels, not the sum over merged levels.
//
// Latency hiding. A level's critical path should be one gather of the predecessors' arrival
// keys. Everything that does not depend on the previous level is fetched ahead:
//   * segment descriptors (positions, in-edge and payload-piece ranges of each level) five
//     levels ahead, by asynchronous copies into a ring in shared memory, each waited for one
//     level after it was issued;
//   * every CTA stages the task list, row starts, in-edges and payload-piece descriptors of the
//     next three levels in shared memory with TMA bulk copies (four buffers, completion on
//     mbarriers); segments too large to stage are prefetched into L2 three levels ahead. All of
//     it is issued by a producer warp that takes no arrivals, so its issue time (~0.35 us per
//     level) is off the arrival warps' path;
//   * in cluster jobs, each CTA prefetches the x and y ranges of its next-level pieces into L2;
//   * graphs whose keys outgrow L1 run software-pipelined: a thread reads its next level's task
//     (id, in-edge range) while its current key loads are in flight, and issues that task's
//     first key loads as the very first thing of the next level. A level's gather is bound by
//     the SM's rate of scattered L1 misses (about one per cycle: ~900 for a 250-task level with
//     3.5 in-edges a task) plus an L2 round trip; set-up work beside it costs nothing as long as
//     it does not wait in the same queue.
// Balance. Each CTA of a team takes a contiguous slice of every level's tasks (one per thread)
// and of its payload pieces; the CTA's warps claim pieces one at a time from a shared counter,
// warps without arrivals at once, the others when their arrivals are done.
#pragma once

#include "kernels.cuh"

namespace hf {

constexpr int kTeamThreads = 256;
constexpr int kTeamBufs = 4;       // staged levels: the current one and three ahead
// Segment descriptors ride a ring in shared memory, fetched kRingAhead levels ahead by
// asynchronous copies (one commit group per level); a level's barrier waits only for the group
// of the level before, so no fetch latency sits on a level's own path. An entry must have landed
// when the look-ahead stages its level (kTeamBufs - 1 levels ahead): kRingAhead = kTeamBufs + 1.
constexpr int kStageAhead = kTeamBufs - 1;  // levels staged ahead of the current one
constexpr int kRingAhead = kTeamBufs + 1;
constexpr int kRing = 8;           // ring slots (a power of two above kRingAhead)
static_assert(kRing > kRingAhead && (kRing & (kRing - 1)) == 0, "ring slots");
// kTeamThreads arrival threads (one task each per level) and a producer warp: the thread that
// runs a CTA's look-ahead (segment ring, stage copies) is its lane 0; the warp also claims
// payload pieces and, in cluster jobs, warms L2 with the next level's pieces.
constexpr int kTeamLead = kTeamThreads;
constexpr int kTeamBlock = kTeamThreads + 32;
// Stage buffers live in dynamic shared memory, sized per plan (TeamArgs::stage_n tasks,
// stage_e in-edges and stage_p piece descriptors per level; stage_n a multiple of 4, stage_e of
// 2): node[stage_n + 8] (copied from a 16-byte aligned start, up to 3 extra entries in front),
// ptr[stage_n + 12] (one more row start), in[stage_e + 2], pdesc[stage_p].
__host__ __device__ constexpr size_t team_stage_bytes(int stage_n, int stage_e, int stage_p) {
    return (size_t)(stage_n + 8) * 4 + (size_t)(stage_n + 12) * 4 + (size_t)(stage_e + 2) * 8 +
           (size_t)stage_p * sizeof(TeamPiece);
}

// One stage buffer carved out of dynamic shared memory.
struct TeamStage {
    int32_t* node;
    int32_t* ptr;
    int2* in;
    TeamPiece* pdesc;
};

__device__ __forceinline__ TeamStage team_stage_view(unsigned char* base, int b, int stage_n, int stage_e, int stage_p) {
    unsigned char* p = base + (size_t)b * team_stage_bytes(stage_n, stage_e, stage_p);
    TeamStage st;
    st.node = reinterpret_cast<int32_t*>(p);
    st.ptr = st.node + stage_n + 8;
    st.in = reinterpret_cast<int2*>(st.ptr + stage_n + 12);
    st.pdesc = reinterpret_cast<TeamPiece*>(st.in + stage_e + 2);
    return st;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking: has the phase with this parity completed? (acquire at CTA scope, like try_wait,
// but never suspends the thread)
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* bar, unsigned parity) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s), "r"(parity)
        : "memory");
    return ok != 0;
}

// all but the most recent commit group of this thread's asynchronous copies have landed
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// asynchronous 8-byte global -> shared copy (completion: cp_async_wait_all by the issuer)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}

// TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// L2 bulk prefetch of the whole 16-byte blocks inside [p, p + bytes)
__device__ __forceinline__ void prefetch_l2_range(const void* p, int64_t bytes) {
    uint64_t a0 = ((uint64_t)p + 15) & ~15ull;
    const uint64_t a1 = ((uint64_t)p + (uint64_t)bytes) & ~15ull;
    while (a1 > a0) {
        const unsigned b = (unsigned)(a1 - a0 < 65536 ? a1 - a0 : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"(b) : "memory");
        a0 += b;
    }
}

// The staging sources and capacities, copied from TeamArgs into shared memory at kernel start,
// where the look-ahead reads them.
struct TeamSrc {
    const int32_t* ls_node;
    const int32_t* ls_ptr;
    const int2* ls_in;
    const TeamPiece* pdesc;
    int32_t stage_n, stage_e, stage_p, pad_;
};

template <class S>
__device__ __forceinline__ bool team_fits(const S& a, const int4 sg) {
    return sg.y > sg.x && sg.y - sg.x <= a.stage_n && sg.w - sg.z <= a.stage_e;
}

// (64-bit difference: a range never overflows into a "fitting" one)
template <class S>
__device__ __forceinline__ bool team_desc_fits(const S& a, const int2 si) {
    return si.x >= 0 && si.y > si.x && (int64_t)si.y - (int64_t)si.x <= (int64_t)a.stage_p;
}

// Issued by one thread: stage segment sg (positions [x, y), in-edges [z, w)) into st, and the
// level's piece descriptors si = [i0, i1) when they fit. The level-sorted arrays are allocated
// with slack so that rounding the ends up to 16 bytes stays inside them.
__device__ __forceinline__ void team_stage(const TeamSrc& a, const TeamStage& st, unsigned long long* bar, const int4 sg,
                                           const int2 si) {
    const int a0 = sg.x & ~3, a1 = (sg.y + 3) & ~3, b1 = (sg.y + 4) & ~3;
    const int c0 = sg.z & ~1, c1 = (sg.w + 1) & ~1;
    const unsigned bn = (unsigned)(a1 - a0) * 4u, bp = (unsigned)(b1 - a0) * 4u, bi = (unsigned)(c1 - c0) * 8u;
    const unsigned bd = team_desc_fits(a, si) ? (unsigned)(si.y - si.x) * (unsigned)sizeof(TeamPiece) : 0u;
    mbar_arrive_expect_tx(bar, bn + bp + bi + bd);
    bulk_g2s(st.node, a.ls_node + a0, bn, bar);
    bulk_g2s(st.ptr, a.ls_ptr + a0, bp, bar);
    if (bi) bulk_g2s(st.in, a.ls_in + c0, bi, bar);
    if (bd) bulk_g2s(st.pdesc, a.pdesc + si.x, bd, bar);
}

__device__ __forceinline__ void team_prefetch_seg(const TeamSrc& a, const int4 sg) {
    if (sg.y <= sg.x) return;
    prefetch_l2_range(a.ls_node + sg.x, 4ll * (sg.y - sg.x));
    prefetch_l2_range(a.ls_ptr + sg.x, 4ll * (sg.y - sg.x + 1));
    prefetch_l2_range(a.ls_in + sg.z, 8ll * (sg.w - sg.z));
}

// look-ahead for one level, by the lead thread of each CTA: stage it if it fits, else (CTA 0 of
// the team) prefetch it into L2. Inline: the sources come from shared memory, so the address
// arithmetic stays within the three-CTAs-per-SM register budget.
__device__ __forceinline__ bool team_ahead(const TeamSrc& a, int rank, const TeamStage& st, unsigned long long* bar,
                                           const int4 sg, const int2 si) {
    if (team_fits(a, sg)) {
        team_stage(a, st, bar, sg, si);
        return true;
    }
    if (rank == 0) team_prefetch_seg(a, sg);
    return false;
}

// The slice [x0 + n * r / k, x0 + n * (r + 1) / k) of a range of n that CTA r of a team of k takes.
// lk = log2(k) when k is a power of two (every planned team), else -1 (a 64-bit division, which
// costs as much as a level's gather).
__device__ __forceinline__ int team_slice(int x0, int n, int r, int k, int lk) {
    const int64_t m = (int64_t)n * r;
    return x0 + (int)(lk >= 0 ? m >> lk : m / k);
}

// L2 prefetch of the x and y ranges of staged pieces [i0, i1) (indices into the stage buffer's
// descriptors; one warp, lanes strided); saxpy pieces only (copies touch host memory, host
// tasks no memory).
__device__ __forceinline__ void team_prefetch_pieces(const TeamPiece* dsc, int i0, int i1, int lane) {
    for (int it = i0 + lane; it < i1; it += 32) {
        const TeamPiece d = dsc[it];
        if ((d.op != kPaySaxpyF32 && d.op != kPaySaxpyI32) || d.cnt <= 0) continue;
        prefetch_l2_range(d.src, 4ll * d.cnt);
        prefetch_l2_range(d.dst, 4ll * d.cnt);
    }
}

// One FP32 saxpy piece by one warp, with 32-bit indexing (a piece is at most a few thousand
// elements): a 512-element piece is one round trip of 16-byte loads, the ragged head and tail
// loaded alongside; same access pattern as warp_saxpy_f32.
__device__ __forceinline__ void team_saxpy_f32(float* __restrict__ y, const float* __restrict__ x, int cnt, float a,
                                               int lane) {
    if ((((uintptr_t)y ^ (uintptr_t)x) & 15) != 0) {
        for (int i = lane; i < cnt; i += 32) y[i] = __fmaf_rn(a, __ldcg(x + i), __ldcg(y + i));
        return;
    }
    int head = (int)(((16 - ((uintptr_t)y & 15)) & 15) >> 2);
    if (head > cnt) head = cnt;
    const int nv = (cnt - head) >> 2, tail0 = head + 4 * nv;
    // lanes [0, head) take the unaligned leading elements, the next cnt - tail0 lanes the
    // trailing ones (at most 3 + 3)
    const bool scalar = lane < head + (cnt - tail0);
    const int li = lane < head ? lane : tail0 + (lane - head);
    float sx = 0.f, sy = 0.f;
    if (scalar) {
        sx = __ldcg(x + li);
        sy = __ldcg(y + li);
    }
    float4* __restrict__ y4 = reinterpret_cast<float4*>(y + head);
    const float4* __restrict__ x4 = reinterpret_cast<const float4*>(x + head);
    for (int k = lane; k - lane < nv; k += 128) {
        float4 xv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = k + 32 * u < nv ? k + 32 * u : nv - 1;
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
    if (scalar) y[li] = __fmaf_rn(a, sx, sy);
}

__device__ __forceinline__ void team_run_piece(const TeamPiece& d, int lane) {
    if (d.op == kPaySaxpyF32)
        team_saxpy_f32(reinterpret_cast<float*>(d.dst), reinterpret_cast<const float*>(d.src), d.cnt,
                       __uint_as_float(d.a), lane);
    else if (d.op == kPaySaxpyI32)
        warp_saxpy_i32(reinterpret_cast<int32_t*>(d.dst), reinterpret_cast<const int32_t*>(d.src), d.cnt, d.a, lane);
    else if (d.op == kPayCopy)
        warp_copy(d.dst, d.src, d.cnt, lane);
}

// ---------------------------------------------------------------- host tasks

// The host tasks of one level (thread 0 of the team's first CTA, after the level's device work):
// post each to the mailbox in mapped host memory, where the host proxy thread runs it, and
// wait until all of them have run (bounded by spin_limit_ns). The system-scope fence makes the
// graph's earlier device writes (push copies into host memory) visible to the callbacks; the
// acquire of each done flag orders the callbacks' writes before later levels. Returns false
// when a callback did not finish in time, or when the run is already aborting (nothing is
// posted then): the caller ends the team's run.
__device__ __noinline__ bool team_host_tasks(const TeamArgs& a, int seg) {
    const int2 hr = __ldg(a.seg_host + seg);
    if (hr.y <= hr.x) return true;
    if (ld_relaxed(&a.ctrl->abort)) return false;
    __threadfence_system();
    for (int h = hr.x; h < hr.y; ++h) st_release_sys(a.post + atomicAdd(a.post_ctr, 1), __ldg(a.host_order + h));
    for (int h = hr.x; h < hr.y; ++h) {
        const int k = __ldg(a.host_order + h);
        const uint64_t t0 = gtimer();
        while (ld_acquire_sys(a.hdone + k) == 0) {
            if (gtimer() - t0 > a.spin_limit_ns) return false;
            __nanosleep(200);
        }
    }
    return true;
}

// ---------------------------------------------------------------- thread-block cluster helpers

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size() {
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}

// every thread of every CTA of the cluster; release/acquire at cluster scope
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The same barrier with a relaxed arrive: it orders nothing by itself; a thread whose writes other
// CTAs read after the barrier releases them first with fence_cluster (the fence and the arrive
// form the release), and the wait still acquires
__device__ __forceinline__ void cluster_sync_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }

// store a job into CTA `rank`'s copy of the shared variable `local`
__device__ __forceinline__ void st_cluster_job(TeamJob* local, unsigned rank, const TeamJob j) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(local);
    unsigned d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(s), "r"(rank));
    asm volatile("st.shared::cluster.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(d), "r"(j.graph), "r"(j.flags), "r"(j.seg0),
                 "r"(j.levels)
                 : "memory");
}

// Failure of a team (a staged copy or a host task ran out of its time limit): the run's status
// becomes `status` (first failure wins), the run aborts (no new job starts), and the team's
// failure flag -- in the shared memory of every CTA of the team -- is raised. Every CTA reads
// its own flag after the level's barrier, so all threads of all CTAs of the team see the same
// value there and leave the job together; no CTA is left waiting at a barrier.
__device__ __noinline__ void team_fail(const TeamArgs& a, int* s_fail, int k, int status) {
    atomicCAS(&a.ctrl->status, 0, status);
    atomicExch(&a.ctrl->abort, 1);
    if (k == 1) {
        *(volatile int*)s_fail = 1;
        return;
    }
    const unsigned s = (unsigned)__cvta_generic_to_shared(s_fail);
    for (int r = 0; r < k; ++r) {
        unsigned d;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(s), "r"(r));
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(d), "r"(1) : "memory");
    }
    fence_cluster();  // (released before the level's barrier, whose arrive may be relaxed)
}

// ---------------------------------------------------------------- one level

// Arrival keys are loaded and stored with an L2 evict-last policy: a predecessor may sit
// anywhere earlier in its graph, and the keys should stay in L2 while the payload pieces stream
// through it with evict-first hints.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Predecessors' keys were written by this CTA (solo job: ordinary loads, L1 may hold them) or
// by another CTA of the cluster (loads from L2, after the cluster barrier's acquire).
template <bool SOLO>
__device__ __forceinline__ uint32_t team_pred_key(const TeamArgs& a, int u, uint64_t pol) {
    uint32_t v;
    if (SOLO)
        asm volatile("ld.global.ca.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a.key + u), "l"(pol) : "memory");
    else
        asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a.key + u), "l"(pol) : "memory");
    return v;
}

__device__ __forceinline__ void team_store_key(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// max over in-edges [e0, e1) of key(arr[u] + d): all key loads of a batch of up to 8 in-edges
// are issued before the first is used, so a task's gather costs one round trip
template <bool SOLO>
__device__ __forceinline__ uint32_t team_fold(const TeamArgs& a, const int2* in, int e0, int e1, uint64_t pol) {
    uint32_t best = 0u;
    for (int e = e0; e < e1; e += 8) {
        const int cnt = e1 - e < 8 ? e1 - e : 8;
        uint32_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) kk[j] = team_pred_key<SOLO>(a, in[e + j].x, pol);
        // the delays are read again once the keys are in (fewer live registers)
        const volatile int* dl = reinterpret_cast<const volatile int*>(in + e) + 1;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) best = max(best, f2key(__fadd_rn(key2f(kk[j]), __int_as_float(dl[2 * j]))));
    }
    return best;
}

template <bool SOLO>
__device__ __forceinline__ uint32_t team_task_key(const TeamArgs& a, int v, const int2* in, int e0, int e1,
                                                  uint64_t pol) {
    if (e0 == e1) return a.key0 ? __ldg(a.key0 + v) : kKeyPosZero;
    return team_fold<SOLO>(a, in, e0, e1, pol);
}

// team_task_key, running `between()` once while the first batch of key loads is in flight (the
// loads are issued, their first use comes after it), so that work for the next level costs no
// time on this level's path
template <bool SOLO, class F>
__device__ __forceinline__ uint32_t team_task_key_hook(const TeamArgs& a, int v, const int2* in, int e0, int e1,
                                                       uint64_t pol, F&& between) {
    if (e0 == e1) {
        const uint32_t k0 = a.key0 ? __ldg(a.key0 + v) : kKeyPosZero;
        between();
        return k0;
    }
    uint32_t best = 0u;
    for (int e = e0; e < e1; e += 8) {
        const int cnt = e1 - e < 8 ? e1 - e : 8;
        uint32_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) kk[j] = team_pred_key<SOLO>(a, in[e + j].x, pol);
        if (e == e0) between();
        const volatile int* dl = reinterpret_cast<const volatile int*>(in + e) + 1;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) best = max(best, f2key(__fadd_rn(key2f(kk[j]), __int_as_float(dl[2 * j]))));
    }
    return best;
}

// ---------------------------------------------------------------- keys in distributed shared memory
//
// A level's gather in a cluster job loads its predecessors' keys, written by the team's CTAs at
// earlier levels, through L2 (0.6-0.9 us per level measured; a load from a cluster peer's shared
// memory is about 0.1-0.2 us). A graph whose keys fit in the shared memory of its cluster's CTAs
// therefore keeps them there for the whole job: task i of the graph (its id minus the graph's
// first id) in CTA i & (k - 1) of the cluster of k = 2^lk CTAs, at slot i >> lk, loaded and
// stored through distributed shared memory; the cluster barrier orders a level's stores before
// the next level's loads. The keys go to global memory once, after the last level, each CTA
// writing its own slots. (Single-CTA jobs keep their keys in global memory: measured, a table in
// their own shared memory did not shorten a level, and the larger shared-memory carve-out left
// less L1 to the other single-CTA jobs' key loads.)

// distributed-shared-memory address of task i's key in its owner CTA
__device__ __forceinline__ unsigned sk_addr(unsigned skey_s, int i, int lk) {
    unsigned d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(d)
                 : "r"(skey_s + 4u * (unsigned)(i >> lk)), "r"(i & ((1 << lk) - 1)));
    return d;
}

// (no memory clobber: the loads may be scheduled freely within the level; the level barriers
// are volatile and order them)
__device__ __forceinline__ uint32_t sk_load(unsigned addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void sk_store(unsigned addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// team_task_key with the graph's keys in distributed shared memory (kbase: the graph's first
// task id): the in-edge records of a batch of up to 8 are read first, then every key load is
// issued, then they are combined
__device__ __forceinline__ uint32_t team_task_key_sk(const TeamArgs& a, int v, const int2* in, int e0, int e1,
                                                     unsigned skey_s, int kbase, int lk) {
    if (e0 == e1) return a.key0 ? __ldg(a.key0 + v) : kKeyPosZero;
    uint32_t best = 0u;
    for (int e = e0; e < e1; e += 8) {
        const int cnt = e1 - e < 8 ? e1 - e : 8;
        int2 r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) r[j] = in[e + j];
        uint32_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) kk[j] = sk_load(sk_addr(skey_s, r[j].x - kbase, lk));
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) best = max(best, f2key(__fadd_rn(key2f(kk[j]), __int_as_float(r[j].y))));
    }
    return best;
}

// ---------------------------------------------------------------- one graph

// Bounded wait (spin_limit_ns) for stage buffer b's next completion; false if it never came.
__device__ __forceinline__ bool team_wait_stage(unsigned long long* bar, unsigned parity, uint64_t limit_ns) {
    uint64_t t0 = 0;
    while (!mbar_try_wait(bar, parity)) {
        const uint64_t now = gtimer();
        if (!t0) t0 = now;
        else if (now - t0 > limit_ns) return false;
    }
    return true;
}

// Runs job `job` on a team of k CTAs (this one is `rank`; SOLO: k = 1): level by level, staged
// levels (task list, in-edges, piece descriptors) from shared memory, the rest from global
// memory (prefetched into L2), payload pieces spread over the team's warps, then the team
// barrier (CTA barrier for a solo job, cluster barrier otherwise). Returns false when the team
// failed (a staged copy or a host task ran out of time, see team_fail): every thread of every
// CTA of the team returns false after the same level barrier, and the lead thread has first
// waited (bounded) for the stage copies it still had in flight; the kernel then ends.
// A thread whose wait for a staged level runs out reads that level from global memory instead
// (the same data), so the level completes and the team reaches its barrier.
// SK (cluster jobs only): the graph's keys live in distributed shared memory (see above; skey:
// this CTA's table). Only in the kernel without payloads: with them the extra path would spill
// registers.
template <bool PAY, bool SOLO, bool REC, bool SK>
__device__ __forceinline__ bool team_run_graph(const TeamArgs& a, const TeamJob& job, int k, int rank,
                                               const TeamSrc& src, const TeamStage* sview, unsigned long long* mbar,
                                               int4* ring, int2* iring, int* pcnt, int* s_fail, unsigned& phase,
                                               uint32_t* skey) {
    const int t = threadIdx.x;
    const int lane = t & 31;
    static_assert(!(SK && SOLO), "shared key tables are for cluster jobs");
    const int L = job.levels;
    const int lk = (k & (k - 1)) == 0 ? __ffs(k) - 1 : -1;
    const int2 z2 = make_int2(0, 0);
    const int kbase = SK ? __ldg(a.task_off + job.graph) : 0;
    const unsigned skey_s = SK ? (unsigned)__cvta_generic_to_shared(skey) : 0u;
    unsigned inflight = 0;  // lead thread: stage buffers with a copy issued and not yet seen complete
    // Software pipelining across levels (pipe: jobs flagged kJobPipelined): while its first task's
    // key loads are in flight, a thread tests (without waiting) whether the next level's stage
    // buffer has landed and, if so, reads its first task of that level (id, in-edge range, stage
    // pointer) from it; the kernel without payloads then issues that task's first eight key loads
    // as the very first thing of the next level. `seen`: buffers whose current completion this
    // thread has already observed; pv/pe0/pe1/pin (valid: pvalid): the task read ahead.
    unsigned seen = 0;
    int pv = 0, pe0 = 0, pe1 = 0;
    bool pvalid = false;
    const int2* pin = nullptr;  // the read-ahead task's in-edges (its level's stage buffer)
    const bool pipe = (job.flags & kJobPipelined) != 0;
    // cluster jobs whose payloads touch disjoint memory (kJobPayloadLocal): a level releases its
    // arrival keys alone (each thread that stored one fences), not the pieces' stores
    const bool plocal = PAY && !SOLO && (job.flags & kJobPayloadLocal) != 0;
    const uint64_t pol = l2_keep_policy();
    // segment descriptors and item ranges ride a ring in shared memory, fetched by the lead
    // thread kRingAhead levels ahead (the first kRingAhead here); level l uses stage buffer
    // l % kTeamBufs, staged kTeamBufs - 1 levels ahead
    if (t == kTeamLead) {
        cp_async_wait_all();  // (the previous job's ring copies have all landed; none in flight)
        pcnt[0] = pcnt[1] = 0;
        for (int q = 0; q < kRingAhead && q < L; ++q) {
            ring[q] = __ldg(a.seg + job.seg0 + q);
            iring[q] = PAY ? __ldg(a.seg_items + job.seg0 + q) : z2;
        }
        for (int q = 0; q < kStageAhead && q < L; ++q)
            if (team_ahead(src, rank, sview[q], &mbar[q], ring[q], PAY ? iring[q] : z2)) inflight |= 1u << q;
    }
    __syncthreads();
    if (a.g_start && rank == 0 && t == 0) a.g_start[job.graph] = (int64_t)gtimer();
    for (int l = 0; l < L; ++l) {
        const int b = l % kTeamBufs;
        // the read-ahead task's first key loads go out before the rest of the level's set-up
        uint32_t kk0[8];
        int c0n = -1;
        if (!PAY && !REC && !SK && pvalid) {  // (the payload kernel has no registers to spare)
            c0n = min(pe1 - pe0, 8);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < c0n) kk0[j] = team_pred_key<SOLO>(a, pin[pe0 + j].x, pol);
        }
        const int4 s0 = ring[l & (kRing - 1)];
        const int2 i0 = PAY ? iring[l & (kRing - 1)] : z2;
        if (t == kTeamLead) {
            const int la = l + kStageAhead;
            if (la < L && team_ahead(src, rank, sview[la % kTeamBufs], &mbar[la % kTeamBufs],
                                     ring[la & (kRing - 1)], PAY ? iring[la & (kRing - 1)] : z2))
                inflight |= 1u << (la % kTeamBufs);  // (the item ring is filled only with payloads)
            if (l + kRingAhead < L) {
                cp_async16(&ring[(l + kRingAhead) & (kRing - 1)], a.seg + job.seg0 + l + kRingAhead);
                if (PAY) cp_async8(&iring[(l + kRingAhead) & (kRing - 1)], a.seg_items + job.seg0 + l + kRingAhead);
            }
            cp_async_commit();  // one group per level (empty near the end)
        }
        if (PAY && t == kTeamLead) pcnt[(l + 1) & 1] = 0;  // the next level's piece counter (free since the barrier)
        // level l's task list, row starts and in-edges (every CTA of a team stages the whole level):
        // from the stage buffer, which holds them from position nb, in-edge eb and item ib on
        // (indices are rebased; a pointer is never moved outside its buffer), else from memory
        const int32_t* node = a.ls_node;
        const int32_t* ptr = a.ls_ptr;
        const int2* in = a.ls_in;
        const TeamPiece* dsc = PAY ? a.pdesc : nullptr;
        int nb = 0, eb = 0, ib = 0;
        if (team_fits(a, s0)) {
            bool landed = ((seen >> b) & 1u) != 0;  // observed during the previous level
            seen &= ~(1u << b);
            if (!landed && team_wait_stage(&mbar[b], (phase >> b) & 1u, a.spin_limit_ns)) {
                phase ^= 1u << b;
                landed = true;
            }
            if (landed) {
                if (t == kTeamLead) inflight &= ~(1u << b);
                nb = s0.x & ~3;
                eb = s0.z & ~1;
                const TeamStage sv = sview[b];
                node = sv.node;
                ptr = sv.ptr;
                in = sv.in;
                if (PAY && team_desc_fits(a, i0)) {
                    dsc = sv.pdesc;
                    ib = i0.x;
                }
            } else {  // a bulk copy that never landed: this level from memory, then the team ends
                team_fail(a, s_fail, k, (int)HF_ETIMEDOUT);
            }
        }
        // this CTA's slice of the level's tasks: one per thread
        {
            const int p1 = team_slice(s0.x, s0.y - s0.x, rank + 1, k, lk);
            bool nvalid = false;
            int nv = 0, ne0 = 0, ne1 = 0;
            const int2* nin = nullptr;
            auto look_next = [&]() {
                if (!pipe || l + 1 >= L) return;
                const int4 s1 = ring[(l + 1) & (kRing - 1)];
                if (!team_fits(a, s1)) return;
                const int b1 = (l + 1) % kTeamBufs;
                if (!mbar_test_wait(&mbar[b1], (phase >> b1) & 1u)) return;
                phase ^= 1u << b1;
                seen |= 1u << b1;
                if (t == kTeamLead) inflight &= ~(1u << b1);
                const int q = team_slice(s1.x, s1.y - s1.x, rank, k, lk) + t;
                if (t < kTeamThreads && q < team_slice(s1.x, s1.y - s1.x, rank + 1, k, lk)) {
                    const TeamStage sv = sview[b1];
                    const int nb1 = s1.x & ~3, eb1 = s1.z & ~1;
                    nv = sv.node[q - nb1];
                    ne0 = sv.ptr[q - nb1] - eb1;
                    ne1 = sv.ptr[q + 1 - nb1] - eb1;
                    nin = sv.in;
                    nvalid = true;
                }
            };
            int p = team_slice(s0.x, s0.y - s0.x, rank, k, lk) + t;
            const bool stored = t < kTeamThreads && p < p1;  // this thread stores at least one key
            if (!pipe) {
                // (jobs that are not pipelined keep the plain loop: with the pipelined path compiled
                // in their levels measured slower, keys in L1 leaving nothing to hide)
            } else if (t < kTeamThreads && p < p1) {  // the first task: pipelined
                int v, e0, e1;
                if (pvalid) {
                    v = pv;
                    e0 = pe0;
                    e1 = pe1;
                } else {
                    v = node[p - nb];
                    e0 = ptr[p - nb] - eb;
                    e1 = ptr[p + 1 - nb] - eb;
                }
                const uint64_t c0 = REC ? gtimer() : 0;
                if (c0n >= 0) {  // its first key loads went out at the top of the level
                    look_next();
                    uint32_t best = e0 == e1 ? (a.key0 ? __ldg(a.key0 + v) : kKeyPosZero) : 0u;
                    const volatile int* dl = reinterpret_cast<const volatile int*>(in + e0) + 1;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < c0n) best = max(best, f2key(__fadd_rn(key2f(kk0[j]), __int_as_float(dl[2 * j]))));
                    if (e1 - e0 > 8) best = max(best, team_fold<SOLO>(a, in, e0 + 8, e1, pol));
                    team_store_key(a.key + v, best, pol);
                } else if (SK) {
                    sk_store(sk_addr(skey_s, v - kbase, lk), team_task_key_sk(a, v, in, e0, e1, skey_s, kbase, lk));
                    if (REC) a.t_cost[v] = (float)(gtimer() - c0);
                    look_next();
                } else if (REC) {
                    team_store_key(a.key + v, team_task_key<SOLO>(a, v, in, e0, e1, pol), pol);
                    a.t_cost[v] = (float)(gtimer() - c0);
                    look_next();
                } else {
                    team_store_key(a.key + v, team_task_key_hook<SOLO>(a, v, in, e0, e1, pol, look_next), pol);
                }
                p += kTeamThreads;
            } else {
                look_next();
            }
            pvalid = false;
            for (; t < kTeamThreads && p < p1; p += kTeamThreads) {
                const int v = node[p - nb];
                const uint64_t c0 = REC ? gtimer() : 0;
                if (SK)
                    sk_store(sk_addr(skey_s, v - kbase, lk),
                             team_task_key_sk(a, v, in, ptr[p - nb] - eb, ptr[p + 1 - nb] - eb, skey_s, kbase, lk));
                else
                    team_store_key(a.key + v,
                                   team_task_key<SOLO>(a, v, in, ptr[p - nb] - eb, ptr[p + 1 - nb] - eb, pol), pol);
                if (REC) a.t_cost[v] = (float)(gtimer() - c0);  // the gather's time (loads in, key out)
            }
            pvalid = nvalid;
            pv = nv;
            pe0 = ne0;
            pe1 = ne1;
            pin = nin;
            if (plocal && stored) fence_cluster();  // the keys, before this thread's pieces
        }
        // this CTA's slice of the level's payload pieces: each warp takes the next piece from a
        // shared counter, the warps without arrivals at once, the others after them. In cluster
        // jobs the last warp first warms L2 with the CTA's pieces of the next level, when that
        // level's staged descriptors have landed.
        if (PAY) {
            if (!SOLO && (t >> 5) == (kTeamLead >> 5) && l + 1 < L) {
                const int b1 = (l + 1) % kTeamBufs;
                const int2 i1 = iring[(l + 1) & (kRing - 1)];
                // landed: observed by this thread's look at the next level, or by a test now
                // (never a wait: the prefetch is not worth holding the warp)
                if (team_fits(a, ring[(l + 1) & (kRing - 1)]) && team_desc_fits(a, i1) &&
                    (((seen >> b1) & 1u) || mbar_test_wait(&mbar[b1], (phase >> b1) & 1u)))
                    team_prefetch_pieces(sview[b1].pdesc, team_slice(i1.x, i1.y - i1.x, rank, k, lk) - i1.x,
                                         team_slice(i1.x, i1.y - i1.x, rank + 1, k, lk) - i1.x, lane);
            }
            const int q0 = team_slice(i0.x, i0.y - i0.x, rank, k, lk);
            const int q1 = team_slice(i0.x, i0.y - i0.x, rank + 1, k, lk);
            for (;;) {
                int it = 0;
                if (lane == 0) it = q0 + atomicAdd(&pcnt[l & 1], 1);
                it = __shfl_sync(0xffffffffu, it, 0);
                if (it >= q1) break;
                const uint64_t c0 = REC ? gtimer() : 0;
                team_run_piece(dsc[it - ib], lane);
                if (REC) {  // a payload task's cost: its pieces' warp times summed
                    __syncwarp();
                    if (lane == 0) atomicAdd(a.t_cost + dsc[it - ib].task, (float)(gtimer() - c0));
                }
            }
        }
        if (a.seg_host && rank == 0 && t == 0 && !team_host_tasks(a, job.seg0 + l))
            team_fail(a, s_fail, k, (int)HF_ETIMEDOUT);
        // the ring group of level l - 1 (entry l - 1 + kRingAhead, staged at level l + 1); this
        // level's own group stays in flight across the barrier
        if (t == kTeamLead) cp_async_wait_group1();
        if (SOLO) {
            __syncthreads();
        } else if (plocal) {  // the CTA's shared state (piece counter, ring) by the CTA barrier
            __syncthreads();
            cluster_sync_relaxed();
        } else {
            cluster_sync();
        }
        if (*(volatile int*)s_fail) {  // the same value in every thread of the team (see team_fail)
            if (t == kTeamLead) {      // stage and ring copies still in flight land before the CTA ends
                for (int q = 0; q < kTeamBufs; ++q)
                    if ((inflight >> q) & 1u) team_wait_stage(&mbar[q], (phase >> q) & 1u, a.spin_limit_ns);
                cp_async_wait_all();
            }
            return false;
        }
    }
    if (SK) {  // after the last level's barrier: each CTA writes its own slots out
        const int n = __ldg(a.task_off + job.graph + 1) - kbase;
        const int ns = n > rank ? (n - rank + k - 1) >> lk : 0;  // tasks rank, rank + k, ... below n
        for (int q = t; q < ns; q += kTeamBlock) a.key[kbase + rank + (q << lk)] = skey[q];
    }
    if (a.g_end && rank == 0 && t == 0) a.g_end[job.graph] = (int64_t)gtimer();
    return true;
}

// ---------------------------------------------------------------- the kernel

// Phase 1 (cluster launches with cluster jobs): CTA 0 of each cluster takes the next cluster
// job and hands it to every CTA of its cluster through distributed shared memory; the cluster
// runs it as one team. Phase 2: every CTA takes solo jobs until none is left.
// REC: instrument bit 2 runs, which record per-task costs (t_cost); a separate instantiation, so
// that the kernel of ordinary runs carries no recording code.
// CSK: a cluster class whose every graph keeps its keys in distributed shared memory; its kernel
// has the cluster path with shared keys alone (no single-CTA phase), which keeps the payload
// kernel within its register budget.
template <bool PAY, bool REC, bool CSK>
__device__ __forceinline__ void k_team_body(const TeamArgs& a) {
    extern __shared__ __align__(16) unsigned char s_stage[];  // kTeamBufs stage buffers
    __shared__ TeamStage s_view[kTeamBufs];
    __shared__ TeamSrc s_src;
    __shared__ __align__(8) unsigned long long mbar[kTeamBufs];
    __shared__ __align__(16) TeamJob s_job;
    __shared__ int4 s_ring[kRing];
    __shared__ int2 s_iring[kRing];
    __shared__ int s_pcnt[2];  // payload piece counters, alternating by level
    __shared__ int s_fail;     // the team failed (team_fail); read after each level's barrier
    const int t = threadIdx.x;
    if (t == 0) {
        s_fail = 0;
        s_src = TeamSrc{a.ls_node, a.ls_ptr, a.ls_in, a.pdesc, a.stage_n, a.stage_e, a.stage_p, 0};
        for (int b = 0; b < kTeamBufs; ++b) {
            mbar_init(&mbar[b], 1);
            s_view[b] = team_stage_view(s_stage, b, a.stage_n, a.stage_e, a.stage_p);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // the key table follows the stage buffers (a.key_cap entries; 16-byte aligned offset)
    uint32_t* skey = reinterpret_cast<uint32_t*>(s_stage + kTeamBufs * team_stage_bytes(a.stage_n, a.stage_e, a.stage_p));
    unsigned phase = 0;  // bit b: parity of buffer b's next completion
    const int k = (int)cluster_size();
    if (k > 1 && a.ncjobs > 0) {
        const int rank = (int)cluster_rank();
        cluster_sync();  // every CTA of the cluster has started before any DSMEM store
        for (;;) {
            if (rank == 0 && t == 0) {  // no new job once the run is aborting
                const int j = ld_relaxed(&a.ctrl->abort) ? a.ncjobs : atomicAdd(a.team + kTeamNextC, 1);
                const TeamJob job = j < a.ncjobs ? a.jobs[j] : TeamJob{-1, 0, 0, 0};
                for (int r = 0; r < k; ++r) st_cluster_job(&s_job, (unsigned)r, job);
            }
            cluster_sync();
            const TeamJob job = s_job;
            cluster_sync();  // all have read s_job before CTA 0 may overwrite it
            if (job.graph < 0) break;
            bool ok;
            if constexpr (CSK)
                ok = team_run_graph<PAY, false, REC, true>(a, job, k, rank, s_src, s_view, mbar, s_ring, s_iring,
                                                           s_pcnt, &s_fail, phase, skey);
            else
                ok = !PAY && (job.flags & kJobSharedKeys) ? team_run_graph<PAY, false, REC, !PAY>(a, job, k, rank, s_src, s_view, mbar,
                                                                               s_ring, s_iring, s_pcnt, &s_fail, phase,
                                                                               skey)
                                       : team_run_graph<PAY, false, REC, false>(a, job, k, rank, s_src, s_view, mbar,
                                                                                s_ring, s_iring, s_pcnt, &s_fail,
                                                                                phase, skey);
            if (!ok) return;
        }
    }
    if constexpr (CSK) return;  // (a cluster class has no single-CTA jobs)
    for (;;) {
        if (t == 0) {
            const int j = ld_relaxed(&a.ctrl->abort) ? a.njobs : a.ncjobs + atomicAdd(a.team + kTeamNext, 1);
            s_job = j < a.njobs ? a.jobs[j] : TeamJob{-1, 0, 0, 0};
        }
        __syncthreads();
        const TeamJob job = s_job;
        __syncthreads();
        if (job.graph < 0) break;
        if (!team_run_graph<PAY, true, REC, false>(a, job, 1, 0, s_src, s_view, mbar, s_ring, s_iring, s_pcnt,
                                                   &s_fail, phase, skey))
            return;
    }
}

// The class launches of a run are chained by programmatic dependent launch (see plan_run): each
// CTA allows the next class to launch as soon as it starts, and waits for the previous class's
// grid to complete only when it is done (a no-op for the first class), so the next class's
// kernel completes after every earlier one.
// Register budgets: the kernel without payloads runs one CTA per SM (the pipelined levels keep
// ~150 registers a thread live; a second CTA on the SM would share its L1 miss rate anyway), the
// payload kernel two (96 registers: piece streaming wants the warps).
template <bool PAY, bool REC, bool CSK = false>
__global__ void __launch_bounds__(kTeamBlock, PAY ? 2 : 1) k_team(const TeamArgs a) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    k_team_body<PAY, REC, CSK>(a);
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace hf
