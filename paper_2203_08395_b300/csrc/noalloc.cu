// noalloc.cu -- arrival propagation over a caller-built successor list, with no allocation.
//
// hf_run_csr_noalloc is the one entry point of this library that never allocates: its
// scratch (per-task packed state, ready queue, control words) lives in a file-scope device
// array that the CUDA module reserves on every GPU where the library is loaded, and stays
// reserved until the process exits. It serves callers that cannot call cudaMalloc: code
// running inside another framework's memory pool or under a fixed memory budget, plug-ins
// that the host application forbids to allocate, and hot loops where an allocation (and the
// device synchronisation cudaMalloc/cudaFree can imply) is not acceptable. The caller still
// owns and passes every input and output buffer.
//
// The kernel is a compact variant of the persistent ready-queue executor: one 64-bit word
// per task packs {arrival key, predecessors still pending}, a single CAS per edge folds the
// max-plus update and the decrement together, and the last predecessor publishes the
// successor in a FIFO of pre-claimed slots. The result is the same bit pattern as every
// other executor of the library (max of correctly rounded binary32 sums under the total
// order -inf < ... < -0 < +0 < ... < +inf).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "hf.h"
#include "hf_internal.h"

namespace {

constexpr int64_t kNaTasks = HF_NOALLOC_MAX_TASKS;
constexpr int64_t kNaQueueWord = kNaTasks;                  // state words [0, kNaTasks)
constexpr int64_t kNaCtrlWord = kNaTasks + kNaTasks / 2;    // queue: kNaTasks int32 slots
constexpr int64_t kNaWords = kNaCtrlWord + 64;              // control: 128 int32 words
// control words (int32 index): each counter on its own 128-byte line
constexpr int kHead = 0, kTail = 32, kDone = 64, kStatus = 96, kBad = 97;
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;
constexpr uint32_t kNaKeyNegInf = 0x007FFFFFu;  // key of -inf
constexpr unsigned kFullMask = 0xffffffffu;

}  // namespace

// The scratch: HF_NOALLOC_MAX_TASKS x 12 bytes plus 512 bytes of control words (12 MiB + 512 B).
// Host code must not use this name as an address: it takes the device address from
// cudaGetSymbolAddress once per device and passes it to the kernels.
static __device__ __align__(256) unsigned long long hf_noalloc_scratch[kNaWords];

namespace {

struct NaView {
    unsigned long long* state;
    int32_t* queue;
    int32_t* ctrl;
};

__device__ __forceinline__ NaView na_view(void* base) {
    unsigned long long* w = static_cast<unsigned long long*>(base);
    return NaView{w, reinterpret_cast<int32_t*>(w + kNaQueueWord), reinterpret_cast<int32_t*>(w + kNaCtrlWord)};
}

// order-preserving map binary32 -> uint32 (unsigned order of keys = total order of floats)
__device__ __forceinline__ uint32_t na_key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float na_val(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ uint64_t na_now() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int na_ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int na_ld_relaxed(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long na_ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void na_st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every call starts here: the array keeps the previous call's contents, so each state word,
// queue slot and control word this call reads is rewritten first.
__global__ void k_na_clear(void* scratch, int n) {
    const NaView s = na_view(scratch);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        s.state[i] = (unsigned long long)kNaKeyNegInf << 32;  // key -inf, nothing pending yet
        s.queue[i] = -1;                                       // slot not yet published
    }
    if (blockIdx.x == 0 && threadIdx.x < 128) s.ctrl[threadIdx.x] = 0;
}

// Validates the CSR and counts each task's predecessors into the low half of its state word.
__global__ void k_na_count(void* scratch, int n, int m, const int32_t* row_ptr, const int32_t* succ,
                           const float* delay) {
    const NaView s = na_view(scratch);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t hi = n > m ? n : m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) {
        bool bad = false;
        if (i < n) {
            const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
            bad |= r0 < 0 || r1 < r0 || r1 > m;
            if (i == 0) bad |= r0 != 0 || row_ptr[n] != m;
        }
        if (i < m) {
            const int t = succ[i];
            if (t < 0 || t >= n || !isfinite(delay[i])) bad = true;
            else atomicAdd(s.state + t, 1ull);
        }
        if (bad) atomicOr(s.ctrl + kBad, 1);
    }
}

// Sources (no predecessor) take their arrival and enter the ready queue; arr0 of a task with
// predecessors is never read.
__global__ void k_na_seed(void* scratch, int n, const float* arr0) {
    const NaView s = na_view(scratch);
    if (s.ctrl[kBad]) return;
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += wstride) {
        const int64_t i = i0 + lane;
        bool seed = false;
        uint32_t k = 0;
        if (i < n && (uint32_t)s.state[i] == 0u) {  // arr0 is read for sources only
            const float a = arr0 ? arr0[i] : 0.f;
            if (!isfinite(a)) {
                atomicOr(s.ctrl + kBad, 1);
            } else {
                seed = true;
                k = na_key(a);
            }
        }
        const unsigned b = __ballot_sync(kFullMask, seed);
        int base = 0;
        if (lane == 0 && b) base = atomicAdd(s.ctrl + kTail, __popc(b));
        base = __shfl_sync(kFullMask, base, 0);
        if (seed) {
            s.state[i] = (unsigned long long)k << 32;
            s.queue[base + __popc(b & ((1u << lane) - 1u))] = (int)i;
        }
    }
}

// The executor proper. A warp claims queue slots (one per lane, up to its share of the
// backlog), waits for each slot to be published, and runs the tasks it finds: writes the
// task's final arrival and releases every successor with one CAS on the successor's packed
// word (max of keys, pending - 1). The CAS that takes pending to zero publishes the successor.
// Waits are bounded: without any new publication for spin_limit_ns the call ends with
// HF_ETIMEDOUT (the edges hold a cycle, or a task never became ready); a warp measures the time
// since it last saw the queue tail or the completion count move.
__global__ void __launch_bounds__(kNaThreads) k_na_run(void* scratch, int n, const int32_t* row_ptr,
                                                        const int32_t* succ, const float* delay, float* arr,
                                                        uint64_t spin_limit_ns) {
    const NaView s = na_view(scratch);
    if (s.ctrl[kBad]) return;
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * (kNaThreads / 32);
    int slot = -1;
    int last_tail = -1, last_done = -1;  // progress seen by lane 0: publications or completions
    uint64_t t_last = na_now();
    for (;;) {
        if (__ballot_sync(kFullMask, slot >= 0) == 0) {  // claim new slots
            int base = n, c = 0;
            if (lane == 0) {
                const int h = na_ld_relaxed(s.ctrl + kHead);
                if (h < n) {
                    const int backlog = na_ld_relaxed(s.ctrl + kTail) - h;
                    c = min(max(backlog / nwarps, 1), 32);
                    base = atomicAdd(s.ctrl + kHead, c);
                }
            }
            base = __shfl_sync(kFullMask, base, 0);
            c = __shfl_sync(kFullMask, c, 0);
            if (base >= n) break;  // every slot is claimed: the work left belongs to other warps
            if (lane < c && base + lane < n) slot = base + lane;
        }
        const int v = slot >= 0 ? na_ld_acquire(s.queue + slot) : -1;
        const unsigned got = __ballot_sync(kFullMask, v >= 0);
        if (got == 0) {
            int stop = 0;
            if (lane == 0) {
                const int t = na_ld_relaxed(s.ctrl + kTail), dn = na_ld_relaxed(s.ctrl + kDone);
                const uint64_t now = na_now();
                if (t != last_tail || dn != last_done) {
                    last_tail = t;
                    last_done = dn;
                    t_last = now;
                }
                if (na_ld_relaxed(s.ctrl + kStatus) != 0) stop = 1;
                else if (now - t_last > spin_limit_ns) {
                    atomicCAS(s.ctrl + kStatus, 0, (int)HF_ETIMEDOUT);
                    stop = 1;
                }
            }
            if (__shfl_sync(kFullMask, stop, 0)) break;
            __nanosleep(100);
            continue;
        }
        if (v >= 0) {
            slot = -1;
            // the release store that published v follows the CAS that made its word final
            const float av = na_val((uint32_t)(na_ld_relaxed64(s.state + v) >> 32));
            arr[v] = av;
            const int e1 = row_ptr[v + 1];
            for (int e = row_ptr[v]; e < e1; ++e) {
                const int t = succ[e];
                const uint32_t kc = na_key(__fadd_rn(av, delay[e]));
                unsigned long long old = na_ld_relaxed64(s.state + t), assumed;
                do {
                    assumed = old;
                    const uint32_t k = max((uint32_t)(assumed >> 32), kc);
                    const unsigned long long nw = ((unsigned long long)k << 32) | (uint32_t)((uint32_t)assumed - 1u);
                    old = atomicCAS(s.state + t, assumed, nw);
                } while (old != assumed);
                if ((uint32_t)assumed == 1u) na_st_release(s.queue + atomicAdd(s.ctrl + kTail, 1), t);
            }
        }
        if (lane == 0) atomicAdd(s.ctrl + kDone, __popc(got));
    }
}

struct NaDevice {
    bool ready = false;
    void* scratch = nullptr;  // device address of hf_noalloc_scratch on this device
    int grid_run = 0;
    int grid_fill = 0;
};

std::mutex g_na_mu;
NaDevice g_na_dev[kNaMaxDevices];

// Once per device, with that device current: look up the array's device address and size the
// grids. Runs inside the first call on each device.
hf_status na_setup(int dev, NaDevice* out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaDevice& d = g_na_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, hf_noalloc_scratch);
        if (e != cudaSuccess) return hf::cuda_fail(e, "cudaGetSymbolAddress(hf_noalloc_scratch)");
        int sms = 0, occ = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return hf::cuda_fail(e, "cudaDeviceGetAttribute");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_na_run, kNaThreads, 0);
        if (e != cudaSuccess) return hf::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        d.scratch = ptr;
        d.grid_run = sms * std::min(std::max(occ, 1), 2);
        d.grid_fill = sms * 4;
        d.ready = true;
    }
    *out = d;
    return HF_OK;
}

}  // namespace

using hf::cuda_fail;
using hf::fail;

extern "C" hf_status hf_run_csr_noalloc(int32_t n_tasks, int32_t n_edges, const int32_t* row_ptr,
                                        const int32_t* succ, const float* delay, const float* arr0, float* arr,
                                        uint64_t spin_limit_ns, void* stream) {
    if (n_tasks < 0 || n_edges < 0) return fail(HF_EINVAL, "n_tasks and n_edges must be >= 0");
    if (n_tasks > HF_NOALLOC_MAX_TASKS)
        return fail(HF_EINVAL, "n_tasks = " + std::to_string(n_tasks) + " exceeds the static scratch limit of " +
                                   std::to_string((long long)HF_NOALLOC_MAX_TASKS) + " tasks");
    if (n_tasks == 0) return n_edges == 0 ? HF_OK : fail(HF_EINVAL, "edges without tasks");
    if (!row_ptr || !arr) return fail(HF_EINVAL, "row_ptr and arr must not be NULL");
    if (n_edges > 0 && (!succ || !delay)) return fail(HF_EINVAL, "succ and delay must not be NULL when n_edges > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return fail(HF_ENOTSUP, "device ordinal beyond 63");
    NaDevice d;
    hf_status st = na_setup(dev, &d);
    if (st != HF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int fill_blocks = (int)std::min<int64_t>(d.grid_fill, ((int64_t)std::max(n_tasks, n_edges) + kNaThreads - 1) / kNaThreads);
    k_na_clear<<<fill_blocks, kNaThreads, 0, s>>>(d.scratch, n_tasks);
    k_na_count<<<fill_blocks, kNaThreads, 0, s>>>(d.scratch, n_tasks, n_edges, row_ptr, succ, delay);
    k_na_seed<<<fill_blocks, kNaThreads, 0, s>>>(d.scratch, n_tasks, arr0);
    k_na_run<<<d.grid_run, kNaThreads, 0, s>>>(d.scratch, n_tasks, row_ptr, succ, delay, arr,
                                               spin_limit_ns ? spin_limit_ns : 2000000000ull);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "hf_run_csr_noalloc launch");
    int32_t h[4] = {0, 0, 0, 0};  // done (unused slot), status, bad
    const char* ctrl = static_cast<const char*>(d.scratch) + kNaCtrlWord * 8;
    if ((e = cudaMemcpyAsync(&h[0], ctrl + 4 * kDone, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h[2], ctrl + 4 * kStatus, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "hf_run_csr_noalloc status copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "hf_run_csr_noalloc sync");
    if (h[3]) return fail(HF_EINVAL, "bad input: row_ptr not a CSR of n_edges edges, successor out of range, "
                                     "or a non-finite delay or arr0");
    if (h[2] == HF_ETIMEDOUT)
        return fail(HF_ETIMEDOUT, "no task became ready for spin_limit_ns (the edges form a cycle?)");
    if (h[0] != n_tasks)
        return fail(HF_EQUEUE, "ran " + std::to_string(h[0]) + " of " + std::to_string(n_tasks) + " tasks");
    return HF_OK;
}
