// costmodel.cu -- the learned cost model: an MLP 12 -> 64 -> 64 -> 1 with ReLU, BF16 weights
// and activations, FP32 accumulation, FP32 master weights and Adam (Kingma & Ba, ICLR 2015,
// Algorithm 1). It predicts a task's log cost (log ns) from 12 per-task features; the
// executor turns predictions into critical-path priorities and an executor choice (plan.cu).
//
// Kernels: forward on the tensor cores (warp-level BF16 MMAs with FP32 accumulation, 16 rows per
// warp tile), a fused forward+backward that reduces the batch's weight gradients in shared
// memory (one block of 64 rows, one thread per row on CUDA cores) before one atomicAdd per
// parameter and block, and an element-wise Adam step. On the hot path the executor only reads
// the resulting priorities and plans.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hf_internal.h"

struct hf_costmodel {
    float* d_params = nullptr;  // HF_COSTMODEL_PARAMS master weights
    float* d_m = nullptr;       // Adam first moments
    float* d_v = nullptr;       // Adam second moments
    float* d_grad = nullptr;    // training scratch
    float* d_loss = nullptr;
    int32_t* d_idx = nullptr;   // training row order
    size_t cap_idx = 0;
    int64_t step = 0;
};

namespace hf {

constexpr int kIn = 12, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = 768, kOffW2 = 832, kOffB2 = 4928, kOffW3 = 4992, kOffB3 = 5056;
constexpr int kNP = HF_COSTMODEL_PARAMS;
static_assert(kOffB3 + 1 == kNP, "parameter layout");
constexpr int kRows = 64;  // rows per block in the gradient kernel

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ bool is_weight(int i) {
    return i < kOffB1 || (i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3);
}

// parameters into shared memory, weights rounded to BF16 (the model's storage precision)
__device__ __forceinline__ void stage_params(float* s, const float* __restrict__ P) {
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) {
        const float v = P[i];
        s[i] = is_weight(i) ? bf16r(v) : v;
    }
}

// forward pass of one row; h1/h2 returned (BF16-rounded values), y returned
__device__ __forceinline__ float row_forward(const float* s, const float* x, float* h1, float* h2) {
#pragma unroll 4
    for (int o = 0; o < kH; ++o) {
        float z = s[kOffB1 + o];
#pragma unroll
        for (int k = 0; k < kIn; ++k) z = fmaf(s[kOffW1 + o * kIn + k], x[k], z);
        h1[o] = bf16r(fmaxf(z, 0.f));
    }
    float y = s[kOffB3];
    for (int o = 0; o < kH; ++o) {
        float z = s[kOffB2 + o];
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(s[kOffW2 + o * kH + k], h1[k], z);
        h2[o] = bf16r(fmaxf(z, 0.f));
        y = fmaf(s[kOffW3 + o], h2[o], y);
    }
    return y;
}

// ---- forward pass on the tensor cores (inference over every task of a plan)
//
// Each warp runs 16-row tiles through warp-level BF16 MMAs with FP32 accumulation
// (mma.sync m16n8k16): layer 1 is one 16x16 A tile (the 12 features, zero-padded to 16) times
// eight 16x8 B tiles of W1^T, layer 2 four 16x16 A tiles times eight B tiles of W2^T per k-step;
// the FP32 accumulators of layer 1, after bias, ReLU and BF16 rounding, are exactly the A
// fragments of layer 2 (the accumulator of n-tiles 2k and 2k + 1 is A's k-tile k), so the
// activations never leave registers; layer 3 (64 -> 1) is a dot product reduced over the four
// threads that hold a row. Same rounding points as row_forward (BF16 inputs, weights and hidden
// activations; FP32 accumulation in a different order).
constexpr int kW1Ld = 24;  // bf16 row pitch of W1 (16 used): conflict-free fragment loads
constexpr int kW2Ld = 72;  // bf16 row pitch of W2 (64 used)

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                                                     int64_t n, float* __restrict__ y) {
    __shared__ __align__(16) __nv_bfloat16 w1[kH * kW1Ld];
    __shared__ __align__(16) __nv_bfloat16 w2[kH * kW2Ld];
    __shared__ float b1[kH], b2[kH], w3[kH];
    __shared__ float b3;
    for (int i = threadIdx.x; i < kH * kW1Ld; i += blockDim.x) {
        const int o = i / kW1Ld, k = i % kW1Ld;
        w1[i] = __float2bfloat16_rn(k < kIn ? P[kOffW1 + o * kIn + k] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kW2Ld; i += blockDim.x) {
        const int o = i / kW2Ld, k = i % kW2Ld;
        w2[i] = __float2bfloat16_rn(k < kH ? P[kOffW2 + o * kH + k] : 0.f);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        b1[i] = P[kOffB1 + i];
        b2[i] = P[kOffB2 + i];
        w3[i] = bf16r(P[kOffW3 + i]);
    }
    if (threadIdx.x == 0) b3 = P[kOffB3];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int64_t tiles = (n + 15) / 16;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < tiles; tile += nwarps) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        // layer 1: A = features of rows r0 / r1, columns 2tq, 2tq+1 (and +8 when below 12)
        uint32_t a[4];
        {
            float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f, x4 = 0.f, x5 = 0.f, x6 = 0.f, x7 = 0.f;
            if (r0 < n) {
                x0 = X[r0 * kIn + 2 * tq];
                x1 = X[r0 * kIn + 2 * tq + 1];
                if (tq < 2) {
                    x4 = X[r0 * kIn + 2 * tq + 8];
                    x5 = X[r0 * kIn + 2 * tq + 9];
                }
            }
            if (r1 < n) {
                x2 = X[r1 * kIn + 2 * tq];
                x3 = X[r1 * kIn + 2 * tq + 1];
                if (tq < 2) {
                    x6 = X[r1 * kIn + 2 * tq + 8];
                    x7 = X[r1 * kIn + 2 * tq + 9];
                }
            }
            a[0] = pack_bf16x2(x0, x1);
            a[1] = pack_bf16x2(x2, x3);
            a[2] = pack_bf16x2(x4, x5);
            a[3] = pack_bf16x2(x6, x7);
        }
        uint32_t h[4][4];  // layer-2 A fragments: k-tile kk from layer-1 n-tiles 2kk, 2kk+1
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * tq;
            float d[4] = {b1[c], b1[c + 1], b1[c], b1[c + 1]};
            const __nv_bfloat16* wr = w1 + (8 * j + g) * kW1Ld + 2 * tq;
            mma_bf16_16816(d, a, *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
            const uint32_t lo = pack_bf16x2(fmaxf(d[0], 0.f), fmaxf(d[1], 0.f));  // row g
            const uint32_t hi = pack_bf16x2(fmaxf(d[2], 0.f), fmaxf(d[3], 0.f));  // row g + 8
            h[j >> 1][(j & 1) * 2 + 0] = lo;
            h[j >> 1][(j & 1) * 2 + 1] = hi;
        }
        // layer 2 and the 64 -> 1 dot product
        float s0 = 0.f, s1 = 0.f;  // rows g, g + 8: this thread's columns
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * tq;
            float d[4] = {b2[c], b2[c + 1], b2[c], b2[c + 1]};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const __nv_bfloat16* wr = w2 + (8 * j + g) * kW2Ld + 16 * kk + 2 * tq;
                mma_bf16_16816(d, h[kk], *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
            }
            s0 = fmaf(w3[c], bf16r(fmaxf(d[0], 0.f)), s0);
            s0 = fmaf(w3[c + 1], bf16r(fmaxf(d[1], 0.f)), s0);
            s1 = fmaf(w3[c], bf16r(fmaxf(d[2], 0.f)), s1);
            s1 = fmaf(w3[c + 1], bf16r(fmaxf(d[3], 0.f)), s1);
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (tq == 0) {
            if (r0 < n) y[r0] = b3 + s0;
            if (r1 < n) y[r1] = b3 + s1;
        }
    }
}

// Fused forward + backward of mean((y - t)^2) over `total` rows; this block takes rows
// [blockIdx.x * 64, +64) of the (optionally index-gathered) row set. Gradients go to grad[P]
// (accumulated with atomicAdd), the loss to *loss.
__global__ void __launch_bounds__(kRows) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                    const float* __restrict__ T, const int32_t* __restrict__ idx,
                                                    int64_t n, float inv_total, float* __restrict__ grad,
                                                    float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* s = sm;                              // kNP
    float* XS = s + kNP + 3;                    // [kRows][kIn]
    float* H1 = XS + kRows * kIn;               // [kRows][kH]
    float* H2 = H1 + kRows * kH;
    float* DZ2 = H2 + kRows * kH;
    float* DZ1 = DZ2 + kRows * kH;
    float* DY = DZ1 + kRows * kH;               // [kRows]
    stage_params(s, P);
    __syncthreads();
    const int t = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * kRows + t;
    float x[kIn], h1[kH], h2[kH];
    float dy = 0.f, l = 0.f;
    if (r < n) {
        const int64_t i = idx ? (int64_t)idx[r] : r;
#pragma unroll
        for (int k = 0; k < kIn; ++k) x[k] = bf16r(X[i * kIn + k]);
        const float yv = row_forward(s, x, h1, h2);
        const float d = yv - T[i];
        dy = 2.f * d * inv_total;
        l = d * d * inv_total;
    } else {
#pragma unroll
        for (int k = 0; k < kIn; ++k) x[k] = 0.f;
#pragma unroll
        for (int k = 0; k < kH; ++k) h1[k] = h2[k] = 0.f;
    }
    float dz2[kH];
#pragma unroll
    for (int o = 0; o < kH; ++o) dz2[o] = h2[o] > 0.f ? dy * s[kOffW3 + o] : 0.f;
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int o = 0; o < kH; ++o) a = fmaf(s[kOffW2 + o * kH + k], dz2[o], a);
        DZ1[t * kH + k] = h1[k] > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) XS[t * kIn + k] = x[k];
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        H1[t * kH + k] = h1[k];
        H2[t * kH + k] = h2[k];
        DZ2[t * kH + k] = dz2[k];
    }
    DY[t] = dy;
    // loss: warp sums, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((t & 31) == 0 && l != 0.f) atomicAdd(loss, l);
    __syncthreads();
    // block reductions over the 64 rows; thread t owns output unit t of each layer
    {
        float gb2 = 0.f, gw3 = 0.f, gb1 = 0.f;
        for (int q = 0; q < kRows; ++q) {
            gb2 += DZ2[q * kH + t];
            gw3 = fmaf(DY[q], H2[q * kH + t], gw3);
            gb1 += DZ1[q * kH + t];
        }
        atomicAdd(grad + kOffB2 + t, gb2);
        atomicAdd(grad + kOffW3 + t, gw3);
        atomicAdd(grad + kOffB1 + t, gb1);
        if (t == 0) {
            float gb3 = 0.f;
            for (int q = 0; q < kRows; ++q) gb3 += DY[q];
            atomicAdd(grad + kOffB3, gb3);
        }
        for (int k0 = 0; k0 < kH; k0 += 16) {
            float a[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = 0.f;
            for (int q = 0; q < kRows; ++q) {
                const float d = DZ2[q * kH + t];
#pragma unroll
                for (int j = 0; j < 16; ++j) a[j] = fmaf(d, H1[q * kH + k0 + j], a[j]);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) atomicAdd(grad + kOffW2 + t * kH + k0 + j, a[j]);
        }
        float a1[kIn];
#pragma unroll
        for (int j = 0; j < kIn; ++j) a1[j] = 0.f;
        for (int q = 0; q < kRows; ++q) {
            const float d = DZ1[q * kH + t];
#pragma unroll
            for (int j = 0; j < kIn; ++j) a1[j] = fmaf(d, XS[q * kIn + j], a1[j]);
        }
#pragma unroll
        for (int j = 0; j < kIn; ++j) atomicAdd(grad + kOffW1 + t * kIn + j, a1[j]);
    }
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                       const float* __restrict__ G, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float g = G[i];
    const float m = 0.9f * M[i] + 0.1f * g;
    const float v = 0.999f * V[i] + 0.001f * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

static size_t grad_smem() { return sizeof(float) * (kNP + 3 + kRows * kIn + 4 * kRows * kH + kRows); }

hf_status mlp_forward(const float* params, const float* X, int64_t n, float* y, cudaStream_t s) {
    if (n <= 0) return HF_OK;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    // 4 warps per block, one 16-row tile per warp at a time; at most 8 blocks per SM
    const int64_t tiles = (n + 15) / 16;
    const int64_t blocks = std::min<int64_t>((tiles + 3) / 4, (int64_t)sms * 8);
    k_mlp_forward<<<(unsigned)blocks, 128, 0, s>>>(params, X, n, y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "k_mlp_forward");
}

static hf_status mlp_grad(const float* params, const float* X, const float* T, const int32_t* idx, int64_t n,
                          float* grad, float* loss, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        attr = true;
    }
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kNP, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (n <= 0) return HF_OK;
    const int64_t blocks = (n + kRows - 1) / kRows;
    k_mlp_grad<<<(unsigned)blocks, kRows, grad_smem(), s>>>(params, X, T, idx, n, 1.0f / (float)n, grad, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "k_mlp_grad");
}

static hf_status adam(hf_costmodel* cm, const float* grad, float lr, cudaStream_t s) {
    cm->step++;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)cm->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)cm->step));
    k_adam<<<(kNP + 255) / 256, 256, 0, s>>>(cm->d_params, cm->d_m, cm->d_v, grad, lr, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "k_adam");
}

const float* costmodel_params(const hf_costmodel* cm) { return cm->d_params; }

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014) for weight initialisation and shuffles
static uint64_t mix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unit(uint64_t& x) { return (double)(mix64(x) >> 11) * 0x1.0p-53; }

}  // namespace hf

using namespace hf;

extern "C" {

hf_status hf_costmodel_create(hf_costmodel** out, uint64_t seed) {
    if (!out) return fail(HF_EINVAL, "out is NULL");
    *out = nullptr;
    hf_costmodel* cm = new (std::nothrow) hf_costmodel();
    if (!cm) return fail(HF_ENOMEM, "host allocation failed");
    cm->d_params = (float*)dev_alloc(sizeof(float) * kNP, nullptr);
    cm->d_m = (float*)dev_alloc(sizeof(float) * kNP, nullptr);
    cm->d_v = (float*)dev_alloc(sizeof(float) * kNP, nullptr);
    cm->d_grad = (float*)dev_alloc(sizeof(float) * kNP, nullptr);
    cm->d_loss = (float*)dev_alloc(sizeof(float) * 4, nullptr);
    if (!cm->d_params || !cm->d_m || !cm->d_v || !cm->d_grad || !cm->d_loss) {
        hf_costmodel_destroy(cm);
        return fail(HF_ENOMEM, "device allocation failed: cost model");
    }
    std::vector<float> p(kNP, 0.f);
    uint64_t st = seed ^ 0xC057C057C057ull;
    const double l1 = std::sqrt(6.0 / kIn), l2 = std::sqrt(6.0 / kH);
    for (int i = 0; i < kNP; ++i) {
        if (i < kOffB1) p[i] = (float)((2.0 * unit(st) - 1.0) * l1);
        else if ((i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3)) p[i] = (float)((2.0 * unit(st) - 1.0) * l2);
    }
    hf_status s = hf_costmodel_set_params(cm, p.data());
    if (s != HF_OK) {
        hf_costmodel_destroy(cm);
        return s;
    }
    *out = cm;
    return HF_OK;
}

hf_status hf_costmodel_destroy(hf_costmodel* cm) {
    if (!cm) return HF_OK;
    cudaDeviceSynchronize();
    dev_free(cm->d_params, nullptr);
    dev_free(cm->d_m, nullptr);
    dev_free(cm->d_v, nullptr);
    dev_free(cm->d_grad, nullptr);
    dev_free(cm->d_loss, nullptr);
    dev_free(cm->d_idx, nullptr);
    delete cm;
    return HF_OK;
}

hf_status hf_costmodel_set_params(hf_costmodel* cm, const float* params) {
    if (!cm || !params) return fail(HF_EINVAL, "NULL argument");
    for (int i = 0; i < kNP; ++i)
        if (!std::isfinite(params[i])) return fail(HF_EINVAL, "parameter " + std::to_string(i) + " not finite");
    cudaError_t e = cudaMemcpy(cm->d_params, params, sizeof(float) * kNP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(cm->d_m, 0, sizeof(float) * kNP);
    if (e == cudaSuccess) e = cudaMemset(cm->d_v, 0, sizeof(float) * kNP);
    if (e != cudaSuccess) return cuda_fail(e, "cost model upload");
    cm->step = 0;
    return HF_OK;
}

hf_status hf_costmodel_get_params(hf_costmodel* cm, float* params) {
    if (!cm || !params) return fail(HF_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(params, cm->d_params, sizeof(float) * kNP, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HF_OK : cuda_fail(e, "cost model download");
}

hf_status hf_costmodel_save(hf_costmodel* cm, const char* path) {
    if (!cm || !path) return fail(HF_EINVAL, "NULL argument");
    std::vector<float> p(kNP);
    hf_status s = hf_costmodel_get_params(cm, p.data());
    if (s != HF_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(HF_EINVAL, std::string("cannot open ") + path);
    const size_t w = std::fwrite(p.data(), sizeof(float), kNP, f);
    std::fclose(f);
    return w == (size_t)kNP ? HF_OK : fail(HF_EINVAL, "short write");
}

hf_status hf_costmodel_load(hf_costmodel* cm, const char* path) {
    if (!cm || !path) return fail(HF_EINVAL, "NULL argument");
    std::vector<float> p(kNP);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(HF_EINVAL, std::string("cannot open ") + path);
    const size_t r = std::fread(p.data(), sizeof(float), kNP, f);
    std::fclose(f);
    if (r != (size_t)kNP) return fail(HF_EINVAL, "cost model file has the wrong size");
    return hf_costmodel_set_params(cm, p.data());
}

hf_status hf_costmodel_forward(hf_costmodel* cm, const float* X, int64_t n, float* y, void* stream) {
    if (!cm || n < 0 || (n > 0 && (!X || !y))) return fail(HF_EINVAL, "bad argument");
    return mlp_forward(cm->d_params, X, n, y, (cudaStream_t)stream);
}

hf_status hf_costmodel_grad(hf_costmodel* cm, const float* X, const float* t, int64_t n, float* grad, float* loss,
                            void* stream) {
    if (!cm || n < 0 || !grad || !loss || (n > 0 && (!X || !t))) return fail(HF_EINVAL, "bad argument");
    return mlp_grad(cm->d_params, X, t, nullptr, n, grad, loss, (cudaStream_t)stream);
}

hf_status hf_costmodel_adam_step(hf_costmodel* cm, const float* grad, float lr, void* stream) {
    if (!cm || !grad || !(lr > 0.f)) return fail(HF_EINVAL, "bad argument");
    return adam(cm, grad, lr, (cudaStream_t)stream);
}

hf_status hf_costmodel_train(hf_costmodel* cm, const float* X, const float* t, int64_t n, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float* final_loss, void* stream) {
    if (!cm || n <= 0 || !X || !t || epochs < 0 || batch <= 0 || !(lr > 0.f))
        return fail(HF_EINVAL, "bad argument");
    if (n > INT32_MAX) return fail(HF_EINVAL, "too many rows");
    cudaStream_t s = (cudaStream_t)stream;
    if (cm->cap_idx < (size_t)n) {
        dev_free(cm->d_idx, s);
        cm->d_idx = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)n, s);
        cm->cap_idx = cm->d_idx ? (size_t)n : 0;
        if (!cm->d_idx) return fail(HF_ENOMEM, "device allocation failed: row order");
    }
    std::vector<int32_t> order((size_t)n);
    uint64_t st = seed;
    hf_status rs;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates
            const int64_t j = (int64_t)(unit(st) * (double)(i + 1));
            std::swap(order[(size_t)i], order[(size_t)(j > i ? i : j)]);
        }
        cudaError_t e = cudaMemcpyAsync(cm->d_idx, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `order` is rewritten next epoch
        if (e != cudaSuccess) return cuda_fail(e, "row order upload");
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            if ((rs = mlp_grad(cm->d_params, X, t, cm->d_idx + b0, nb, cm->d_grad, cm->d_loss, s)) != HF_OK) return rs;
            if ((rs = adam(cm, cm->d_grad, lr, s)) != HF_OK) return rs;
        }
    }
    if (final_loss) {
        if ((rs = mlp_grad(cm->d_params, X, t, nullptr, n, cm->d_grad, cm->d_loss, s)) != HF_OK) return rs;
        cudaError_t e = cudaMemcpyAsync(final_loss, cm->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "loss copy");
    }
    return HF_OK;
}

}  // extern "C"
