/*
 * kahn.c -- CPU oracle for the task-graph executor. TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this file's
 * library. The product path never calls it and shares no code with it.
 *
 * What it computes, plainly and sequentially:
 *
 *   A task graph is a DAG whose nodes are tasks and whose edges are dependency constraints
 *   (Section III-A). A task runs only after every task that precedes it has finished
 *   ("Add a Dependency Link", Section III-A); the graph must be acyclic (same passage).
 *   Execution here is Kahn's algorithm with one FIFO queue on one thread: all tasks with no
 *   predecessor enter the queue in increasing id order; popping a task runs its payload,
 *   stamps its completion and releases its successors in the order their edges were added.
 *
 *   Payloads:
 *     - every task carries an arrival time; a source starts at arr0 (default +0), any other
 *       task at -inf, and finishing task u raises arr[v] to max(arr[v], arr[u] + d(u,v)) for
 *       each successor v (timing-graph max-plus propagation; the paper's timing-analysis
 *       setting, Section IV-A). The addition is one IEEE-754 binary32 add, round to nearest
 *       even; the max uses the total order -inf < ... < -0 < +0 < ... < +inf;
 *     - saxpy kernel tasks compute y[i] = a*x[i] + y[i] (Listing 1's kernel, Section I): the
 *       FP32 form with one fused multiply-add (fmaf), the int32 form with two's-complement
 *       wrap-around;
 *     - pull and push tasks copy bytes host -> device and device -> host (Section III-A,
 *       Pull Task / Push Task); here both ends are host arrays, so a copy is a memmove.
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OP_NONE = 0, OP_SAXPY_F32 = 1, OP_SAXPY_I32 = 2, OP_COPY = 3 };

/* a is below b in the total order used for max (no NaN inputs) */
static int below(float a, float b) {
    if (a < b) return 1;
    if (a > b) return 0;
    /* equal values: only +0 and -0 compare equal while differing; -0 is below +0 */
    return signbit(a) && !signbit(b);
}

/*
 * Runs the graph once. Arrays are indexed by task id (n tasks) or edge id (m edges).
 *   arr0      n source arrivals, or NULL for +0 everywhere
 *   op        n payload codes (OP_*), or NULL for "max-plus only"
 *   p0, p1    per-task pointers: saxpy y (p0) and x (p1); copy destination (p0) and source (p1)
 *   len       per-task element count (saxpy) or byte count (copy)
 *   a_f, a_i  per-task saxpy scalars
 * Outputs (any may be NULL): arr_out[n], order_out[n] (task ids in execution order),
 * stamp_out[n] (position of each task in that order, -1 if it never ran).
 * Returns the number of tasks executed; fewer than n means the graph has a cycle.
 */
int64_t oracle_kahn(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const float* delay,
                    const float* arr0, const uint8_t* op, void* const* p0, void* const* p1,
                    const int64_t* len, const float* a_f, const int32_t* a_i, float* arr_out,
                    int32_t* order_out, int64_t* stamp_out) {
    if (n < 0 || m < 0) return -1;
    int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t* pending = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    float* arr = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!first || !next || !pending || !arr || !fifo) {
        free(first); free(next); free(pending); free(arr); free(fifo);
        return -2;
    }
    for (int32_t v = 0; v < n; ++v) first[v] = -1;
    /* successor lists as singly linked lists; inserting edges from last to first leaves each
     * list in the order the edges were added */
    for (int64_t e = m - 1; e >= 0; --e) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n) {
            free(first); free(next); free(pending); free(arr); free(fifo);
            return -1;
        }
        next[e] = first[u];
        first[u] = e;
        pending[v]++;
    }
    int64_t qhead = 0, qtail = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (pending[v] == 0) {
            arr[v] = arr0 ? arr0[v] : 0.0f;
            fifo[qtail++] = v;
        } else {
            arr[v] = -INFINITY;
        }
        if (stamp_out) stamp_out[v] = -1;
    }
    int64_t done = 0;
    while (qhead < qtail) {
        const int32_t u = fifo[qhead++];
        const int code = op ? op[u] : OP_NONE;
        if (code == OP_SAXPY_F32) {
            float* y = (float*)p0[u];
            const float* x = (const float*)p1[u];
            const float a = a_f[u];
            for (int64_t i = 0; i < len[u]; ++i) y[i] = fmaf(a, x[i], y[i]);
        } else if (code == OP_SAXPY_I32) {
            int32_t* y = (int32_t*)p0[u];
            const int32_t* x = (const int32_t*)p1[u];
            const uint32_t a = (uint32_t)a_i[u];
            for (int64_t i = 0; i < len[u]; ++i)
                y[i] = (int32_t)(a * (uint32_t)x[i] + (uint32_t)y[i]);
        } else if (code == OP_COPY) {
            if (len[u] > 0) memmove(p0[u], p1[u], (size_t)len[u]);
        }
        if (order_out) order_out[done] = u;
        if (stamp_out) stamp_out[u] = done;
        done++;
        for (int64_t e = first[u]; e >= 0; e = next[e]) {
            const int32_t v = dst[e];
            const float cand = arr[u] + delay[e];
            if (below(arr[v], cand)) arr[v] = cand;
            if (--pending[v] == 0) fifo[qtail++] = v;
        }
    }
    if (arr_out) memcpy(arr_out, arr, sizeof(float) * (size_t)n);
    free(first); free(next); free(pending); free(arr); free(fifo);
    return done;
}

/* Element-wise FP32 saxpy on a sample: y[i] = fmaf(a, x[i], y[i]) (Listing 1's kernel). */
void oracle_saxpy_f32(int64_t k, float a, const float* x, float* y) {
    for (int64_t i = 0; i < k; ++i) y[i] = fmaf(a, x[i], y[i]);
}
