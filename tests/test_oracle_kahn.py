"""Pins for the Kahn oracle (oracle/kahn.c) against things other than itself.

* brute-force enumeration of every source->task path on tiny DAGs (bit-exact: each path sum
  is a left-to-right chain of FP32 adds and rounding is monotone, so the recursive max equals
  the max over paths exactly);
* an FP64 longest-path recomputation (relative error bounded by depth * 2^-24);
* closed forms: unit delays give the longest hop count (networkx topological generations),
  a chain gives FP32 prefix sums, a complete bipartite layer gives max_j d_j;
* the paper's worked examples: the saxpy graph (Section I, Listing 1: every y ends as 4) and
  the eight-task dependency graph (Section III-A, Figure 2);
* semantics: every task runs exactly once and after all its predecessors; cycles are caught.
"""
import itertools

import networkx as nx
import numpy as np
import pytest

import oracle
from golden_io import load


def _bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


def _tiny_dag(rng, n):
    perm = rng.permutation(n)
    p = rng.uniform(0.2, 0.7)
    src, dst = [], []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                src.append(perm[i])
                dst.append(perm[j])
                if rng.random() < 0.1:  # duplicate edge with another delay
                    src.append(perm[i])
                    dst.append(perm[j])
    m = len(src)
    kind = rng.integers(0, 4)
    if kind == 0:
        d = rng.uniform(0.01, 1.0, m)
    elif kind == 1:
        d = rng.normal(0, 10, m)  # negative delays allowed
    elif kind == 2:
        d = rng.choice([0.0, -0.0, 1e-8, 1.0, 3.0, 1e7, -1e-8], m)
    else:
        d = np.exp(rng.normal(-2, 0.5, m))
    arr0 = rng.choice([0.0, -0.0, 1.5, -2.25, 1e-30], n).astype(np.float32)
    return (np.array(src, np.int32), np.array(dst, np.int32), np.asarray(d, np.float32), arr0)


def _f32_total_max(vals):
    """max under -inf < ... < -0 < +0 < ... (bit order key)."""
    best = None
    for x in vals:
        x = np.float32(x)
        if best is None:
            best = x
            continue
        if x > best or (x == best and np.signbit(best) and not np.signbit(x)):
            best = x
    return best


def _brute_force(n, src, dst, d, arr0):
    """Max over every path from a source to v of the left-to-right FP32 path sum."""
    succ = {u: [] for u in range(n)}
    indeg = np.zeros(n, int)
    for e in range(len(src)):
        succ[int(src[e])].append(e)
        indeg[dst[e]] += 1
    sums = {v: [] for v in range(n)}

    def walk(v, s):
        sums[v].append(s)
        for e in succ[v]:
            walk(int(dst[e]), np.float32(s + d[e]))

    for s in range(n):
        if indeg[s] == 0:
            walk(s, np.float32(arr0[s]))
    return np.array([_f32_total_max(sums[v]) for v in range(n)], np.float32)


def test_bruteforce_paths_bit_exact_1000_tiny_dags():
    rng = np.random.default_rng(12345)
    for seed in range(1000):
        n = int(rng.integers(1, 10))
        src, dst, d, arr0 = _tiny_dag(rng, n)
        arr, order, stamp, cnt = oracle.kahn(n, src, dst, d, arr0)
        assert cnt == n
        ref = _brute_force(n, src, dst, d, arr0)
        np.testing.assert_array_equal(_bits(arr), _bits(ref), err_msg="seed %d" % seed)


def test_negative_zero_is_below_positive_zero():
    # two sources at -0 and +0 feeding one task through zero delays -> +0 wins
    src = np.array([0, 1], np.int32)
    dst = np.array([2, 2], np.int32)
    d = np.array([-0.0, -0.0], np.float32)
    arr0 = np.array([-0.0, 0.0, 0.0], np.float32)
    arr, *_ = oracle.kahn(3, src, dst, d, arr0)
    assert _bits(arr)[2] == 0  # +0.0
    arr, *_ = oracle.kahn(3, src, dst, d, np.array([-0.0, -0.0, 0.0], np.float32))
    assert _bits(arr)[2] == 0x80000000  # -0 + -0 = -0


def _fp64_longest(n, src, dst, d):
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    best = np.full(n, -np.inf)
    preds = {v: [] for v in range(n)}
    for e in range(len(src)):
        G.add_edge(int(src[e]), int(dst[e]))
        preds[int(dst[e])].append(e)
    for v in nx.topological_sort(G):
        if not preds[v]:
            best[v] = 0.0
        for e in preds[v]:
            best[v] = max(best[v], best[int(src[e])] + float(d[e]))
    return best


def test_fp64_longest_path_within_rounding_bound():
    from paper_2203_08395_b300 import synth

    g = synth.layered(3, 3000, 30, 1, 4)
    arr, *_ = oracle.kahn(g.n, g.src, g.dst, g.delay)
    ref = _fp64_longest(g.n, g.src, g.dst, g.delay)
    depth = 30
    rel = np.abs(arr.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-30)
    assert np.all(rel <= depth * 2.0 ** -24)
    assert np.count_nonzero(arr.astype(np.float64) != ref) > 0  # FP32 really rounds


def test_unit_delays_give_longest_hop_count():
    from paper_2203_08395_b300 import synth

    for seed in range(3):
        g = synth.random_dag(seed, 2000, 1, 6)
        n, _, src, dst, _ = g
        arr, *_ = oracle.kahn(n, src, dst, np.ones(src.size, np.float32))
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(src.tolist(), dst.tolist()))
        lev = np.zeros(n)
        for k, gen in enumerate(nx.topological_generations(G)):
            lev[list(gen)] = k
        np.testing.assert_array_equal(arr, lev.astype(np.float32))


def test_chain_is_fp32_prefix_sum():
    rng = np.random.default_rng(7)
    n = 1000
    d = rng.uniform(0.01, 1.0, n - 1).astype(np.float32)
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    arr, *_ = oracle.kahn(n, src, dst, d)
    ref = np.concatenate([[np.float32(0)], np.cumsum(d, dtype=np.float32)])
    np.testing.assert_array_equal(_bits(arr), _bits(ref))


def test_complete_bipartite_layer():
    rng = np.random.default_rng(8)
    S, T = 17, 9
    src = np.repeat(np.arange(S), T).astype(np.int32)
    dst = np.tile(np.arange(S, S + T), S).astype(np.int32)
    d = rng.uniform(-5, 5, S * T).astype(np.float32)
    arr, *_ = oracle.kahn(S + T, src, dst, d)
    for j in range(T):
        np.testing.assert_equal(arr[S + j], d[dst == S + j].max())
    assert np.all(arr[:S] == 0)


def test_single_and_empty():
    arr, order, stamp, cnt = oracle.kahn(1, [], [], [])
    assert cnt == 1 and arr[0] == 0 and list(order) == [0]
    arr, order, stamp, cnt = oracle.kahn(0, [], [], [])
    assert cnt == 0


def test_cycle_leaves_tasks_unrun():
    src = np.array([0, 1, 2, 3], np.int32)
    dst = np.array([1, 2, 1, 4], np.int32)
    arr, order, stamp, cnt = oracle.kahn(5, src, dst, np.ones(4, np.float32))
    # 0 and 3 are sources, 4 follows 3; the cycle 1 -> 2 -> 1 never becomes ready
    assert cnt == 3 and sorted(order.tolist()) == [0, 3, 4]
    assert stamp[1] == -1 and stamp[2] == -1


def test_every_task_once_after_all_predecessors():
    from paper_2203_08395_b300 import synth

    for seed in range(5):
        n, _, src, dst, d = synth.random_dag(seed, 5000, 1, 6, window=50)
        arr, order, stamp, cnt = oracle.kahn(n, src, dst, d)
        assert cnt == n
        assert np.array_equal(np.sort(order), np.arange(n))
        assert np.all(stamp[src] < stamp[dst])


def test_self_loop_is_a_cycle():
    arr, order, stamp, cnt = oracle.kahn(2, [0, 1], [1, 1], [1.0, 1.0])
    assert cnt == 1


def test_paper_saxpy_graph_every_y_is_4():
    gold = load("paper_saxpy_graph.txt")
    P = gold["params"]
    N = P["N"]
    names = [t[0] for t in gold["tasks"]]
    ix = {nm: i for i, nm in enumerate(names)}
    # host vectors and device buffers; host tasks are modelled as copies of their fill values
    hx, hy = np.zeros(N, np.int32), np.zeros(N, np.int32)
    fill_x, fill_y = np.full(N, P["x"], np.int32), np.full(N, P["y"], np.int32)
    dx, dy = np.zeros(N, np.int32), np.zeros(N, np.int32)
    n = len(names)
    op = np.zeros(n, np.uint8)
    p0 = np.zeros(n, np.uint64)
    p1 = np.zeros(n, np.uint64)
    ln = np.zeros(n, np.int64)
    a_i = np.zeros(n, np.int32)
    host = {"x": hx, "y": hy}
    dev = {"pull_x": dx, "pull_y": dy}
    for t in gold["tasks"]:
        i = ix[t[0]]
        if t[1] == "host":
            op[i], p0[i], p1[i], ln[i] = oracle.OP_COPY, host[t[2]].ctypes.data, (
                fill_x if t[2] == "x" else fill_y).ctypes.data, 4 * N
        elif t[1] == "pull":
            op[i], p0[i], p1[i], ln[i] = oracle.OP_COPY, dev[t[0]].ctypes.data, host[t[2]].ctypes.data, 4 * N
        elif t[1] == "saxpy_i32":
            op[i], p0[i], p1[i], ln[i], a_i[i] = (oracle.OP_SAXPY_I32, dev[t[3]].ctypes.data,
                                                  dev[t[2]].ctypes.data, N, P["a"])
        elif t[1] == "push":
            op[i], p0[i], p1[i], ln[i] = oracle.OP_COPY, host[t[3]].ctypes.data, dev[t[2]].ctypes.data, 4 * N
    src = np.array([ix[a] for a, b in gold["edges"]], np.int32)
    dst = np.array([ix[b] for a, b in gold["edges"]], np.int32)
    arr, order, stamp, cnt = oracle.kahn(n, src, dst, np.zeros(src.size, np.float32), None, op, p0, p1, ln,
                                         None, a_i)
    assert cnt == n
    assert np.all(hy == P["expect_y"]) and np.all(hx == P["expect_x"])
    assert np.all(stamp[src] < stamp[dst])


def test_paper_dependency_graph_order():
    gold = load("paper_dependency_graph.txt")
    names = [t[0] for t in gold["tasks"]]
    ix = {nm: i for i, nm in enumerate(names)}
    src = np.array([ix[a] for a, b in gold["edges"]], np.int32)
    dst = np.array([ix[b] for a, b in gold["edges"]], np.int32)
    assert len(names) == 8 and src.size == 7
    arr, order, stamp, cnt = oracle.kahn(8, src, dst, np.ones(7, np.float32))
    assert cnt == 8
    assert np.all(stamp[src] < stamp[dst])
    for a, b in gold["reach"]:
        assert stamp[ix[a]] < stamp[ix[b]]
    # with unit delays the arrival is the hop depth: pull1 -> kernel1 -> kernel2 -> push2
    assert arr[ix["push2"]] == 4.0 and arr[ix["kernel2"]] == 3.0


def test_saxpy_f32_closed_forms():
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, 10000).astype(np.float32)
    y = rng.uniform(-1, 1, 10000).astype(np.float32)
    # a = 2: 2x is exact, so fma == one rounding of the exact 2x + y (exact in FP64)
    np.testing.assert_array_equal(oracle.saxpy_f32(2.0, x, y),
                                  (2.0 * x.astype(np.float64) + y.astype(np.float64)).astype(np.float32))
    # a = 1: a plain FP32 add
    np.testing.assert_array_equal(oracle.saxpy_f32(1.0, x, y), x + y)
    # a = 0.5 and a = -4: exact scalings
    np.testing.assert_array_equal(oracle.saxpy_f32(0.5, x, y),
                                  (0.5 * x.astype(np.float64) + y.astype(np.float64)).astype(np.float32))
    np.testing.assert_array_equal(oracle.saxpy_f32(-4.0, x, y),
                                  (-4.0 * x.astype(np.float64) + y.astype(np.float64)).astype(np.float32))


def test_saxpy_i32_wraps_mod_2_32():
    x = np.array([2**31 - 1, -2**31, 123456789, -5], np.int32)
    y = np.array([5, -1, 2**30, 7], np.int32)
    a = 3
    n = 4
    op = np.full(1, oracle.OP_SAXPY_I32, np.uint8)
    yy = y.copy()
    arr, order, stamp, cnt = oracle.kahn(1, [], [], [], None, op, [yy.ctypes.data], [x.ctypes.data], [n],
                                         None, [a])
    ref = [((a * int(xi) + int(yi) + 2**31) % 2**32) - 2**31 for xi, yi in zip(x, y)]
    assert yy.tolist() == ref


def _bl_brute(n, src, dst, c):
    succ = {u: [] for u in range(n)}
    for e in range(len(src)):
        succ[int(src[e])].append(int(dst[e]))
    # paths from v to a sink; sum c along the path from the sink end backwards, as the
    # recursion does: b(v) = c(v) + b(s)
    memo = {}

    def paths(v):
        if not succ[v]:
            return [[v]]
        out = []
        for s in succ[v]:
            for p in paths(s):
                out.append([v] + p)
        return out

    res = np.zeros(n, np.float32)
    for v in range(n):
        sums = []
        for p in paths(v):
            s = np.float32(c[p[-1]])
            for w in reversed(p[:-1]):
                s = np.float32(s + c[w])
            sums.append(s)
        res[v] = _f32_total_max(sums)
    return res


def test_bottom_levels_bruteforce():
    rng = np.random.default_rng(21)
    for seed in range(200):
        n = int(rng.integers(1, 9))
        src, dst, _, _ = _tiny_dag(rng, n)
        c = rng.uniform(0.0, 5.0, n).astype(np.float32)
        b = oracle.bottom_levels(n, src, dst, c)
        np.testing.assert_array_equal(_bits(b), _bits(_bl_brute(n, src, dst, c)))
