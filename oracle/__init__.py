"""CPU oracle for the task-graph executor. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package. It shares no code with the CUDA path (``paper_2203_08395_b300``) and never
imports it; the two meet only in the seeded input generators (``paper_2203_08395_b300.synth``),
which hold none of the method's arithmetic.

Contents
  kahn.c       sequential Kahn executor (arrivals, saxpy, copies, execution order)
  __init__.py  ctypes loader for kahn.c and the task-graph driver below
  mlp.py       FP64 cost-model MLP (forward, backward, Adam) and per-task features

Every function is pinned by ``tests/test_oracle_*.py`` against something other than itself
(brute-force path enumeration, closed forms, the paper's worked examples, library routines,
finite differences). Parity pins and the one unpinned reading are listed in each docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OP_NONE, OP_SAXPY_F32, OP_SAXPY_I32, OP_COPY = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile kahn.c (no fast-math, no FP contraction) into liboracle.so."""
    src = os.path.join(_HERE, "kahn.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp = ctypes.c_void_p
        L.oracle_kahn.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                  vp, vp, vp]
        L.oracle_kahn.restype = ctypes.c_int64
        L.oracle_saxpy_f32.argtypes = [ctypes.c_int64, ctypes.c_float, vp, vp]
        L.oracle_saxpy_f32.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def kahn(n, src, dst, delay, arr0=None, op=None, p0=None, p1=None, length=None, a_f=None, a_i=None):
    """Run the sequential Kahn oracle. Returns (arrivals f32[n], order i32[count], stamp i64[n],
    count). count < n means a cycle. Pointers in p0/p1 must stay alive during the call."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    delay = np.ascontiguousarray(delay, np.float32)
    assert src.size == dst.size == delay.size
    if arr0 is not None:
        arr0 = np.ascontiguousarray(arr0, np.float32)
        assert arr0.size == n
    if op is not None:
        op = np.ascontiguousarray(op, np.uint8)
        p0 = np.ascontiguousarray(p0, np.uint64)
        p1 = np.ascontiguousarray(p1, np.uint64)
        length = np.ascontiguousarray(length, np.int64)
        a_f = np.ascontiguousarray(a_f if a_f is not None else np.zeros(n), np.float32)
        a_i = np.ascontiguousarray(a_i if a_i is not None else np.zeros(n), np.int32)
    arr = np.empty(n, np.float32)
    order = np.empty(n, np.int32)
    stamp = np.empty(n, np.int64)
    cnt = lib().oracle_kahn(n, src.size, _ptr(src), _ptr(dst), _ptr(delay), _ptr(arr0), _ptr(op), _ptr(p0),
                            _ptr(p1), _ptr(length), _ptr(a_f), _ptr(a_i), _ptr(arr), _ptr(order), _ptr(stamp))
    if cnt < 0:
        raise ValueError("oracle_kahn: bad input (rc=%d)" % cnt)
    return arr, order[:cnt], stamp, int(cnt)


def saxpy_f32(a, x, y):
    """y <- fmaf(a, x, y) element-wise (returns a new array)."""
    x = np.ascontiguousarray(x, np.float32)
    y = np.array(y, np.float32, copy=True)
    lib().oracle_saxpy_f32(x.size, float(a), x.ctypes.data, y.ctypes.data)
    return y


def run_spec(g, with_data=True):
    """Execute a workload graph description (``synth.GraphSpec``) on the oracle.

    Builds host stand-ins for every buffer: each saxpy task's x (its pull's device buffer when
    it has a pull task, else its initial device data) and y; each pull's host source; each
    push's host destination. Returns a dict with ``arr`` (f32[n]), ``order``, ``stamp``,
    ``count``, ``y`` (list of final y arrays per saxpy task) and ``push`` (list of host arrays
    per push task).
    """
    return execute(prepare(g, with_data))


def execute(prep):
    """Run a graph prepared by ``prepare`` (the part the CPU baseline times)."""
    arr, order, stamp, cnt = kahn(*prep["args"])
    return dict(arr=arr, order=order, stamp=stamp, count=cnt, y=prep["y"], push=prep["push"], x=prep["x"])


def prepare(g, with_data=True):
    """Host stand-ins for every buffer of ``g`` and the argument tuple of ``kahn``."""
    from paper_2203_08395_b300.synth import KIND_SAXPY_I32  # generator constants only

    n = g.n
    if not with_data or g.sx_task.size == 0:
        return dict(args=(n, g.src, g.dst, g.delay, g.arr0), y=[], push=[], x=[])
    op = np.zeros(n, np.uint8)
    p0 = np.zeros(n, np.uint64)
    p1 = np.zeros(n, np.uint64)
    length = np.zeros(n, np.int64)
    a_f = np.zeros(n, np.float32)
    a_i = np.zeros(n, np.int32)
    keep = []
    xs, ys = [], []
    for j, t in enumerate(g.sx_task):
        i32 = int(g.kind[t]) == KIND_SAXPY_I32
        if int(g.sx_pull[j]) >= 0:
            x = np.zeros(int(g.sx_n[j]), np.int32 if i32 else np.float32)  # device buffer of the pull
        else:
            x = g.init_x(j)
        y = g.init_y(j)
        xs.append(x)
        ys.append(y)
        op[t] = OP_SAXPY_I32 if i32 else OP_SAXPY_F32
        p0[t] = y.ctypes.data
        p1[t] = x.ctypes.data
        length[t] = y.size
        a_f[t] = g.sx_a[j]
        a_i[t] = int(g.sx_a[j])
    for i, t in enumerate(g.pl_task):
        j = int(g.pl_saxpy[i])
        h = g.pull_data(j)
        keep.append(h)
        op[t] = OP_COPY
        p0[t] = xs[j].ctypes.data
        p1[t] = h.ctypes.data
        length[t] = h.nbytes
    pushes = []
    for i, t in enumerate(g.ps_task):
        j = int(g.ps_saxpy[i])
        h = np.zeros_like(ys[j])
        pushes.append(h)
        op[t] = OP_COPY
        p0[t] = h.ctypes.data
        p1[t] = ys[j].ctypes.data
        length[t] = h.nbytes
    return dict(args=(n, g.src, g.dst, g.delay, g.arr0, op, p0, p1, length, a_f, a_i), y=ys, push=pushes, x=xs,
                keep=keep)


def bottom_levels(n, src, dst, cost):
    """Bottom-level (critical-path) weights b(v) = c(v) + max over successors s of b(s),
    b(sink) = c(sink), computed as arrivals on the reversed graph: reversed edge s->v carries
    delay c(v) and sinks start at c(sink). Exact for the same reason arrivals are: each sum has
    fixed inputs and rounding is monotone, so fl(max_s b(s) + c) = max_s fl(b(s) + c)."""
    cost = np.ascontiguousarray(cost, np.float32)
    rs = np.ascontiguousarray(dst, np.int32)
    rd = np.ascontiguousarray(src, np.int32)
    arr, _, _, cnt = kahn(n, rs, rd, cost[rd], arr0=cost)
    if cnt != n:
        raise ValueError("cycle")
    return arr
