"""Seeded synthetic workloads for the task-graph executor (shared by the CUDA path and the oracle).

Holds none of the method's arithmetic: it draws graph shapes, delays, task kinds, payload sizes
and payload data, and nothing else. The drawing itself happens in ``synth.c`` (splitmix64 /
xoshiro256**), so a workload is a pure function of its seed.

Workload shapes follow the paper's task model (host/pull/push/kernel tasks, explicit edges,
Section III-A) and its timing-analysis setting (million-scale task graphs, Section IV-A):

* ``layered``   -- random layered timing DAG (first predecessor from the previous level);
* ``circuit``   -- circuit-like DAG: geometric fan-in, power-law fan-out, lognormal delays;
* ``mixed``     -- random DAG of max-plus nodes, saxpy kernel tasks (Listing 1's kernel in
                   FP32) and pull/push copy tasks around some saxpy tasks;
* ``batch``     -- many independent layered DAGs of uneven sizes.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhfsynth.so")

# task kinds of a workload description (the C ABI's kinds + kernel ops are derived from these)
KIND_MAXPLUS = 0  # kernel task, max-plus payload only
KIND_SAXPY = 1    # kernel task, FP32 saxpy payload y = a*x + y
KIND_PULL = 2     # pull task: host -> device copy (fills the x buffer of one saxpy task)
KIND_PUSH = 3     # push task: device -> host copy (reads the y buffer of one saxpy task)
KIND_SAXPY_I32 = 4  # kernel task, int32 saxpy (the paper's Listing 1 kernel)


class _Dag(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("levels", ctypes.c_int32),
        ("m", ctypes.c_int64),
        ("src", ctypes.POINTER(ctypes.c_int32)),
        ("dst", ctypes.POINTER(ctypes.c_int32)),
        ("delay", ctypes.POINTER(ctypes.c_float)),
    ]


def build_lib(force: bool = False) -> str:
    """Compile synth.c into libhfsynth.so (gcc, OpenMP) next to this file."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        import subprocess

        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, src, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_lib()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        L.synth_layered.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    P(_Dag)]
        L.synth_circuit.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_double, P(_Dag)]
        L.synth_random.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_double, ctypes.c_double, P(_Dag)]
        L.synth_dag_free.argtypes = [P(_Dag)]
        L.synth_pick.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_void_p]
        L.synth_loguniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_void_p]
        L.synth_uniform_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_void_p]
        L.synth_fill_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.synth_fill_i32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        L.synth_fill_multi_f32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.synth_fill_multi_i32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        for f in ("synth_layered", "synth_circuit", "synth_random", "synth_pick", "synth_loguniform",
                  "synth_uniform_f32", "synth_fill_f32", "synth_fill_i32", "synth_fill_multi_f32",
                  "synth_fill_multi_i32"):
            getattr(L, f).restype = ctypes.c_int
        L.synth_value_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double]
        L.synth_value_f32.restype = ctypes.c_float
        _lib = L
    return _lib


def _take(d: _Dag):
    m = int(d.m)
    if m:
        src = np.ctypeslib.as_array(d.src, shape=(m,)).copy()
        dst = np.ctypeslib.as_array(d.dst, shape=(m,)).copy()
        dly = np.ctypeslib.as_array(d.delay, shape=(m,)).copy()
    else:
        src = np.zeros(0, np.int32)
        dst = np.zeros(0, np.int32)
        dly = np.zeros(0, np.float32)
    n, levels = int(d.n), int(d.levels)
    lib().synth_dag_free(ctypes.byref(d))
    return n, levels, src, dst, dly


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed (rc=%d)" % (what, rc))


def layered_dag(seed, n, levels, fin_lo, fin_hi, d_lo=0.01, d_hi=1.0):
    d = _Dag()
    _check(lib().synth_layered(seed, n, levels, fin_lo, fin_hi, 0, d_lo, d_hi, ctypes.byref(d)), "layered")
    return _take(d)


def circuit_dag(seed, n, levels, p_geom=0.4, fin_max=8, alpha=2.2, wmax=512, fout_max=512, mu=-2.0,
                sigma=0.5):
    d = _Dag()
    _check(lib().synth_circuit(seed, n, levels, p_geom, fin_max, alpha, wmax, fout_max, mu, sigma,
                               ctypes.byref(d)), "circuit")
    return _take(d)


def random_dag(seed, n, fin_lo, fin_hi, window=0, d_lo=0.01, d_hi=1.0):
    d = _Dag()
    _check(lib().synth_random(seed, n, fin_lo, fin_hi, window, d_lo, d_hi, ctypes.byref(d)), "random")
    return _take(d)


def pick(seed, stream, n, k):
    out = np.empty(k, np.int32)
    _check(lib().synth_pick(seed, stream, n, k, out.ctypes.data), "pick")
    return out


def loguniform(seed, stream, k, lo, hi):
    out = np.empty(k, np.int64)
    _check(lib().synth_loguniform(seed, stream, k, lo, hi, out.ctypes.data), "loguniform")
    return out


def uniform_f32(seed, stream, k, lo, hi):
    out = np.empty(k, np.float32)
    _check(lib().synth_uniform_f32(seed, stream, k, lo, hi, out.ctypes.data), "uniform")
    return out


def fill_f32(seed, stream, n, lo=-1.0, hi=1.0, first=0, out=None):
    """Counter-based FP32 data: element i depends only on (seed, stream, first + i)."""
    if out is None:
        out = np.empty(n, np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size >= n
    _check(lib().synth_fill_f32(seed, stream, first, n, lo, hi, out.ctypes.data), "fill_f32")
    return out


def fill_i32(seed, stream, n, lo, hi, first=0, out=None):
    if out is None:
        out = np.empty(n, np.int32)
    assert out.dtype == np.int32 and out.flags.c_contiguous and out.size >= n
    _check(lib().synth_fill_i32(seed, stream, first, n, lo, hi, out.ctypes.data), "fill_i32")
    return out


def fill_multi(seed, streams, counts, offsets, out, lo, hi):
    """Buffer j = the counter-based data of stream streams[j] (counts[j] elements), written
    at out[offsets[j]:]; identical to fill_f32 / fill_i32 per buffer."""
    streams = np.ascontiguousarray(streams, np.uint64)
    counts = np.ascontiguousarray(counts, np.int64)
    offsets = np.ascontiguousarray(offsets, np.int64)
    assert streams.size == counts.size == offsets.size
    if counts.size:
        assert int((offsets + counts).max()) <= out.size
    if out.dtype == np.float32:
        rc = lib().synth_fill_multi_f32(seed, streams.size, streams.ctypes.data, counts.ctypes.data,
                                        offsets.ctypes.data, lo, hi, out.ctypes.data)
    else:
        assert out.dtype == np.int32
        rc = lib().synth_fill_multi_i32(seed, streams.size, streams.ctypes.data, counts.ctypes.data,
                                        offsets.ctypes.data, int(lo), int(hi), out.ctypes.data)
    _check(rc, "fill_multi")
    return out


# ------------------------------------------------------------------ workload descriptions


@dataclass
class GraphSpec:
    """One task graph: edge list, task kinds and payload descriptions (no data yet).

    Saxpy task j (``sx_task[j]``) updates its own y buffer of ``sx_n[j]`` elements with
    ``y = a*x + y``. Its x comes from pull task ``sx_pull[j]`` when that is >= 0 (the pull
    copies host data into the device buffer, the paper's pull-as-gateway pattern), else from a
    device buffer filled before the run. Push task ``ps_task[i]`` copies the y buffer of saxpy
    ``ps_saxpy[i]`` back to a host buffer.

    Element data is counter-based: saxpy j's device x uses stream 4j, its y stream 4j+1, the
    host data behind its pull stream 4j+2, all with seed ``data_seed`` and values in [-1, 1)
    (int32 saxpy: integers in [-1000, 1000]).
    """

    name: str
    n: int
    src: np.ndarray
    dst: np.ndarray
    delay: np.ndarray
    kind: np.ndarray
    levels: int = 0
    sx_task: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    sx_n: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    sx_a: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))
    sx_pull: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    pl_task: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    pl_saxpy: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ps_task: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ps_saxpy: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    arr0: Optional[np.ndarray] = None
    data_seed: int = 0

    @property
    def m(self):
        return int(self.src.size)

    @property
    def saxpy_elems(self):
        return int(self.sx_n.sum()) if self.sx_n.size else 0

    def x_stream(self, j):
        return 4 * int(j)

    def y_stream(self, j):
        return 4 * int(j) + 1

    def pull_stream(self, j):
        return 4 * int(j) + 2

    def saxpy_is_i32(self, j):
        return int(self.kind[self.sx_task[j]]) == KIND_SAXPY_I32

    def init_x(self, j, first=0, n=None):
        n = int(self.sx_n[j]) - first if n is None else n
        if self.saxpy_is_i32(j):
            return fill_i32(self.data_seed, self.x_stream(j), n, -1000, 1000, first)
        return fill_f32(self.data_seed, self.x_stream(j), n, -1.0, 1.0, first)

    def init_y(self, j, first=0, n=None):
        n = int(self.sx_n[j]) - first if n is None else n
        if self.saxpy_is_i32(j):
            return fill_i32(self.data_seed, self.y_stream(j), n, -1000, 1000, first)
        return fill_f32(self.data_seed, self.y_stream(j), n, -1.0, 1.0, first)

    def pull_data(self, j, first=0, n=None):
        n = int(self.sx_n[j]) - first if n is None else n
        if self.saxpy_is_i32(j):
            return fill_i32(self.data_seed, self.pull_stream(j), n, -1000, 1000, first)
        return fill_f32(self.data_seed, self.pull_stream(j), n, -1.0, 1.0, first)


@dataclass
class Workload:
    name: str
    graphs: List[GraphSpec]

    @property
    def n_tasks(self):
        return sum(g.n for g in self.graphs)

    @property
    def n_edges(self):
        return sum(g.m for g in self.graphs)

    @property
    def saxpy_elems(self):
        return sum(g.saxpy_elems for g in self.graphs)


def _maxplus_graph(name, n, levels, src, dst, dly):
    return GraphSpec(name=name, n=n, src=src, dst=dst, delay=dly, kind=np.zeros(n, np.uint8), levels=levels)


def layered(seed=0, n=10_000, levels=40, fin_lo=1, fin_hi=4, name=None):
    """Random layered timing DAG (delays U[0.01, 1.0), sources arrive at +0)."""
    n_, lv, s, d, w = layered_dag(seed, n, levels, fin_lo, fin_hi)
    return _maxplus_graph(name or "layered_n%d_L%d_s%d" % (n, levels, seed), n_, lv, s, d, w)


def circuit(seed=0, n=1_000_000, levels=2000, name=None):
    """Circuit-like timing DAG: geometric fan-in (p=0.4, max 8), power-law fan-out
    (alpha 2.2, cap 512), lognormal delays exp(-2 + 0.5 z)."""
    n_, lv, s, d, w = circuit_dag(seed, n, levels)
    return _maxplus_graph(name or "circuit_n%d_L%d_s%d" % (n, levels, seed), n_, lv, s, d, w)


def _add_saxpy_mix(g: GraphSpec, seed, frac, nmin, nmax, n_copy, a=2.0, i32=False):
    """Turn a max-plus graph into a mixed one: `frac` of its tasks become saxpy kernel tasks
    with sizes log-uniform on [nmin, nmax]; `n_copy` of those get a pull task (host -> x)
    before them and a push task (y -> host) after them. Pull tasks take the lowest ids
    (a kernel task names its pull, so the pull is created first, as in the paper's
    listings), the original tasks follow shifted by n_copy, the push tasks come last."""
    n = g.n
    k = int(round(frac * n))
    sx = pick(seed, 11, n, k)
    kind = g.kind.copy()
    kind[sx] = KIND_SAXPY_I32 if i32 else KIND_SAXPY
    c = int(n_copy)
    g.sx_n = loguniform(seed, 12, k, nmin, nmax)
    g.sx_a = np.full(k, a, np.float32)
    g.sx_pull = np.full(k, -1, np.int32)
    src, dst, dly = g.src + c, g.dst + c, g.delay
    g.sx_task = (sx + c).astype(np.int32)
    if c:
        sel = pick(seed, 13, k, c)  # indices into the saxpy list
        pl = np.arange(0, c, dtype=np.int32)
        ps = np.arange(n + c, n + 2 * c, dtype=np.int32)
        g.sx_pull[sel] = pl
        g.pl_task, g.pl_saxpy = pl, sel.astype(np.int32)
        g.ps_task, g.ps_saxpy = ps, sel.astype(np.int32)
        cd = uniform_f32(seed, 14, 2 * c, 0.01, 1.0)
        src = np.concatenate([src, pl, g.sx_task[sel]]).astype(np.int32)
        dst = np.concatenate([dst, g.sx_task[sel], ps]).astype(np.int32)
        dly = np.concatenate([dly, cd])
        kind = np.concatenate([np.full(c, KIND_PULL, np.uint8), kind, np.full(c, KIND_PUSH, np.uint8)])
    g.src, g.dst, g.delay, g.kind = src.astype(np.int32), dst.astype(np.int32), dly.astype(np.float32), kind
    g.n = n + 2 * c
    g.data_seed = seed
    return g


def mixed(seed=0, n=100_000, frac_saxpy=0.10, nmin=4096, nmax=1 << 20, n_copy=1000, fin_lo=1, fin_hi=6,
          window=0, name=None):
    """Mixed-task random DAG: 90% max-plus nodes, 10% FP32 saxpy tasks (log-uniform sizes),
    plus `n_copy` pull and push tasks around randomly chosen saxpy tasks."""
    n_, _, s, d, w = random_dag(seed, n, fin_lo, fin_hi, window)
    g = _maxplus_graph(name or "mixed_n%d_s%d" % (n, seed), n_, 0, s, d, w)
    return _add_saxpy_mix(g, seed, frac_saxpy, nmin, nmax, n_copy)


def batch(seed=0, graphs=256, nmin=1_000, nmax=200_000, fin_lo=1, fin_hi=6, width=250,
          frac_saxpy=0.0, sx_min=256, sx_max=4096, name=None):
    """Batch of independent layered DAGs with log-uniform sizes; graph g uses seed 1000*seed + g
    and max(4, round(N_g / width)) levels. With frac_saxpy > 0 each graph also gets that share
    of FP32 saxpy tasks (sizes log-uniform on [sx_min, sx_max])."""
    sizes = loguniform(seed, 21, graphs, nmin, nmax)
    out = []
    for gi, ng in enumerate(sizes):
        ng = int(ng)
        lv = max(4, int(round(ng / width)))
        gs = 1000 * seed + gi
        g = layered(gs, ng, lv, fin_lo, fin_hi, name="g%d" % gi)
        if frac_saxpy > 0:
            _add_saxpy_mix(g, gs, frac_saxpy, sx_min, sx_max, 0)
        out.append(g)
    return Workload(name or "batch%d_s%d" % (graphs, seed), out)


def paper_saxpy_example(N=65536):
    """The paper's saxpy graph (Listing 1, Fig. 1): host_x, host_y, pull_x, pull_y, kernel,
    push_x, push_y with edges host_x->pull_x, host_y->pull_y, pull_x->kernel,
    pull_y->kernel, kernel->push_x, kernel->push_y. Task ids in that order; int32 data;
    host tasks fill x with 1 and y with 2; the kernel computes y = 2*x + y."""
    names = ["host_x", "host_y", "pull_x", "pull_y", "kernel", "push_x", "push_y"]
    edges = [(0, 2), (1, 3), (2, 4), (3, 4), (4, 5), (4, 6)]
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    return names, src, dst, N


def paper_dependency_example():
    """The paper's eight-task, seven-edge graph (Fig. 2, Listing 8): task ids in listing order."""
    names = ["host1", "host2", "pull1", "pull2", "push1", "push2", "kernel1", "kernel2"]
    ix = {nm: i for i, nm in enumerate(names)}
    pairs = [("host1", "pull1"), ("host2", "pull2"), ("pull1", "kernel1"), ("pull2", "kernel2"),
             ("kernel1", "push1"), ("kernel1", "kernel2"), ("kernel2", "push2")]
    src = np.array([ix[a] for a, _ in pairs], np.int32)
    dst = np.array([ix[b] for _, b in pairs], np.int32)
    return names, src, dst


# ------------------------------------------------------------------ named configurations

def config(name: str, seed: int = 0) -> Workload:
    """The five evaluation configurations (see the project design notes for the recipe), and
    batch32 / batch32_mixed: the batch recipe with 32 graphs, a small case for profiling."""
    if name == "layered10k":
        return Workload("layered10k", [layered(seed, 10_000, 40, 1, 4)])
    if name == "circuit1m":
        return Workload("circuit1m", [circuit(seed, 1_000_000, 2000)])
    if name == "mixed100k":
        return Workload("mixed100k", [mixed(seed)])
    if name == "batch256":
        return batch(seed, name="batch256")
    if name == "batch256_mixed":
        return batch(seed, frac_saxpy=0.10, name="batch256_mixed")
    if name == "batch32":
        return batch(seed, graphs=32, name="batch32")
    if name == "batch32_mixed":
        return batch(seed, graphs=32, frac_saxpy=0.10, name="batch32_mixed")
    raise KeyError(name)


CONFIG_NAMES = ["layered10k", "circuit1m", "mixed100k", "batch256", "batch256_mixed"]


def log_uniform_mean(lo, hi):
    return (hi - lo) / math.log(hi / lo)
