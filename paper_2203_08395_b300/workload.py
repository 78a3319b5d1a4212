"""Places a synthetic workload (``synth.Workload``) on the device through the C ABI.

Builds one hf graph per ``synth.GraphSpec`` (tasks added in id order: runs of max-plus tasks
with hf_add_tasks_bulk, saxpy/pull/push tasks with hf_add_task, edges with hf_precede_bulk)
and owns the payload buffers: saxpy x and y live in two device pools (torch tensors, every
buffer 16-byte aligned), pull sources and push targets in page-locked host pools. Batches put
all graphs into one hf_batch. Nothing here computes anything of the method.
"""
from __future__ import annotations

import numpy as np

from . import hf
from . import synth as S


def _align4(n):
    return (int(n) + 3) // 4 * 4


class GraphOnDevice:
    def __init__(self, spec: S.GraphSpec, device="cuda", fill_data=True):
        import torch

        self.spec = spec
        self.device = device
        k = spec.sx_task.size
        i32 = np.array([spec.saxpy_is_i32(j) for j in range(k)], bool)
        dt = torch.float32
        if k and i32.any():
            assert i32.all(), "a graph mixes FP32 and int32 saxpy tasks"
            dt = torch.int32
        self.dtype = dt
        sizes = spec.sx_n.astype(np.int64)
        al = np.array([_align4(s) for s in sizes], np.int64)
        self.y_off = np.concatenate([[0], np.cumsum(al)])[:-1] if k else np.zeros(0, np.int64)
        has_x = spec.sx_pull < 0 if k else np.zeros(0, bool)
        xal = np.where(has_x, al, 0)
        self.x_off = np.concatenate([[0], np.cumsum(xal)])[:-1] if k else np.zeros(0, np.int64)
        ny, nx = int(al.sum()), int(xal.sum())
        self.y = torch.zeros(max(ny, 4), dtype=dt, device=device)
        self.x = torch.zeros(max(nx, 4), dtype=dt, device=device)
        self.y0 = None
        # pulls: host source pool; pushes: host target pool (page-locked)
        pl_sizes = [int(sizes[j]) for j in spec.pl_saxpy]
        ps_sizes = [int(sizes[j]) for j in spec.ps_saxpy]
        self.pl_off = np.concatenate([[0], np.cumsum([_align4(s) for s in pl_sizes])]).astype(np.int64)
        self.ps_off = np.concatenate([[0], np.cumsum([_align4(s) for s in ps_sizes])]).astype(np.int64)
        self.pull_host = torch.zeros(max(int(self.pl_off[-1]), 4), dtype=dt, pin_memory=True)
        self.push_host = torch.zeros(max(int(self.ps_off[-1]), 4), dtype=dt, pin_memory=True)
        if fill_data:
            self.fill()
        self.g = None
        self._build()

    # ------------------------------------------------------------------ data
    def fill(self):
        """(Re)write every payload buffer with its seeded initial data."""
        import torch

        spec = self.spec
        k = spec.sx_task.size
        if not k:
            return
        i32 = self.dtype == torch.int32
        npdt = np.int32 if i32 else np.float32
        lo, hi = (-1000, 1000) if i32 else (-1.0, 1.0)
        js = np.arange(k, dtype=np.int64)
        hy = np.zeros(self.y.numel(), npdt)
        S.fill_multi(spec.data_seed, 4 * js + 1, spec.sx_n, self.y_off, hy, lo, hi)
        hx = np.zeros(self.x.numel(), npdt)
        own = spec.sx_pull < 0
        S.fill_multi(spec.data_seed, 4 * js[own], spec.sx_n[own], self.x_off[own], hx, lo, hi)
        self.y.copy_(torch.from_numpy(hy))
        self.x.copy_(torch.from_numpy(hx))
        if spec.pl_saxpy.size:
            jp = spec.pl_saxpy.astype(np.int64)
            S.fill_multi(spec.data_seed, 4 * jp + 2, spec.sx_n[jp], self.pl_off[:-1], self.pull_host.numpy(), lo, hi)
        self.push_host.zero_()
        self.y0 = self.y.clone()

    def reset_y(self):
        """Restore every y buffer to its initial data (device copy, on the current stream)."""
        if self.y0 is not None:
            self.y.copy_(self.y0)
        self.push_host.zero_()

    def y_of(self, j):
        o, n = int(self.y_off[j]), int(self.spec.sx_n[j])
        return self.y[o:o + n]

    def push_of(self, i):
        o, n = int(self.ps_off[i]), int(self.spec.sx_n[self.spec.ps_saxpy[i]])
        return self.push_host[o:o + n]

    # ------------------------------------------------------------------ graph
    def _build(self):
        spec = self.spec
        g = hf.hf_graph_create(spec.n, spec.m)
        self.g = g
        kind = spec.kind
        sx_index = {int(t): j for j, t in enumerate(spec.sx_task)}
        pl_index = {int(t): i for i, t in enumerate(spec.pl_task)}
        ps_index = {int(t): i for i, t in enumerate(spec.ps_task)}
        esz = self.y.element_size()
        arr0 = spec.arr0
        v = 0
        n = spec.n
        special = np.nonzero(kind != S.KIND_MAXPLUS)[0]
        sp_i = 0
        while v < n:
            nxt = int(special[sp_i]) if sp_i < special.size else n
            if nxt > v:  # run of max-plus tasks [v, nxt)
                first = hf.hf_add_tasks_bulk(g, nxt - v, None if arr0 is None else arr0[v:nxt])
                assert first == v
                v = nxt
                continue
            kd = int(kind[v])
            if kd in (S.KIND_SAXPY, S.KIND_SAXPY_I32):
                j = sx_index[v]
                p = hf.hf_saxpy_payload()
                p.op = hf.HF_K_SAXPY_I32 if kd == S.KIND_SAXPY_I32 else hf.HF_K_SAXPY_F32
                p.a_f = float(spec.sx_a[j])
                p.a_i = int(spec.sx_a[j])
                p.n = int(spec.sx_n[j])
                p.y_pull = -1
                p.y_dev = self.y.data_ptr() + esz * int(self.y_off[j])
                if spec.sx_pull[j] >= 0:
                    p.x_pull = int(spec.sx_pull[j])
                    p.x_dev = None
                else:
                    p.x_pull = -1
                    p.x_dev = self.x.data_ptr() + esz * int(self.x_off[j])
                t = hf.hf_add_task(g, hf.HF_KERNEL, p)
            elif kd == S.KIND_PULL:
                i = pl_index[v]
                j = int(spec.pl_saxpy[i])
                p = hf.hf_pull_payload()
                p.host_ptr = self.pull_host.data_ptr() + esz * int(self.pl_off[i])
                p.bytes = esz * int(spec.sx_n[j])
                t = hf.hf_add_task(g, hf.HF_PULL, p)
            elif kd == S.KIND_PUSH:
                i = ps_index[v]
                j = int(spec.ps_saxpy[i])
                p = hf.hf_push_payload()
                p.src_pull = -1
                p.src_dev = self.y.data_ptr() + esz * int(self.y_off[j])
                p.host_ptr = self.push_host.data_ptr() + esz * int(self.ps_off[i])
                p.bytes = esz * int(spec.sx_n[j])
                t = hf.hf_add_task(g, hf.HF_PUSH, p)
            else:
                raise ValueError("unknown task kind %d" % kd)
            assert t == v
            v += 1
            sp_i += 1
        hf.hf_precede_bulk(g, spec.src, spec.dst, spec.delay)

    def run(self, stream=None, **opts):
        hf.hf_run(self.g, stream, hf.hf_run_opts_default(**opts))

    def run_host(self, delay, arr_out, stream=None, **opts):
        hf.hf_run_host(self.g, delay, arr_out, stream, hf.hf_run_opts_default(**opts))

    def sync(self, check=True):
        return hf.hf_sync_status(self.g, check)

    def arrivals(self):
        return hf.hf_get_arrivals(self.g, self.spec.n)

    def close(self):
        if self.g is not None:
            hf.hf_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchOnDevice:
    """All graphs of a workload in one hf_batch (one launch per run)."""

    def __init__(self, wl: S.Workload, device="cuda", fill_data=True):
        self.wl = wl
        self.graphs = [GraphOnDevice(g, device, fill_data) for g in wl.graphs]
        self.b = hf.hf_batch_create()
        for i, gd in enumerate(self.graphs):
            assert hf.hf_batch_add(self.b, gd.g) == i

    @property
    def n_tasks(self):
        return self.wl.n_tasks

    @property
    def n_edges(self):
        return self.wl.n_edges

    def run(self, stream=None, **opts):
        hf.hf_batch_run(self.b, stream, hf.hf_run_opts_default(**opts))

    def run_host(self, delay, arr_out, stream=None, **opts):
        hf.hf_batch_run_host(self.b, delay, arr_out, stream, hf.hf_run_opts_default(**opts))

    def sync(self, check=True):
        return hf.hf_batch_sync_status(self.b, check)

    def arrivals(self, i):
        return hf.hf_batch_get_arrivals(self.b, i, self.wl.graphs[i].n)

    def reset_y(self):
        for gd in self.graphs:
            gd.reset_y()

    def close(self):
        if self.b is not None:
            hf.hf_batch_destroy(self.b)
            self.b = None
        for gd in self.graphs:
            gd.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# placeholder payload address for partitioning-only graphs: aligned and non-NULL, never
# dereferenced (such graphs are never run)
_NO_BUFFER = 256


def _structure_graph(spec: S.GraphSpec):
    """An hf graph with the tasks, kinds, payload sizes and edges of `spec` but no payload
    buffers, for host-side analysis only (placement, sharding): it must never run."""
    g = hf.hf_graph_create(spec.n, spec.m)
    kind = spec.kind
    sx_index = {int(t): j for j, t in enumerate(spec.sx_task)}
    pl_index = {int(t): i for i, t in enumerate(spec.pl_task)}
    ps_index = {int(t): i for i, t in enumerate(spec.ps_task)}
    special = np.nonzero(kind != S.KIND_MAXPLUS)[0]
    v, sp_i, n = 0, 0, spec.n
    while v < n:
        nxt = int(special[sp_i]) if sp_i < special.size else n
        if nxt > v:
            hf.hf_add_tasks_bulk(g, nxt - v, None if spec.arr0 is None else spec.arr0[v:nxt])
            v = nxt
            continue
        kd = int(kind[v])
        if kd in (S.KIND_SAXPY, S.KIND_SAXPY_I32):
            j = sx_index[v]
            p = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_I32 if kd == S.KIND_SAXPY_I32 else hf.HF_K_SAXPY_F32,
                                    a_f=float(spec.sx_a[j]), a_i=int(spec.sx_a[j]), n=int(spec.sx_n[j]),
                                    x_pull=int(spec.sx_pull[j]), y_pull=-1, x_dev=_NO_BUFFER, y_dev=_NO_BUFFER)
            hf.hf_add_task(g, hf.HF_KERNEL, p)
        elif kd == S.KIND_PULL:
            j = int(spec.pl_saxpy[pl_index[v]])
            hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=_NO_BUFFER, bytes=4 * int(spec.sx_n[j])))
        elif kd == S.KIND_PUSH:
            j = int(spec.ps_saxpy[ps_index[v]])
            hf.hf_add_task(g, hf.HF_PUSH, hf.hf_push_payload(src_pull=-1, src_dev=_NO_BUFFER, host_ptr=_NO_BUFFER,
                                                             bytes=4 * int(spec.sx_n[j])))
        else:
            raise ValueError("unknown task kind %d" % kd)
        v += 1
        sp_i += 1
    hf.hf_precede_bulk(g, spec.src, spec.dst, spec.delay)
    return g


def partition(wl: S.Workload, ndev: int):
    """Sharding of a workload's graphs over `ndev` devices with hf_batch_partition (graphs packed
    by decreasing heuristic cost, each onto the least-loaded device: the balanced bin packing of
    the paper's Algorithm 1). Host only: it works on structure-only copies of the graphs, so a
    rank can learn its share before it puts any graph on its device. Returns (device of each
    graph, predicted load per device)."""
    b = hf.hf_batch_create()
    gs = []
    try:
        for spec in wl.graphs:
            g = _structure_graph(spec)
            gs.append(g)
            hf.hf_batch_add(b, g)
        return hf.hf_batch_partition(b, len(wl.graphs), ndev)
    finally:
        hf.hf_batch_destroy(b)
        for g in gs:
            hf.hf_graph_destroy(g)


def share(wl: S.Workload, rank: int, world: int):
    """Rank `rank`'s share of `wl` under `partition` (a Workload of its graphs, in batch order)."""
    if world <= 1:
        return wl, list(range(len(wl.graphs)))
    dev, _ = partition(wl, world)
    idx = [i for i in range(len(wl.graphs)) if dev[i] == rank]
    return S.Workload("%s_shard%dof%d" % (wl.name, rank, world), [wl.graphs[i] for i in idx]), idx
