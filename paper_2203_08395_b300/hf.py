"""Thin Python binding of the C ABI in include/hf.h (argument marshalling only).

Every function here has the name of the C call it wraps and raises ``HfError`` when that call
returns a status other than HF_OK. All work happens in libhf.so (CUDA, sm_103a); importing this
module fails loudly when the library is missing. PyTorch provides device memory (through the
allocator hook) and streams; nothing here computes anything of the method.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhf.so")

HF_OK, HF_EINVAL, HF_ENOMEM, HF_ECYCLE, HF_ESTATE, HF_ETIMEDOUT, HF_EQUEUE, HF_ECUDA, HF_ENOTSUP = range(9)
HF_HOST, HF_PULL, HF_PUSH, HF_KERNEL = 0, 1, 2, 3
HF_K_MAXPLUS, HF_K_SAXPY_F32, HF_K_SAXPY_I32 = 0, 1, 2
HF_MODE_LEVELSYNC, HF_MODE_PERSISTENT, HF_MODE_AUTO, HF_MODE_TEAM = 0, 1, 2, 3
HF_PRIO_FIFO, HF_PRIO_HEURISTIC, HF_PRIO_LEARNED = 0, 1, 2

STATUS_NAMES = {0: "HF_OK", 1: "HF_EINVAL", 2: "HF_ENOMEM", 3: "HF_ECYCLE", 4: "HF_ESTATE", 5: "HF_ETIMEDOUT",
                6: "HF_EQUEUE", 7: "HF_ECUDA", 8: "HF_ENOTSUP"}


class HfError(RuntimeError):
    def __init__(self, status, where, message=""):
        self.status = status
        super().__init__("%s: %s%s" % (where, STATUS_NAMES.get(status, str(status)),
                                       (" (%s)" % message) if message else ""))


class hf_maxplus_payload(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("arr0", ctypes.c_float)]


class hf_saxpy_payload(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a_i", ctypes.c_int32), ("a_f", ctypes.c_float),
                ("x_pull", ctypes.c_int32), ("y_pull", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("n", ctypes.c_int64), ("x_dev", ctypes.c_void_p), ("y_dev", ctypes.c_void_p)]


class hf_pull_payload(ctypes.Structure):
    _fields_ = [("host_ptr", ctypes.c_void_p), ("bytes", ctypes.c_size_t)]


class hf_push_payload(ctypes.Structure):
    _fields_ = [("src_pull", ctypes.c_int32), ("pad_", ctypes.c_int32), ("src_dev", ctypes.c_void_p),
                ("host_ptr", ctypes.c_void_p), ("bytes", ctypes.c_size_t)]


HOST_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p)


class hf_host_payload(ctypes.Structure):
    _fields_ = [("fn", HOST_FN), ("arg", ctypes.c_void_p)]


class hf_run_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("priority", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("claim", ctypes.c_int32), ("local_keep", ctypes.c_int32),
                ("chunk_elems", ctypes.c_int64), ("spin_limit_ns", ctypes.c_uint64),
                ("instrument", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("stall_task", ctypes.c_int32), ("time_kernel", ctypes.c_int32),
                ("payload_warps", ctypes.c_int32), ("team_size", ctypes.c_int32),
                ("team_scale", ctypes.c_int32), ("steal_ring", ctypes.c_int32),
                ("copy_warps", ctypes.c_int32), ("team_fold", ctypes.c_int32),
                ("team_global_keys", ctypes.c_int32)]


class hf_graph_info_t(ctypes.Structure):
    _fields_ = [("tasks", ctypes.c_int64), ("edges", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("sources", ctypes.c_int32), ("kind_count", ctypes.c_int64 * 4), ("payload_tasks", ctypes.c_int64),
                ("finalized", ctypes.c_int32), ("pad_", ctypes.c_int32)]


PRED_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_keep = []  # callbacks that must outlive the library's use of them


def load():
    """Load libhf.so; raise if it has not been built (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhf.so not built: run paper_2203_08395_b300/build.py (or __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "hf_graph_create": [P(vp), i64, i64],
        "hf_graph_destroy": [vp],
        "hf_add_task": [vp, ctypes.c_int, vp, ctypes.c_size_t, P(i32)],
        "hf_add_tasks_bulk": [vp, i64, vp, P(i32)],
        "hf_precede": [vp, i32, i32],
        "hf_precede_w": [vp, i32, i32, ctypes.c_float],
        "hf_precede_bulk": [vp, i64, vp, vp, vp],
        "hf_finalize": [vp],
        "hf_graph_info": [vp, P(hf_graph_info_t)],
        "hf_get_levels": [vp, vp],
        "hf_run": [vp, vp, P(hf_run_opts)],
        "hf_run_host": [vp, vp, P(hf_run_opts), vp, vp],
        "hf_sync_status": [vp],
        "hf_get_arrivals": [vp, vp, ctypes.c_int],
        "hf_get_stamps": [vp, vp, vp, vp],
        "hf_get_task_times": [vp, vp, vp],
        "hf_batch_create": [P(vp)],
        "hf_batch_destroy": [vp],
        "hf_batch_add": [vp, vp, P(i32)],
        "hf_batch_run": [vp, vp, P(hf_run_opts)],
        "hf_batch_run_host": [vp, vp, P(hf_run_opts), vp, vp],
        "hf_batch_sync_status": [vp],
        "hf_batch_get_arrivals": [vp, i32, vp, ctypes.c_int],
        "hf_batch_get_task_times": [vp, i32, vp, vp],
        "hf_batch_get_stamps": [vp, i32, vp, vp, vp],
        "hf_set_allocator": [ALLOC_FN, FREE_FN, vp],
        "hf_kernel_ms": [vp, P(ctypes.c_float)],
        "hf_batch_kernel_ms": [vp, P(ctypes.c_float)],
        "hf_set_delays": [vp, vp, ctypes.c_int, vp],
        "hf_batch_set_delays": [vp, vp, ctypes.c_int, vp],
        "hf_costmodel_create": [P(vp), ctypes.c_uint64],
        "hf_costmodel_destroy": [vp],
        "hf_costmodel_set_params": [vp, vp],
        "hf_costmodel_get_params": [vp, vp],
        "hf_costmodel_save": [vp, ctypes.c_char_p],
        "hf_costmodel_load": [vp, ctypes.c_char_p],
        "hf_costmodel_forward": [vp, vp, i64, vp, vp],
        "hf_costmodel_grad": [vp, vp, vp, i64, vp, vp, vp],
        "hf_costmodel_adam_step": [vp, vp, ctypes.c_float, vp],
        "hf_costmodel_train": [vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64, P(ctypes.c_float), vp],
        "hf_batch_features": [vp, vp, vp],
        "hf_features": [vp, vp, vp],
        "hf_batch_set_costmodel": [vp, vp],
        "hf_batch_refresh_priorities": [vp, vp],
        "hf_batch_task_costs": [vp, i32, vp, vp, vp],
        "hf_batch_bottom_levels": [vp, vp, vp, vp],
        "hf_batch_autotune": [vp, vp, P(hf_run_opts), ctypes.c_int, P(hf_run_opts), P(ctypes.c_float)],
        "hf_batch_get_stats": [vp, vp, i32],
        "hf_batch_predict": [vp, i32, vp, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float)],
        "hf_run_csr_noalloc": [i32, i32, vp, vp, vp, vp, vp, ctypes.c_uint64, vp],
        "hf_batch_get_graph_times": [vp, vp, vp],
        "hf_batch_get_task_costs": [vp, i32, vp],
        "hf_batch_last_launches": [vp, P(i32)],
        "hf_batch_team_plan": [vp, vp],
        "hf_batch_team_keys": [vp, vp],
        "hf_batch_team_flags": [vp, vp],
        "hf_calibration": [vp, vp],
        "hf_dump": [vp, ctypes.c_char_p],
        "hf_place": [vp, i32, vp, vp],
        "hf_batch_partition": [vp, i32, vp, vp],
        "hf_run_n": [vp, vp, P(hf_run_opts), i32],
        "hf_batch_run_n": [vp, vp, P(hf_run_opts), i32],
        "hf_run_until": [vp, vp, P(hf_run_opts), PRED_FN, vp, i32, P(i32)],
        "hf_batch_run_until": [vp, vp, P(hf_run_opts), PRED_FN, vp, i32, P(i32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.hf_run_opts_default.argtypes = [P(hf_run_opts)]
    L.hf_run_opts_default.restype = None
    L.hf_status_string.argtypes = [ctypes.c_int]
    L.hf_status_string.restype = ctypes.c_char_p
    L.hf_last_error.argtypes = []
    L.hf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status, where):
    if status != HF_OK:
        raise HfError(status, where, load().hf_last_error().decode(errors="replace"))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return int(a)


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------- allocator backed by torch

def install_torch_allocator():
    """Route library-owned device allocations through PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _keep.extend([a, f])
    _check(load().hf_set_allocator(a, f, None), "hf_set_allocator")


# ---------------------------------------------------------------- C ABI, one function per call

def hf_run_opts_default(**kw):
    o = hf_run_opts()
    load().hf_run_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def hf_graph_create(reserve_tasks=0, reserve_edges=0):
    g = ctypes.c_void_p()
    _check(load().hf_graph_create(ctypes.byref(g), reserve_tasks, reserve_edges), "hf_graph_create")
    return g


def hf_graph_destroy(g):
    _check(load().hf_graph_destroy(g), "hf_graph_destroy")


def hf_add_task(g, kind, payload=None):
    t = ctypes.c_int32()
    pp = ctypes.byref(payload) if payload is not None else None
    nb = ctypes.sizeof(payload) if payload is not None else 0
    _check(load().hf_add_task(g, kind, pp, nb, ctypes.byref(t)), "hf_add_task")
    return t.value


def hf_add_tasks_bulk(g, n, arr0=None):
    t = ctypes.c_int32()
    if arr0 is not None:
        arr0 = np.ascontiguousarray(arr0, np.float32)
        assert arr0.size == n
    _check(load().hf_add_tasks_bulk(g, n, _ptr(arr0), ctypes.byref(t)), "hf_add_tasks_bulk")
    return t.value


def hf_precede(g, a, b):
    _check(load().hf_precede(g, a, b), "hf_precede")


def hf_precede_w(g, a, b, delay):
    _check(load().hf_precede_w(g, a, b, delay), "hf_precede_w")


def hf_precede_bulk(g, src, dst, delay=None):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    if delay is not None:
        delay = np.ascontiguousarray(delay, np.float32)
        assert delay.size == src.size
    assert src.size == dst.size
    _check(load().hf_precede_bulk(g, src.size, _ptr(src), _ptr(dst), _ptr(delay)), "hf_precede_bulk")


def hf_finalize(g):
    _check(load().hf_finalize(g), "hf_finalize")


def hf_graph_info(g):
    info = hf_graph_info_t()
    _check(load().hf_graph_info(g, ctypes.byref(info)), "hf_graph_info")
    return dict(tasks=info.tasks, edges=info.edges, levels=info.levels, sources=info.sources,
                kind_count=list(info.kind_count), payload_tasks=info.payload_tasks, finalized=bool(info.finalized))


def hf_get_levels(g, n):
    out = np.empty(n, np.int32)
    _check(load().hf_get_levels(g, _ptr(out)), "hf_get_levels")
    return out


def hf_run(g, stream=None, opts=None):
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_run(g, _stream_handle(stream), ctypes.byref(o)), "hf_run")


def hf_run_host(g, delay, arr_out, stream=None, opts=None):
    """hf_run on new delays from page-locked host memory, arrivals written to page-locked host
    memory (float32 tensors or arrays; None for either to skip it). Non-blocking."""
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_run_host(g, _stream_handle(stream), ctypes.byref(o), _ptr(delay), _ptr(arr_out)), "hf_run_host")


def hf_sync_status(g, check=True):
    s = load().hf_sync_status(g)
    if check:
        _check(s, "hf_sync_status")
    return s


def hf_get_arrivals(g, n, out=None, on_device=False):
    """Host: returns a new float32 numpy array (blocking). Device: `out` is a CUDA tensor."""
    if on_device:
        _check(load().hf_get_arrivals(g, _ptr(out), 1), "hf_get_arrivals")
        return out
    out = np.empty(n, np.float32) if out is None else out
    _check(load().hf_get_arrivals(g, _ptr(out), 0), "hf_get_arrivals")
    return out


def hf_get_stamps(g, n):
    s0, s1, c = np.empty(n, np.int64), np.empty(n, np.int64), np.empty(n, np.int32)
    _check(load().hf_get_stamps(g, _ptr(s0), _ptr(s1), _ptr(c)), "hf_get_stamps")
    return s0, s1, c


def hf_get_task_times(g, n):
    t0, t1 = np.empty(n, np.int64), np.empty(n, np.int64)
    _check(load().hf_get_task_times(g, _ptr(t0), _ptr(t1)), "hf_get_task_times")
    return t0, t1


def hf_batch_create():
    b = ctypes.c_void_p()
    _check(load().hf_batch_create(ctypes.byref(b)), "hf_batch_create")
    return b


def hf_batch_destroy(b):
    _check(load().hf_batch_destroy(b), "hf_batch_destroy")


def hf_batch_add(b, g):
    i = ctypes.c_int32()
    _check(load().hf_batch_add(b, g, ctypes.byref(i)), "hf_batch_add")
    return i.value


def hf_batch_run(b, stream=None, opts=None):
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_batch_run(b, _stream_handle(stream), ctypes.byref(o)), "hf_batch_run")


def hf_batch_run_host(b, delay, arr_out, stream=None, opts=None):
    """hf_batch_run on new delays from page-locked host memory (batch edge order), every arrival
    written to page-locked host memory (batch task order). Non-blocking."""
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_batch_run_host(b, _stream_handle(stream), ctypes.byref(o), _ptr(delay), _ptr(arr_out)),
           "hf_batch_run_host")


def hf_batch_sync_status(b, check=True):
    s = load().hf_batch_sync_status(b)
    if check:
        _check(s, "hf_batch_sync_status")
    return s


def hf_batch_get_arrivals(b, index, n, out=None, on_device=False):
    if on_device:
        _check(load().hf_batch_get_arrivals(b, index, _ptr(out), 1), "hf_batch_get_arrivals")
        return out
    out = np.empty(n, np.float32) if out is None else out
    _check(load().hf_batch_get_arrivals(b, index, _ptr(out), 0), "hf_batch_get_arrivals")
    return out


def hf_batch_get_task_times(b, index, n):
    t0, t1 = np.empty(n, np.int64), np.empty(n, np.int64)
    _check(load().hf_batch_get_task_times(b, index, _ptr(t0), _ptr(t1)), "hf_batch_get_task_times")
    return t0, t1


def hf_batch_get_stamps(b, index, n):
    s0, s1, c = np.empty(n, np.int64), np.empty(n, np.int64), np.empty(n, np.int32)
    _check(load().hf_batch_get_stamps(b, index, _ptr(s0), _ptr(s1), _ptr(c)), "hf_batch_get_stamps")
    return s0, s1, c


def hf_kernel_ms(g):
    ms = ctypes.c_float()
    _check(load().hf_kernel_ms(g, ctypes.byref(ms)), "hf_kernel_ms")
    return ms.value


def hf_batch_kernel_ms(b):
    ms = ctypes.c_float()
    _check(load().hf_batch_kernel_ms(b, ctypes.byref(ms)), "hf_batch_kernel_ms")
    return ms.value


def hf_set_delays(g, delay, on_device=False, stream=None):
    """delay: float32 numpy array (host; page-locked tensors copy asynchronously) or a CUDA
    tensor with on_device=True."""
    if not on_device and isinstance(delay, np.ndarray):
        delay = np.ascontiguousarray(delay, np.float32)
    _check(load().hf_set_delays(g, _ptr(delay), 1 if on_device else 0, _stream_handle(stream)), "hf_set_delays")


def hf_batch_set_delays(b, delay, on_device=False, stream=None):
    if not on_device and isinstance(delay, np.ndarray):
        delay = np.ascontiguousarray(delay, np.float32)
    _check(load().hf_batch_set_delays(b, _ptr(delay), 1 if on_device else 0, _stream_handle(stream)),
           "hf_batch_set_delays")


HF_COSTMODEL_PARAMS = 5057
HF_FEATURES = 12


def hf_costmodel_create(seed=0):
    cm = ctypes.c_void_p()
    _check(load().hf_costmodel_create(ctypes.byref(cm), seed), "hf_costmodel_create")
    return cm


def hf_costmodel_destroy(cm):
    _check(load().hf_costmodel_destroy(cm), "hf_costmodel_destroy")


def hf_costmodel_set_params(cm, params):
    params = np.ascontiguousarray(params, np.float32)
    assert params.size == HF_COSTMODEL_PARAMS
    _check(load().hf_costmodel_set_params(cm, _ptr(params)), "hf_costmodel_set_params")


def hf_costmodel_get_params(cm):
    out = np.empty(HF_COSTMODEL_PARAMS, np.float32)
    _check(load().hf_costmodel_get_params(cm, _ptr(out)), "hf_costmodel_get_params")
    return out


def hf_costmodel_save(cm, path):
    _check(load().hf_costmodel_save(cm, path.encode()), "hf_costmodel_save")


def hf_costmodel_load(cm, path):
    _check(load().hf_costmodel_load(cm, path.encode()), "hf_costmodel_load")


def hf_costmodel_forward(cm, X, n, y, stream=None):
    """X: CUDA tensor [n, 12] float32; y: CUDA tensor [n] float32 (written)."""
    _check(load().hf_costmodel_forward(cm, _ptr(X), n, _ptr(y), _stream_handle(stream)), "hf_costmodel_forward")


def hf_costmodel_grad(cm, X, t, n, grad, loss, stream=None):
    _check(load().hf_costmodel_grad(cm, _ptr(X), _ptr(t), n, _ptr(grad), _ptr(loss), _stream_handle(stream)),
           "hf_costmodel_grad")


def hf_costmodel_adam_step(cm, grad, lr, stream=None):
    _check(load().hf_costmodel_adam_step(cm, _ptr(grad), lr, _stream_handle(stream)), "hf_costmodel_adam_step")


def hf_costmodel_train(cm, X, t, n, epochs, batch, lr, seed=0, stream=None):
    loss = ctypes.c_float()
    _check(load().hf_costmodel_train(cm, _ptr(X), _ptr(t), n, epochs, batch, lr, seed, ctypes.byref(loss),
                                     _stream_handle(stream)), "hf_costmodel_train")
    return loss.value


def hf_batch_features(b, X, stream=None):
    _check(load().hf_batch_features(b, _ptr(X), _stream_handle(stream)), "hf_batch_features")


def hf_features(g, X, stream=None):
    _check(load().hf_features(g, _ptr(X), _stream_handle(stream)), "hf_features")


def hf_batch_set_costmodel(b, cm):
    _check(load().hf_batch_set_costmodel(b, cm), "hf_batch_set_costmodel")


def hf_batch_refresh_priorities(b, stream=None):
    _check(load().hf_batch_refresh_priorities(b, _stream_handle(stream)), "hf_batch_refresh_priorities")


def hf_batch_task_costs(b, priority, cost, bottom, stream=None):
    _check(load().hf_batch_task_costs(b, priority, _ptr(cost), _ptr(bottom), _stream_handle(stream)),
           "hf_batch_task_costs")


def hf_batch_bottom_levels(b, cost, bottom, stream=None):
    _check(load().hf_batch_bottom_levels(b, _ptr(cost), _ptr(bottom), _stream_handle(stream)),
           "hf_batch_bottom_levels")


def hf_batch_autotune(b, stream=None, base=None, force=False):
    """Returns (best hf_run_opts, best ms)."""
    best = hf_run_opts()
    ms = ctypes.c_float()
    _check(load().hf_batch_autotune(b, _stream_handle(stream), ctypes.byref(base) if base is not None else None,
                                    1 if force else 0, ctypes.byref(best), ctypes.byref(ms)), "hf_batch_autotune")
    return best, ms.value


def hf_batch_predict(b, priority, stream=None):
    """Returns predicted (level-sync ms, persistent ms, team ms)."""
    ls, pe, tm = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(load().hf_batch_predict(b, priority, _stream_handle(stream), ctypes.byref(ls), ctypes.byref(pe),
                                   ctypes.byref(tm)), "hf_batch_predict")
    return ls.value, pe.value, tm.value


def hf_batch_get_graph_times(b, ngraphs):
    """Per-graph (start, end) %globaltimer ns of the last instrumented team run."""
    s0, s1 = np.empty(ngraphs, np.int64), np.empty(ngraphs, np.int64)
    _check(load().hf_batch_get_graph_times(b, s0.ctypes.data, s1.ctypes.data), "hf_batch_get_graph_times")
    return s0, s1


def hf_batch_get_task_costs(b, index, n):
    """Per-task costs (ns, float32[n]) of the last team run with instrument bit 2: graph `index`,
    or every graph concatenated in batch order for index -1."""
    out = np.empty(n, np.float32)
    _check(load().hf_batch_get_task_costs(b, index, out.ctypes.data), "hf_batch_get_task_costs")
    return out


def hf_batch_last_launches(b):
    n = ctypes.c_int32()
    _check(load().hf_batch_last_launches(b, ctypes.byref(n)), "hf_batch_last_launches")
    return n.value


def hf_batch_team_plan(b, ngraphs):
    """Team size each graph ran on in the last team-executor run (int32 array)."""
    k = np.zeros(ngraphs, np.int32)
    _check(load().hf_batch_team_plan(b, k.ctypes.data), "hf_batch_team_plan")
    return k


TEAM_SHARED_KEYS, TEAM_PIPELINED, TEAM_PAYLOAD_LOCAL = 1, 2, 4


def hf_batch_team_flags(b, ngraphs):
    """How each graph ran in the last team-executor run (int32 array of TEAM_* bits)."""
    f = np.zeros(ngraphs, np.int32)
    _check(load().hf_batch_team_flags(b, f.ctypes.data), "hf_batch_team_flags")
    return f


def hf_batch_team_keys(b, ngraphs):
    """1 where a graph kept its keys in shared memory in the last team-executor run (int32 array)."""
    k = np.zeros(ngraphs, np.int32)
    _check(load().hf_batch_team_keys(b, k.ctypes.data), "hf_batch_team_keys")
    return k


def hf_calibration(stream=None):
    """(level-sync ns/level, persistent ns/hop, team ns/level on one CTA, on a cluster,
    host link GB/s host to device, device to host, both directions at once,
    ns per in-edge gathered on one SM: level-sync, team on one CTA, team on a cluster)."""
    out = np.zeros(10, np.float32)
    _check(load().hf_calibration(_stream_handle(stream), out.ctypes.data), "hf_calibration")
    return tuple(float(x) for x in out)


def hf_place(g, n_tasks, ndev, cost=None):
    """Device of each task (int32 array; -1 for host tasks)."""
    out = np.empty(n_tasks, np.int32)
    c = None if cost is None else np.ascontiguousarray(cost, np.float32)
    _check(load().hf_place(g, ndev, None if c is None else c.ctypes.data, out.ctypes.data), "hf_place")
    return out


def hf_batch_partition(b, n_graphs, ndev):
    """(device of each graph, load of each device)."""
    dev = np.empty(n_graphs, np.int32)
    loads = np.empty(ndev, np.float64)
    _check(load().hf_batch_partition(b, ndev, dev.ctypes.data, loads.ctypes.data), "hf_batch_partition")
    return dev, loads


def hf_dump(g, path):
    _check(load().hf_dump(g, os.fsencode(path)), "hf_dump")


def hf_run_n(g, n, stream=None, opts=None):
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_run_n(g, _stream_handle(stream), ctypes.byref(o), n), "hf_run_n")


def hf_batch_run_n(b, n, stream=None, opts=None):
    o = opts if opts is not None else hf_run_opts_default()
    _check(load().hf_batch_run_n(b, _stream_handle(stream), ctypes.byref(o), n), "hf_batch_run_n")


def _run_until(fn, obj, pred, max_runs, stream, opts, where):
    o = opts if opts is not None else hf_run_opts_default()
    cb = PRED_FN(lambda ctx: 1 if pred() else 0)
    runs = ctypes.c_int32()
    _check(fn(obj, _stream_handle(stream), ctypes.byref(o), cb, None, max_runs, ctypes.byref(runs)), where)
    return runs.value


def hf_run_until(g, pred, max_runs, stream=None, opts=None):
    """Runs until pred() (a Python callable, called after each completed run) is true or
    max_runs runs completed; returns the number of runs."""
    return _run_until(load().hf_run_until, g, pred, max_runs, stream, opts, "hf_run_until")


def hf_batch_run_until(b, pred, max_runs, stream=None, opts=None):
    return _run_until(load().hf_batch_run_until, b, pred, max_runs, stream, opts, "hf_batch_run_until")


STAT_NAMES = ["rounds", "items", "idle", "edges", "cas", "push_local", "push_global", "claims", "pops", "pieces",
              "cyc_round", "cyc_release", "cyc_cas", "cyc_push", "push_ring", "steals"]


def hf_batch_get_stats(b):
    out = np.zeros(16, np.int64)
    _check(load().hf_batch_get_stats(b, _ptr(out), 16), "hf_batch_get_stats")
    return {nm: int(out[i]) for i, nm in enumerate(STAT_NAMES)}


HF_NOALLOC_MAX_TASKS = 1048576


def hf_run_csr_noalloc(n_tasks, n_edges, row_ptr, succ, delay, arr0, arr, spin_limit_ns=0, stream=None):
    """Arrivals of one max-plus graph given as a successor CSR, with no allocation by the
    library (its scratch is a fixed device array). row_ptr (int32, n_tasks + 1), succ (int32),
    delay (float32), arr0 (float32 or None) and arr (float32, written) are device buffers the
    caller owns (CUDA tensors or raw addresses). Blocks until the result is in arr."""
    _check(load().hf_run_csr_noalloc(n_tasks, n_edges, _ptr(row_ptr), _ptr(succ), _ptr(delay), _ptr(arr0),
                                     _ptr(arr), spin_limit_ns, _stream_handle(stream)), "hf_run_csr_noalloc")


def opts_dict(o):
    return {k: getattr(o, k) for k, _ in hf_run_opts._fields_ if not k.endswith("_")}


def hf_status_string(s):
    return load().hf_status_string(s).decode()


def hf_last_error():
    return load().hf_last_error().decode(errors="replace")
