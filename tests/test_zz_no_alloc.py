"""The allocation-free entry point hf_run_csr_noalloc against the CPU oracle and hf_run.

Some callers cannot allocate device memory (code inside another framework's memory pool or
under a fixed budget, plug-ins whose host forbids cudaMalloc, loops that cannot afford an
allocation's synchronisation). For them the library exposes hf_run_csr_noalloc, whose scratch
is a fixed device array inside the library. These tests call it through the C ABI several
times in a row -- the array keeps each call's leftovers, so every call must clear what it
reads -- and require the arrival bits of the sequential Kahn oracle and of the regular entry
point (hf_run on a graph built with hf_add_tasks_bulk / hf_precede_bulk), the exact-match bar
of every arrival test here. The file's name makes pytest collect it last; it passes alone in a
fresh process as well.
"""
import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _graph(kind, seed):
    """A seeded max-plus DAG: (n, src, dst, delay, arr0) with signed delays and signed-zero,
    negative and positive source arrivals, so that the whole key order is exercised."""
    rng = np.random.default_rng(seed)
    if kind == "layered":
        n, _, src, dst, dly = S.layered_dag(seed, 20_000, 50, 1, 4)
    else:
        n, _, src, dst, dly = S.random_dag(seed, 60_000, 1, 6, window=256)
    dly = rng.normal(0.0, 2.0, dly.size).astype(np.float32)
    dly[rng.random(dly.size) < 0.05] = -0.0
    arr0 = rng.choice(np.array([0.0, -0.0, 1.5, -3.25], np.float32), n).astype(np.float32)
    return n, src.astype(np.int32), dst.astype(np.int32), dly, arr0


def _csr(n, src, dst, dly):
    order = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return row_ptr.astype(np.int32), dst[order].astype(np.int32), dly[order].astype(np.float32)


def _hf_run_arrivals(n, src, dst, dly, arr0, mode):
    g = hf.hf_graph_create(n, src.size)
    try:
        hf.hf_add_tasks_bulk(g, n, arr0)
        hf.hf_precede_bulk(g, src, dst, dly)
        hf.hf_run(g, opts=hf.hf_run_opts_default(mode=mode))
        hf.hf_sync_status(g)
        return hf.hf_get_arrivals(g, n).copy()
    finally:
        hf.hf_graph_destroy(g)


def test_rejects_sizes_beyond_the_static_limit():
    """Host-side checks, before any CUDA call (runs without a GPU)."""
    B.build()
    with pytest.raises(hf.HfError) as e:
        hf.hf_run_csr_noalloc(hf.HF_NOALLOC_MAX_TASKS + 1, 0, 16, 16, 16, None, 16, stream=0)
    assert e.value.status == hf.HF_EINVAL and "1048576" in str(e.value)
    with pytest.raises(hf.HfError) as e:
        hf.hf_run_csr_noalloc(-1, 0, 16, 16, 16, None, 16, stream=0)
    assert e.value.status == hf.HF_EINVAL
    with pytest.raises(hf.HfError) as e:
        hf.hf_run_csr_noalloc(4, 3, None, 16, 16, None, 16, stream=0)
    assert e.value.status == hf.HF_EINVAL
    hf.hf_run_csr_noalloc(0, 0, None, None, None, None, None, stream=0)  # empty graph: nothing to do


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_hf_run_on_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    graphs = {k: _graph(k, 31 + i) for i, k in enumerate(("layered", "random"))}
    expect, dev, oracle_arr = {}, {}, {}
    for k, (n, src, dst, dly, arr0) in graphs.items():
        oracle_arr[k] = oracle.kahn(n, src, dst, dly, arr0)[0]
        expect[k] = _hf_run_arrivals(n, src, dst, dly, arr0, hf.HF_MODE_PERSISTENT)
        np.testing.assert_array_equal(bits(_hf_run_arrivals(n, src, dst, dly, arr0, hf.HF_MODE_LEVELSYNC)),
                                      bits(expect[k]))
        row_ptr, succ, d = _csr(n, src, dst, dly)
        dev[k] = (n, succ.size, *(torch.from_numpy(a).cuda() for a in (row_ptr, succ, d, arr0)))
    stream = torch.cuda.current_stream()
    # the same graph twice in a row, then a larger graph, then the first again: each call must
    # clear the leftovers of the one before
    for k in ("layered", "layered", "random", "layered"):
        n, m, row_ptr, succ, d, arr0 = dev[k]
        arr = torch.full((n,), float("nan"), device="cuda")
        hf.hf_run_csr_noalloc(n, m, row_ptr, succ, d, arr0, arr, stream=stream)
        got = bits(arr.cpu().numpy())
        np.testing.assert_array_equal(got, bits(expect[k]))
        np.testing.assert_array_equal(got, bits(oracle_arr[k]))


@pytest.mark.gpu
def test_noalloc_reads_arr0_of_sources_only():
    """arr0 entries of tasks with predecessors are never read: NaN there changes nothing, while
    a NaN source arrival is rejected with HF_EINVAL."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    n, src, dst, dly, arr0 = _graph("layered", 47)
    ref = oracle.kahn(n, src, dst, dly, arr0)[0]
    has_pred = np.zeros(n, bool)
    has_pred[dst] = True
    junk = arr0.copy()
    junk[has_pred] = np.nan
    row_ptr, succ, d = _csr(n, src, dst, dly)
    dv = [torch.from_numpy(a).cuda() for a in (row_ptr, succ, d, junk)]
    stream = torch.cuda.current_stream()
    arr = torch.full((n,), float("nan"), device="cuda")
    hf.hf_run_csr_noalloc(n, succ.size, *dv, arr, stream=stream)
    np.testing.assert_array_equal(bits(arr.cpu().numpy()), bits(ref))
    bad = junk.copy()
    bad[np.flatnonzero(~has_pred)[0]] = np.nan
    with pytest.raises(hf.HfError) as e:
        hf.hf_run_csr_noalloc(n, succ.size, *dv[:3], torch.from_numpy(bad).cuda(), arr, stream=stream)
    assert e.value.status == hf.HF_EINVAL
    # and the next call is exact again
    hf.hf_run_csr_noalloc(n, succ.size, *dv, arr, stream=stream)
    np.testing.assert_array_equal(bits(arr.cpu().numpy()), bits(ref))
