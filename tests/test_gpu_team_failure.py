"""The team executor's failure path, injected on the host (no GPU fault).

A run reports completion or failure through its status (the paper's Section III-B: a run's
future). Here one host-task callback sleeps far longer than the run's spin limit. The team
that posted it must give up after about one limit with HF_ETIMEDOUT, every CTA of that team
leaving together (solo CTAs and thread-block clusters alike), and the run must abort: no new
job starts, and no other level waits out a limit of its own. The next run on the same context
must then be bit-exact against the oracle.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIMIT_NS = 20_000_000  # 20 ms
SLEEP_S = 1.5          # the stuck callback


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    hf.install_torch_allocator()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _batch(n_graphs, levels, per_level):
    """Layered graphs with one host task in each of their first `levels` levels."""
    calls = []
    stuck = {"task": None}
    lock = threading.Lock()
    keep, graphs, specs = [], [], []
    b = hf.hf_batch_create()
    for gi in range(n_graphs):
        n, lv, src, dst, dly = S.layered_dag(300 + gi, per_level * levels, levels, 1, 3)
        host_ids = set(l * per_level + (gi * 7 + l) % per_level for l in range(levels))  # level l = ids [l*w, (l+1)*w)
        g = hf.hf_graph_create()
        for v in range(n):
            if v in host_ids:
                def fn(arg, gi=gi, v=v):
                    with lock:
                        calls.append((gi, v))
                    if stuck["task"] == (gi, v):
                        time.sleep(SLEEP_S)
                f = hf.HOST_FN(fn)
                keep.append(f)
                hf.hf_add_task(g, hf.HF_HOST, hf.hf_host_payload(fn=f, arg=None))
            else:
                hf.hf_add_task(g, hf.HF_KERNEL, None)
        hf.hf_precede_bulk(g, src, dst, dly)
        hf.hf_batch_add(b, g)
        graphs.append(g)
        specs.append(S.GraphSpec(name="t%d" % gi, n=n, src=src, dst=dst, delay=dly, kind=np.zeros(n, np.uint8)))
    return b, graphs, specs, calls, stuck, keep


@pytest.mark.parametrize("team_size", [1, 2, 4])
def test_stuck_host_task_times_out_the_team_run(team_size):
    levels, width = 40, 100
    b, graphs, specs, calls, stuck, keep = _batch(3, levels, width)
    opts = dict(mode=hf.HF_MODE_TEAM, team_size=team_size, spin_limit_ns=LIMIT_NS, time_kernel=1)
    # a clean run first: every host task once, arrivals exact
    hf.hf_batch_run(b, None, hf.hf_run_opts_default(**opts))
    assert hf.hf_batch_sync_status(b, False) == hf.HF_OK
    assert len(calls) == 3 * levels
    # graph 0's host task of level 3 is stuck for SLEEP_S, far beyond the limit
    stuck["task"] = (0, 3 * width + (0 * 7 + 3) % width)
    calls.clear()
    t0 = time.perf_counter()
    hf.hf_batch_run(b, None, hf.hf_run_opts_default(**opts))
    st = hf.hf_batch_sync_status(b, False)
    wall = time.perf_counter() - t0
    assert st == hf.HF_ETIMEDOUT
    # the device gave up after about one limit per team: not one limit for each of the dozens of
    # later host levels (37 x 20 ms for graph 0 alone)
    kms = hf.hf_batch_kernel_ms(b)
    assert kms < 8 * LIMIT_NS / 1e6, kms
    assert wall < SLEEP_S + 2.0, wall  # the proxy thread is joined once the stuck callback returns
    # the run aborted: the teams left before their later levels, so host tasks past the stuck
    # one's level did not all run
    assert len(calls) < 3 * levels
    # the context survives: a clean run afterwards is exact
    stuck["task"] = None
    calls.clear()
    hf.hf_batch_run(b, None, hf.hf_run_opts_default(mode=hf.HF_MODE_TEAM, team_size=team_size))
    assert hf.hf_batch_sync_status(b, False) == hf.HF_OK
    assert sorted(calls) == sorted(set(calls)) and len(calls) == 3 * levels
    for gi, spec in enumerate(specs):
        np.testing.assert_array_equal(bits(hf.hf_batch_get_arrivals(b, gi, spec.n)),
                                      bits(oracle.run_spec(spec)["arr"]))
    hf.hf_batch_destroy(b)
    for g in graphs:
        hf.hf_graph_destroy(g)
    del keep
