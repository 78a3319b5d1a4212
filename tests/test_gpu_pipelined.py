"""GPU parity of the team executor's software-pipelined levels (jobs of graphs with at least
32,768 tasks): a thread reads its next level's task during the current level's gather and issues
its first eight key loads first thing in the next level. The cases the pipelining has to get
right, on one CTA and on clusters, with keys in global and in distributed shared memory, alone
and in a batch, against the oracle bit for bit:

* tasks with more than eight in-edges (the loads issued early cover eight, the rest follow);
* levels that alternate between fitting the stage buffers and being too wide to stage (the
  read-ahead is taken only where the next level was staged and has landed);
* signed delays (including -0) and source arrivals of every sign (the key order end to end).
"""
import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S
from paper_2203_08395_b300.workload import BatchOnDevice, GraphOnDevice

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PIPE_MIN_TASKS = 32768  # graphs from this size on run pipelined (kPipeMinTasks in the library)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.install_torch_allocator()


def _levels_graph(seed, widths, fin_hi, name):
    """Level l has widths[l] tasks; each task past level 0 takes 1..fin_hi distinct predecessors,
    the first in the level before, the others anywhere earlier. Signed delays, some -0, and
    source arrivals of both signs."""
    rng = np.random.default_rng(seed)
    first = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
    src, dst = [], []
    for lv in range(1, len(widths)):
        lo, hi = int(first[lv]), int(first[lv + 1])
        for v in range(lo, hi):
            k = int(rng.integers(1, fin_hi + 1))
            preds = {int(rng.integers(first[lv - 1], first[lv]))}
            while len(preds) < min(k, lo):
                preds.add(int(rng.integers(0, lo)))
            src.extend(preds)
            dst.extend([v] * len(preds))
    n, m = int(first[-1]), len(src)
    delay = rng.normal(0.0, 2.0, m).astype(np.float32)
    delay[rng.random(m) < 0.03] = -0.0
    arr0 = rng.choice(np.array([0.0, -0.0, 1.5, -4.0], np.float32), n)
    order = rng.permutation(m)  # edges in no particular order
    return S.GraphSpec(name=name, n=n, src=np.asarray(src, np.int32)[order], dst=np.asarray(dst, np.int32)[order],
                       delay=delay[order], kind=np.zeros(n, np.uint8), arr0=arr0)


@pytest.fixture(scope="module")
def graphs():
    # 200 levels of 200 tasks, up to 12 in-edges a task: every level staged
    wide_joins = _levels_graph(71, [200] * 200, 12, "wide_joins")
    # 80 levels: four of 250 tasks, then one of 1,200 (too wide to stage), and again
    mixed_fit = _levels_graph(72, ([250] * 4 + [1200]) * 16, 10, "mixed_fit")
    for g in (wide_joins, mixed_fit):
        assert g.n >= PIPE_MIN_TASKS
    counts = np.bincount(wide_joins.dst, minlength=wide_joins.n)
    assert (counts > 8).sum() > 1000 and counts.max() == 12
    return [wide_joins, mixed_fit]


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


@pytest.mark.parametrize("opts", [dict(team_size=1), dict(team_size=2), dict(team_size=4),
                                  dict(team_size=4, team_global_keys=1), dict(team_size=16, team_global_keys=1),
                                  dict(priority=hf.HF_PRIO_HEURISTIC)])
def test_pipelined_levels_single_graph(graphs, opts):
    for spec in graphs:
        ref = _bits(oracle.run_spec(spec)["arr"])
        gd = GraphOnDevice(spec)
        for _ in range(2):  # a second run on the same state gives the same bits
            gd.run(mode=hf.HF_MODE_TEAM, **opts)
            gd.sync()
            np.testing.assert_array_equal(_bits(gd.arrivals()), ref, err_msg="%s %s" % (spec.name, opts))
        gd.close()


@pytest.mark.parametrize("opts", [dict(priority=hf.HF_PRIO_HEURISTIC), dict(team_size=1), dict(team_size=8)])
def test_pipelined_levels_in_a_batch(graphs, opts):
    # the two pipelined graphs beside small ones that run the plain loop, in one launch
    small = [S.layered(80 + i, 3000 + 700 * i, 15, 1, 6) for i in range(6)]
    wl = S.Workload("pipelined_batch", graphs + small)
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, **opts)
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(_bits(bd.arrivals(i)), _bits(oracle.run_spec(spec)["arr"]),
                                      err_msg="%s %s" % (spec.name, opts))
    bd.close()
