"""GPU tests of the team executor's payload ordering on thread-block clusters.

A cluster level releases the payload stores of its tasks only where another payload task of the
graph can observe them: the library checks the payloads' memory ranges on the host and, when no
payload touches memory another one writes, the level's barrier releases the arrival keys alone.
Both cases, against exact expectations:

* a chain of saxpy tasks updating one shared y buffer (each after the one before, through
  dependency edges): every update must see the previous one, whichever CTA ran its pieces;
* saxpy tasks on private buffers only (the relaxed barrier): every buffer and every arrival.

Values are small integers and halves, so y = a*x + y is exact in FP32 with or without a fused
multiply-add, and the expected buffers are computed in float64.
"""
import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEVELS, WIDTH, N_SAX = 30, 200, 6000  # a saxpy of 6,000 elements is 12 pieces of 512


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.install_torch_allocator()


def _build(shared, seed):
    """LEVELS levels of WIDTH max-plus tasks plus three saxpy tasks; saxpy 0 of every level
    updates y_shared (shared=True, each after the previous level's) or a buffer of its own."""
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda")
    xs = [torch.tensor(rng.integers(-8, 9, N_SAX).astype(np.float32), device=dev) for _ in range(3 * LEVELS)]
    y_shared = torch.tensor(rng.integers(-100, 101, N_SAX).astype(np.float32), device=dev)
    ys = [torch.tensor(rng.integers(-100, 101, N_SAX).astype(np.float32), device=dev) for _ in range(3 * LEVELS)]
    a = rng.choice(np.array([0.5, 2.0, -1.0], np.float32), 3 * LEVELS)
    g = hf.hf_graph_create()
    ids = np.zeros((LEVELS, WIDTH + 3), np.int64)
    for lv in range(LEVELS):
        first = hf.hf_add_tasks_bulk(g, WIDTH)
        ids[lv, :WIDTH] = np.arange(first, first + WIDTH)
        for j in range(3):
            q = 3 * lv + j
            y = y_shared if (shared and j == 0) else ys[q]
            p = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=float(a[q]), n=N_SAX, x_pull=-1, y_pull=-1,
                                    x_dev=xs[q].data_ptr(), y_dev=y.data_ptr())
            ids[lv, WIDTH + j] = hf.hf_add_task(g, hf.HF_KERNEL, p)
    src, dst = [], []
    for lv in range(1, LEVELS):
        for i in range(WIDTH + 3):
            v = int(ids[lv, i])
            preds = {int(ids[lv - 1, rng.integers(0, WIDTH + 3)])}
            for _ in range(int(rng.integers(0, 3))):
                preds.add(int(ids[rng.integers(0, lv), rng.integers(0, WIDTH + 3)]))
            if i == WIDTH:  # saxpy 0 after the previous level's saxpy 0 (the shared buffer's order)
                preds.add(int(ids[lv - 1, WIDTH]))
            src.extend(preds)
            dst.extend([v] * len(preds))
    src, dst = np.asarray(src, np.int32), np.asarray(dst, np.int32)
    delay = rng.uniform(0.01, 1.0, src.size).astype(np.float32)
    hf.hf_precede_bulk(g, src, dst, delay)
    n = LEVELS * (WIDTH + 3)
    spec = S.GraphSpec(name="payload_order", n=n, src=src, dst=dst, delay=delay, kind=np.zeros(n, np.uint8))
    # expected buffers: float64 of exact values
    x64 = [x.cpu().numpy().astype(np.float64) for x in xs]
    want_shared = y_shared.cpu().numpy().astype(np.float64)
    want = [y.cpu().numpy().astype(np.float64) for y in ys]
    for lv in range(LEVELS):
        for j in range(3):
            q = 3 * lv + j
            if shared and j == 0:
                want_shared = float(a[q]) * x64[q] + want_shared
            else:
                want[q] = float(a[q]) * x64[q] + want[q]
    start = [y_shared.clone()] + [y.clone() for y in ys]
    # the graph borrows every x and y buffer: the caller keeps them alive while it runs
    return g, spec, (y_shared, ys, xs), (want_shared, want), start


@pytest.mark.parametrize("shared", [True, False])
@pytest.mark.parametrize("opts", [dict(team_size=2), dict(team_size=4), dict(team_size=8),
                                  dict(team_size=4, chunk_elems=256), dict()])
def test_cluster_payload_order(shared, opts):
    g, spec, (y_shared, ys, xs), (want_shared, want), start = _build(shared, 11 if shared else 12)
    ref = oracle.run_spec(spec, with_data=False)["arr"].view(np.uint32)
    for _ in range(2):  # the same result again from the same starting buffers
        y_shared.copy_(start[0])
        for y, s0 in zip(ys, start[1:]):
            y.copy_(s0)
        torch.cuda.synchronize()
        hf.hf_run(g, None, hf.hf_run_opts_default(mode=hf.HF_MODE_TEAM, **opts))
        hf.hf_sync_status(g)
        torch.cuda.synchronize()
        if shared:
            np.testing.assert_array_equal(y_shared.cpu().numpy(), want_shared.astype(np.float32), err_msg=str(opts))
        for q, y in enumerate(ys):
            if shared and q % 3 == 0:
                continue  # (unused: saxpy 0 updates the shared buffer)
            np.testing.assert_array_equal(y.cpu().numpy(), want[q].astype(np.float32), err_msg="%s %d" % (opts, q))
        arr = hf.hf_get_arrivals(g, spec.n)
        np.testing.assert_array_equal(arr.view(np.uint32), ref, err_msg=str(opts))
    hf.hf_graph_destroy(g)
    del xs


def _chain(bufs_x, bufs_y, a, extra=None):
    """One saxpy task per level (y_l = a_l * x_l + y_l), each after the one before, beside 50
    max-plus tasks per level; extra(g, ids) may add tasks. Returns (graph, task ids)."""
    g = hf.hf_graph_create()
    ids = []
    prev = None
    for lv, (x, y) in enumerate(zip(bufs_x, bufs_y)):
        m = hf.hf_add_tasks_bulk(g, 50)
        p = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=float(a[lv]), n=int(y.numel()), x_pull=-1, y_pull=-1,
                                x_dev=x.data_ptr(), y_dev=y.data_ptr())
        s = hf.hf_add_task(g, hf.HF_KERNEL, p)
        if prev is not None:
            for t in list(range(m, m + 50)) + [s]:
                hf.hf_precede(g, prev, t)
        prev = s
        ids.append(s)
    if extra:
        extra(g, ids)
    return g, ids


def test_payload_local_classification_and_overlapping_views():
    """The host check behind the relaxed cluster barrier, through hf_batch_team_flags: private
    buffers qualify; a shared y, overlapping views of one buffer, one task's y read as another's
    x, and a graph with a host task do not. The overlapping-view chain also runs exactly on
    clusters (each update sees the one before)."""
    rng = np.random.default_rng(21)
    dev = torch.device("cuda")
    L, n = 12, 4000
    a = rng.choice(np.array([0.5, 2.0, -1.0], np.float32), L)

    def tens(k):
        return [torch.tensor(rng.integers(-8, 9, n).astype(np.float32), device=dev) for _ in range(k)]

    keep = []
    xs_p, ys_p = tens(L), tens(L)  # private
    base = torch.tensor(rng.integers(-50, 51, (L + 1) * n // 2).astype(np.float32), device=dev)
    ys_v = [base[lv * n // 2: lv * n // 2 + n] for lv in range(L)]  # each overlaps the next by half
    xs_v = tens(L)
    ys_r, xs_r = tens(L), None  # task l reads task l-1's y as its x
    xs_r = [tens(1)[0]] + [ys_r[lv - 1] for lv in range(1, L)]
    xs_h, ys_h = tens(L), tens(L)
    calls = []
    host_fn = hf.HOST_FN(lambda arg: calls.append(1))
    keep += [host_fn]

    def add_host(g, ids):
        h = hf.hf_add_task(g, hf.HF_HOST, hf.hf_host_payload(fn=host_fn, arg=None))
        hf.hf_precede(g, ids[-1], h)

    start_v = base.clone()
    graphs = [_chain(xs_p, ys_p, a)[0], _chain(xs_v, ys_v, a)[0], _chain(xs_r, ys_r, a)[0],
              _chain(xs_h, ys_h, a, add_host)[0]]
    b = hf.hf_batch_create()
    for g in graphs:
        hf.hf_batch_add(b, g)
    # expected overlapping-view result: the updates in chain order, float64 of exact values
    want = start_v.cpu().numpy().astype(np.float64)
    for lv in range(L):
        lo = lv * n // 2
        want[lo:lo + n] = float(a[lv]) * xs_v[lv].cpu().numpy().astype(np.float64) + want[lo:lo + n]
    for ts in (2, 4):
        base.copy_(start_v)
        torch.cuda.synchronize()
        hf.hf_batch_run(b, None, hf.hf_run_opts_default(mode=hf.HF_MODE_TEAM, team_size=ts))
        hf.hf_batch_sync_status(b)
        torch.cuda.synchronize()
        flags = hf.hf_batch_team_flags(b, len(graphs))
        local = [(int(f) & hf.TEAM_PAYLOAD_LOCAL) != 0 for f in flags]
        assert local == [True, False, False, False], (ts, flags)
        assert all((int(f) & hf.TEAM_PIPELINED) == 0 for f in flags)  # (small graphs)
        np.testing.assert_array_equal(base.cpu().numpy(), want.astype(np.float32), err_msg=str(ts))
    hf.hf_batch_destroy(b)
    for g in graphs:
        hf.hf_graph_destroy(g)
    del keep, xs_p, ys_p, xs_v, ys_v, xs_r, ys_r, xs_h, ys_h
