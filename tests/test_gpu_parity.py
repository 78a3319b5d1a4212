"""GPU parity: both executors against the CPU oracle, through the C ABI, bit for bit.

Arrivals must match exactly (each sum has fixed inputs and max is exact, so every schedule
gives the oracle's bits); saxpy and copy results must match exactly (fmaf on both sides).
Covers the paper's worked examples (Section I saxpy graph, Section III-A eight-task graph),
every workload shape at sizes the oracle finishes in seconds, the full-size workloads, edge
cases (empty, single task, deep chain, wide fan-out/fan-in, ragged payload pieces) and the
bounded-wait failure path.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S
from paper_2203_08395_b300.workload import BatchOnDevice, GraphOnDevice

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EXECUTORS = {
    "levelsync": dict(mode=hf.HF_MODE_LEVELSYNC),
    "persistent": dict(mode=hf.HF_MODE_PERSISTENT),
    "persistent_claim8": dict(mode=hf.HF_MODE_PERSISTENT, claim=8),
    "persistent_nolocal": dict(mode=hf.HF_MODE_PERSISTENT, local_keep=0),
    "persistent_1cta": dict(mode=hf.HF_MODE_PERSISTENT, ctas=1),
    "persistent_wide": dict(mode=hf.HF_MODE_PERSISTENT, ctas=148 * 8, claim=4),
    "persistent_payw2": dict(mode=hf.HF_MODE_PERSISTENT, payload_warps=2, claim=8, local_keep=8),
    "persistent_payw7": dict(mode=hf.HF_MODE_PERSISTENT, payload_warps=7, ctas=16),
    # work stealing: per-CTA rings; small rings overflow to the global queue, few CTAs steal a lot
    "steal": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=4096),
    "steal_small": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=64, claim=4),
    "steal_2cta": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=64, ctas=2),
    "steal_1cta": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=128, ctas=1),
    "steal_payw2": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=256, payload_warps=2),
    # copy warps: pulls and pushes from queues of their own (one or two warps per CTA and direction)
    "persistent_copyw1": dict(mode=hf.HF_MODE_PERSISTENT, copy_warps=1),
    "persistent_copyw2_payw2": dict(mode=hf.HF_MODE_PERSISTENT, copy_warps=2, payload_warps=2, claim=4),
    "steal_copyw1": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=128, copy_warps=1, ctas=6),
    "team": dict(mode=hf.HF_MODE_TEAM),
    "team_heur": dict(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC),
    "team_k2": dict(mode=hf.HF_MODE_TEAM, team_size=2),
    "team_k5": dict(mode=hf.HF_MODE_TEAM, team_size=5, ctas=12),
    # every key in global memory (the default keeps a graph's keys in shared memory where they fit)
    "team_global_keys": dict(mode=hf.HF_MODE_TEAM, team_global_keys=1),
    "team_k4_global_keys": dict(mode=hf.HF_MODE_TEAM, team_size=4, team_global_keys=1),
    # one launch: graphs on 8-CTA clusters (or the planner's cluster size) and single CTAs together
    "team_fold8": dict(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC, team_fold=8, team_scale=1),
    "team_fold_auto": dict(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC, team_fold=-1),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    hf.install_torch_allocator()
    torch.cuda.init()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _run(gd, **opts):
    gd.run(**opts)
    gd.sync()
    return gd.arrivals()


@pytest.mark.parametrize("ex", sorted(EXECUTORS))
def test_layered10k_bit_exact(ex):
    spec = S.config("layered10k").graphs[0]
    ref = oracle.run_spec(spec)["arr"]
    gd = GraphOnDevice(spec)
    np.testing.assert_array_equal(bits(_run(gd, **EXECUTORS[ex])), bits(ref))
    # a second run gives the same bits
    np.testing.assert_array_equal(bits(_run(gd, **EXECUTORS[ex])), bits(ref))
    gd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "persistent_claim8", "steal_small", "team", "team_k5",
                                "team_fold_auto"])
def test_random_graphs_100_seeds(ex):
    rng = np.random.default_rng(5)
    for seed in range(100):
        n = int(rng.integers(1, 3000))
        win = int(rng.choice([0, 4, 64]))
        n_, _, src, dst, dly = S.random_dag(seed, n, 1, int(rng.integers(1, 9)), window=win)
        # signed delays and signed-zero source arrivals exercise the full key order
        if seed % 3 == 0:
            dly = rng.normal(0, 3, dly.size).astype(np.float32)
            dly[rng.random(dly.size) < 0.05] = -0.0
        arr0 = rng.choice([0.0, -0.0, 2.5, -7.0], n_).astype(np.float32) if seed % 2 else None
        spec = S.GraphSpec(name="r%d" % seed, n=n_, src=src, dst=dst, delay=dly,
                           kind=np.zeros(n_, np.uint8), arr0=arr0)
        ref = oracle.run_spec(spec)["arr"]
        gd = GraphOnDevice(spec)
        np.testing.assert_array_equal(bits(_run(gd, **EXECUTORS[ex])), bits(ref), err_msg="seed %d" % seed)
        gd.close()


def _permuted(spec, seed):
    """The same graph under a random relabelling of its task ids and a random order of its
    edges: predecessors no longer have lower ids (the generators draw them from lower ids),
    and each task's successor list comes in another order. Saxpy tasks keep their buffers."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(spec.n).astype(np.int32)  # old id -> new id
    eo = rng.permutation(spec.m)
    kind = np.empty_like(spec.kind)
    kind[perm] = spec.kind
    arr0 = None
    if spec.arr0 is not None:
        arr0 = np.empty_like(spec.arr0)
        arr0[perm] = spec.arr0
    ps = S.GraphSpec(name=spec.name + "_perm", n=spec.n, src=perm[spec.src][eo], dst=perm[spec.dst][eo],
                     delay=spec.delay[eo], kind=kind, sx_task=perm[spec.sx_task] if spec.sx_task.size else spec.sx_task,
                     sx_n=spec.sx_n, sx_a=spec.sx_a, sx_pull=spec.sx_pull, arr0=arr0, data_seed=spec.data_seed)
    return ps, perm


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "persistent_payw2", "steal_small", "team", "team_heur",
                                "team_k5"])
def test_permuted_ids(ex):
    """Layered, circuit-like and random DAGs (and a layered graph with saxpy tasks) with their
    task ids relabelled at random: arrivals and saxpy results are the oracle's."""
    rng = np.random.default_rng(3)
    specs = [S.layered(41, 20_000, 60, 1, 5), S.circuit(42, 40_000, 80), S.mixed(43, n=15_000, nmin=1, nmax=3000, n_copy=0,
                                                                              window=64)]
    n_, _, src, dst, dly = S.random_dag(44, 25_000, 1, 6, window=128)
    dly = rng.normal(0, 3, dly.size).astype(np.float32)
    specs.append(S.GraphSpec(name="signed", n=n_, src=src, dst=dst, delay=dly, kind=np.zeros(n_, np.uint8),
                             arr0=rng.choice([0.0, -0.0, 2.5, -7.0], n_).astype(np.float32)))
    for k, spec in enumerate(specs):
        ps, perm = _permuted(spec, 100 + k)
        ref = oracle.run_spec(ps)
        # relabelling moves every arrival with its task and changes none
        np.testing.assert_array_equal(bits(ref["arr"])[perm], bits(oracle.run_spec(spec, with_data=False)["arr"]))
        gd = GraphOnDevice(ps)
        np.testing.assert_array_equal(bits(_run(gd, chunk_elems=256, **EXECUTORS[ex])), bits(ref["arr"]),
                                      err_msg=ps.name)
        _check_payloads(gd, ref)
        gd.close()


@pytest.mark.parametrize("ex", ["persistent", "steal", "steal_2cta"])
def test_validate_exactly_once_and_order(ex):
    spec = S.circuit(1, 200_000, 400)
    gd = GraphOnDevice(spec)
    gd.run(validate=1, **EXECUTORS[ex])
    gd.sync()
    s0, s1, cnt = hf.hf_get_stamps(gd.g, spec.n)
    assert np.all(cnt == 1)
    assert np.all(s0 >= 0) and np.all(s0 < s1)
    assert np.all(s1[spec.src] < s0[spec.dst])
    np.testing.assert_array_equal(bits(gd.arrivals()), bits(oracle.run_spec(spec)["arr"]))
    gd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "persistent_claim8", "steal", "team_heur", "team_k5"])
def test_circuit1m_full_size(ex):
    spec = S.config("circuit1m").graphs[0]
    ref = oracle.run_spec(spec)["arr"]
    gd = GraphOnDevice(spec)
    np.testing.assert_array_equal(bits(_run(gd, **EXECUTORS[ex])), bits(ref))
    gd.close()


def _check_payloads(gd, ref):
    spec = gd.spec
    for j in range(spec.sx_task.size):
        np.testing.assert_array_equal(gd.y_of(j).cpu().numpy().view(np.uint32), ref["y"][j].view(np.uint32),
                                      err_msg="saxpy %d" % j)
    for i in range(spec.ps_task.size):
        np.testing.assert_array_equal(gd.push_of(i).numpy().view(np.uint32), ref["push"][i].view(np.uint32),
                                      err_msg="push %d" % i)


@pytest.mark.parametrize("chunk", [0, 64, 4096])
@pytest.mark.parametrize("ex", ["levelsync", "persistent", "persistent_claim8", "persistent_payw2", "persistent_payw7",
                                "persistent_copyw1", "persistent_copyw2_payw2", "steal", "steal_small", "steal_2cta",
                                "steal_payw2", "steal_copyw1", "team", "team_k2", "team_k5"])
def test_mixed_small_with_payloads(ex, chunk):
    spec = S.mixed(3, n=6000, nmin=1, nmax=20000, n_copy=300)
    ref = oracle.run_spec(spec)
    gd = GraphOnDevice(spec)
    arr = _run(gd, chunk_elems=chunk, **EXECUTORS[ex])
    np.testing.assert_array_equal(bits(arr), bits(ref["arr"]))
    _check_payloads(gd, ref)
    gd.close()


def test_mixed100k_full_size_sampled():
    spec = S.config("mixed100k").graphs[0]
    ref = oracle.run_spec(spec, with_data=False)
    gd = GraphOnDevice(spec)
    rng = np.random.default_rng(0)
    sample = rng.choice(spec.sx_task.size, 64, replace=False)
    for ex in ["levelsync", "persistent", "persistent_copyw1", "steal", "team_heur"]:
        gd.reset_y()
        arr = _run(gd, **EXECUTORS[ex])
        np.testing.assert_array_equal(bits(arr), bits(ref["arr"]))
        for j in sample:
            x = spec.pull_data(j) if spec.sx_pull[j] >= 0 else spec.init_x(j)
            yref = oracle.saxpy_f32(spec.sx_a[j], x, spec.init_y(j))
            np.testing.assert_array_equal(gd.y_of(j).cpu().numpy().view(np.uint32), yref.view(np.uint32))
        for i in range(0, spec.ps_task.size, 50):
            j = int(spec.ps_saxpy[i])
            yref = oracle.saxpy_f32(spec.sx_a[j], spec.pull_data(j), spec.init_y(j))
            np.testing.assert_array_equal(gd.push_of(i).numpy().view(np.uint32), yref.view(np.uint32))
    gd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal", "team", "team_heur", "team_fold8", "team_fold_auto"])
def test_batch256_full_size(ex):
    wl = S.config("batch256")
    bd = BatchOnDevice(wl)
    bd.run(**EXECUTORS[ex])
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        ref = oracle.run_spec(spec)["arr"]
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(ref), err_msg="graph %d" % i)
    bd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "persistent_payw2", "steal_small", "steal_payw2", "team",
                                "team_heur", "team_k2", "team_fold8", "team_fold_auto"])
def test_batch_mixed_small(ex):
    wl = S.batch(2, graphs=12, nmin=500, nmax=20000, frac_saxpy=0.1, sx_min=1, sx_max=3000)
    bd = BatchOnDevice(wl)
    bd.run(chunk_elems=256, **EXECUTORS[ex])
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        ref = oracle.run_spec(spec)
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(ref["arr"]))
        _check_payloads(bd.graphs[i], ref)
    bd.close()


def test_team_plan_reports_team_sizes():
    wl = S.batch(3, graphs=16, nmin=500, nmax=60000, frac_saxpy=0.1)
    bd = BatchOnDevice(wl)
    G = len(wl.graphs)
    with pytest.raises(hf.HfError):
        hf.hf_batch_team_plan(bd.b, G)  # no run yet
    bd.run(mode=hf.HF_MODE_LEVELSYNC)
    bd.sync()
    with pytest.raises(hf.HfError):
        hf.hf_batch_team_plan(bd.b, G)  # no team-executor run yet
    bd.run(mode=hf.HF_MODE_TEAM, team_size=4)
    bd.sync()
    assert (hf.hf_batch_team_plan(bd.b, G) == 4).all()
    bd.run(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC)
    bd.sync()
    k = hf.hf_batch_team_plan(bd.b, G)
    assert set(k.tolist()) <= {1, 2, 4, 8, 16}
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(oracle.run_spec(spec)["arr"]))
    # one launch with 4-CTA clusters: every graph on a 4-CTA cluster or one CTA, a single kernel
    bd.run(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC, team_fold=4, team_scale=1)
    bd.sync()
    k = hf.hf_batch_team_plan(bd.b, G)
    assert set(k.tolist()) <= {1, 4} and hf.hf_batch_last_launches(bd.b) == 1
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(oracle.run_spec(spec)["arr"]))
    bd.close()


# ------------------------------------------------------------------ the paper's examples

def test_paper_saxpy_graph_through_c_abi():
    """Listing 1 / Figure 1: host tasks fill x with 1 and y with 2, pulls copy them to the GPU,
    the int32 kernel computes y = 2x + y, pushes copy both back: every y is 4."""
    from golden_io import load

    gold = load("paper_saxpy_graph.txt")
    P = gold["params"]
    N = P["N"]
    x = torch.zeros(N, dtype=torch.int32, pin_memory=True)
    y = torch.zeros(N, dtype=torch.int32, pin_memory=True)
    host = {"x": x, "y": y}
    fills = {"x": P["x"], "y": P["y"]}
    calls = []

    def make_host(name):
        def fn(arg):
            host[name].fill_(fills[name])
            calls.append(name)
        return hf.HOST_FN(fn)

    g = hf.hf_graph_create()
    ids = {}
    keep = []
    for t in gold["tasks"]:
        nm, kind = t[0], t[1]
        if kind == "host":
            f = make_host(t[2])
            keep.append(f)
            ids[nm] = hf.hf_add_task(g, hf.HF_HOST, hf.hf_host_payload(fn=f, arg=None))
        elif kind == "pull":
            ids[nm] = hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=host[t[2]].data_ptr(), bytes=4 * N))
        elif kind == "saxpy_i32":
            p = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_I32, a_i=P["a"], n=N, x_pull=ids[t[2]], y_pull=ids[t[3]])
            ids[nm] = hf.hf_add_task(g, hf.HF_KERNEL, p)
        elif kind == "push":
            p = hf.hf_push_payload(src_pull=ids[t[2]], host_ptr=host[t[3]].data_ptr(), bytes=4 * N)
            ids[nm] = hf.hf_add_task(g, hf.HF_PUSH, p)
    for a, b in gold["edges"]:
        hf.hf_precede(g, ids[a], ids[b])
    for opts in (dict(mode=hf.HF_MODE_LEVELSYNC), dict(mode=hf.HF_MODE_TEAM), dict(mode=hf.HF_MODE_TEAM, team_size=2),
                 dict(mode=hf.HF_MODE_PERSISTENT), dict(mode=hf.HF_MODE_PERSISTENT, validate=1, chunk_elems=4096),
                 dict(mode=hf.HF_MODE_PERSISTENT, validate=1, copy_warps=1, chunk_elems=4096)):
        x.zero_()
        y.zero_()
        calls.clear()
        hf.hf_run(g, None, hf.hf_run_opts_default(**opts))
        hf.hf_sync_status(g)
        assert sorted(calls) == ["x", "y"], opts
        assert bool((y == P["expect_y"]).all()) and bool((x == P["expect_x"]).all()), opts
        if opts.get("validate"):  # every task once, every edge in order (host tasks included)
            s0, s1, c = hf.hf_get_stamps(g, len(gold["tasks"]))
            assert np.all(c == 1)
            for a, b in gold["edges"]:
                assert s1[ids[a]] < s0[ids[b]], (a, b)
    hf.hf_graph_destroy(g)


@pytest.mark.parametrize("opts", [dict(mode=hf.HF_MODE_TEAM), dict(mode=hf.HF_MODE_TEAM, team_size=4),
                                  dict(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC),
                                  dict(mode=hf.HF_MODE_PERSISTENT), dict(mode=hf.HF_MODE_PERSISTENT, ctas=4),
                                  dict(mode=hf.HF_MODE_PERSISTENT, priority=hf.HF_PRIO_HEURISTIC, payload_warps=2),
                                  dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=256),
                                  dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=64, ctas=4)])
def test_host_tasks_in_a_batch(opts):
    """Host tasks inside a batch run by the team or the persistent executor: each runs exactly
    once, after its predecessors and before its successors (callbacks record the order), and
    every arrival is the oracle's (a host task propagates arrivals like a max-plus task)."""
    rng = np.random.default_rng(21)
    order = []
    keep = []
    b = hf.hf_batch_create()
    graphs, specs = [], []
    for gi in range(4):
        n, _, src, dst, dly = S.layered_dag(100 + gi, 3000 + 500 * gi, 12, 1, 3)
        host_ids = set(int(v) for v in rng.choice(n, 6, replace=False))
        g = hf.hf_graph_create()
        for v in range(n):
            if v in host_ids:
                f = hf.HOST_FN(lambda arg, gi=gi, v=v: order.append((gi, v)))
                keep.append(f)
                hf.hf_add_task(g, hf.HF_HOST, hf.hf_host_payload(fn=f, arg=None))
            else:
                hf.hf_add_task(g, hf.HF_KERNEL, None)
        hf.hf_precede_bulk(g, src, dst, dly)
        hf.hf_batch_add(b, g)
        graphs.append((g, n, src, dst, host_ids))
        specs.append(S.GraphSpec(name="h%d" % gi, n=n, src=src, dst=dst, delay=dly, kind=np.zeros(n, np.uint8)))
    for rep in range(2):
        order.clear()
        hf.hf_batch_run(b, None, hf.hf_run_opts_default(**opts))
        hf.hf_batch_sync_status(b)
        assert sorted(order) == sorted((gi, v) for gi, (_, _, _, _, hs) in enumerate(graphs) for v in hs)
        pos = {t: i for i, t in enumerate(order)}
        for gi, (g, n, src, dst, hs) in enumerate(graphs):
            for u, v in zip(src, dst):  # host-to-host dependencies (direct edges) run in order
                if int(u) in hs and int(v) in hs:
                    assert pos[(gi, int(u))] < pos[(gi, int(v))]
            np.testing.assert_array_equal(bits(hf.hf_batch_get_arrivals(b, gi, n)),
                                          bits(oracle.run_spec(specs[gi])["arr"]))
    hf.hf_batch_destroy(b)
    for g, *_ in graphs:
        hf.hf_graph_destroy(g)


@pytest.mark.parametrize("ring,copyw", [(0, 0), (128, 0), (0, 1), (128, 2)])
def test_paper_saxpy_graph_persistent_without_host_tasks(ring, copyw):
    N = 65536
    x = torch.full((N,), 1, dtype=torch.int32, pin_memory=True)
    y = torch.full((N,), 2, dtype=torch.int32, pin_memory=True)
    g = hf.hf_graph_create()
    px = hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=x.data_ptr(), bytes=4 * N))
    py = hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=y.data_ptr(), bytes=4 * N))
    k = hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_I32, a_i=2, n=N, x_pull=px, y_pull=py))
    sx = hf.hf_add_task(g, hf.HF_PUSH, hf.hf_push_payload(src_pull=px, host_ptr=x.data_ptr(), bytes=4 * N))
    sy = hf.hf_add_task(g, hf.HF_PUSH, hf.hf_push_payload(src_pull=py, host_ptr=y.data_ptr(), bytes=4 * N))
    for a, b in [(px, k), (py, k), (k, sx), (k, sy)]:
        hf.hf_precede(g, a, b)
    hf.hf_run(g, None, hf.hf_run_opts_default(mode=hf.HF_MODE_PERSISTENT, chunk_elems=4096, validate=1, steal_ring=ring,
                                              copy_warps=copyw))
    hf.hf_sync_status(g)
    assert bool((y == 4).all()) and bool((x == 1).all())
    s0, s1, c = hf.hf_get_stamps(g, 5)
    assert np.all(c == 1)
    for a, b in [(px, k), (py, k), (k, sx), (k, sy)]:
        assert s1[a] < s0[b]
    hf.hf_graph_destroy(g)


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal_small", "team", "team_k2"])
def test_saxpy_unaligned_and_ragged(ex):
    """Saxpy tasks on device pointers at every 4-byte offset of x and y (shared and different
    16-byte alignment) and every length 0..40 plus longer ragged ones, chained on the same y
    (each task after the previous one on its buffer), against the oracle's saxpy."""
    rng = np.random.default_rng(11)
    cases = [(ox, oy, n) for ox in range(4) for oy in range(4) for n in (0, 1, 2, 3, 5, 7, 13, 31, 40, 517, 1029)]
    xs = [torch.from_numpy(rng.uniform(-1, 1, n + 8).astype(np.float32)).cuda() for _, _, n in cases]
    ys = [torch.from_numpy(rng.uniform(-1, 1, n + 8).astype(np.float32)).cuda() for _, _, n in cases]
    y0 = [y.cpu().numpy().copy() for y in ys]
    g = hf.hf_graph_create()
    ids = []
    for c, (ox, oy, n) in enumerate(cases):
        p = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=float(1.5 + c % 3), n=n, x_pull=-1, y_pull=-1,
                                x_dev=xs[c].data_ptr() + 4 * ox, y_dev=ys[c].data_ptr() + 4 * oy)
        ids.append((hf.hf_add_task(g, hf.HF_KERNEL, p), hf.hf_add_task(g, hf.HF_KERNEL, p)))
        hf.hf_precede(g, ids[-1][0], ids[-1][1])  # the second saxpy on the same y runs after the first
    hf.hf_run(g, None, hf.hf_run_opts_default(chunk_elems=256, **EXECUTORS[ex]))
    hf.hf_sync_status(g)
    for c, (ox, oy, n) in enumerate(cases):
        a = np.float32(1.5 + c % 3)
        x = xs[c].cpu().numpy()[ox:ox + n]
        want = y0[c].copy()
        want[oy:oy + n] = oracle.saxpy_f32(a, x, oracle.saxpy_f32(a, x, want[oy:oy + n]))
        np.testing.assert_array_equal(ys[c].cpu().numpy().view(np.uint32), want.view(np.uint32),
                                      err_msg="case %s" % (cases[c],))
    hf.hf_graph_destroy(g)


def test_paper_dependency_graph_order():
    from golden_io import load

    gold = load("paper_dependency_graph.txt")
    names = [t[0] for t in gold["tasks"]]
    ix = {nm: i for i, nm in enumerate(names)}
    g = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(g, len(names))
    for a, b in gold["edges"]:
        hf.hf_precede_w(g, ix[a], ix[b], 1.0)
    hf.hf_run(g, None, hf.hf_run_opts_default(mode=hf.HF_MODE_PERSISTENT, validate=1))
    hf.hf_sync_status(g)
    s0, s1, c = hf.hf_get_stamps(g, len(names))
    assert np.all(c == 1)
    for a, b in gold["edges"] + gold["reach"]:
        assert s1[ix[a]] < s0[ix[b]]
    arr = hf.hf_get_arrivals(g, len(names))
    assert arr[ix["push2"]] == 4.0 and arr[ix["kernel2"]] == 3.0
    hf.hf_graph_destroy(g)


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal_2cta", "team", "team_k5"])
def test_edge_cases(ex):
    o = EXECUTORS[ex]
    # empty graph
    g = hf.hf_graph_create()
    hf.hf_run(g, None, hf.hf_run_opts_default(**o))
    hf.hf_sync_status(g)
    hf.hf_graph_destroy(g)
    # single task with a source arrival
    g = hf.hf_graph_create()
    hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_maxplus_payload(op=hf.HF_K_MAXPLUS, arr0=-3.5))
    hf.hf_run(g, None, hf.hf_run_opts_default(**o))
    hf.hf_sync_status(g)
    assert hf.hf_get_arrivals(g, 1)[0] == np.float32(-3.5)
    hf.hf_graph_destroy(g)
    rng = np.random.default_rng(1)
    cases = []
    n = 5000  # deep chain
    cases.append((n, np.arange(n - 1), np.arange(1, n), rng.uniform(0, 1, n - 1)))
    n = 5001  # one task fanning out to 5000, then all of them into one sink
    src = np.concatenate([np.zeros(4999), np.arange(1, 5000)])
    dst = np.concatenate([np.arange(1, 5000), np.full(4999, 5000)])
    cases.append((n, src, dst, rng.normal(0, 1, src.size)))
    n = 3000  # duplicate edges and many sources
    src = rng.integers(0, 1500, 20000)
    dst = rng.integers(1500, 3000, 20000)
    cases.append((n, src, dst, rng.uniform(-1, 1, src.size)))
    for n, src, dst, d in cases:
        spec = S.GraphSpec(name="edge", n=n, src=np.asarray(src, np.int32), dst=np.asarray(dst, np.int32),
                           delay=np.asarray(d, np.float32), kind=np.zeros(n, np.uint8))
        gd = GraphOnDevice(spec)
        np.testing.assert_array_equal(bits(_run(gd, **o)), bits(oracle.run_spec(spec)["arr"]))
        gd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal", "team", "auto"])
def test_run_host_edge_cases(ex):
    """hf_run_host / hf_batch_run_host on degenerate inputs: an empty graph, a graph without
    edges (NULL and non-NULL delays), a single task, and a batch mixing them with a chain."""
    o = dict(mode=hf.HF_MODE_AUTO) if ex == "auto" else EXECUTORS[ex]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    g = hf.hf_graph_create()  # empty: nothing to copy either way
    hf.hf_run_host(g, None, None, None, hf.hf_run_opts_default(**o))
    hf.hf_sync_status(g)
    hf.hf_graph_destroy(g)
    g = hf.hf_graph_create()  # one task, no edges
    hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_maxplus_payload(op=hf.HF_K_MAXPLUS, arr0=2.25))
    out = pin(np.zeros(1))
    hf.hf_run_host(g, pin(np.zeros(0)), out, None, hf.hf_run_opts_default(**o))
    hf.hf_sync_status(g)
    assert out[0].item() == 2.25
    hf.hf_graph_destroy(g)
    specs = [S.GraphSpec(name="lone", n=4, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                         delay=np.zeros(0, np.float32), kind=np.zeros(4, np.uint8)),
             S.GraphSpec(name="chain", n=300, src=np.arange(299, dtype=np.int32), dst=np.arange(1, 300, dtype=np.int32),
                         delay=S.uniform_f32(12, 0, 299, -1.0, 1.0), kind=np.zeros(300, np.uint8)),
             S.GraphSpec(name="one", n=1, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                         delay=np.zeros(0, np.float32), kind=np.zeros(1, np.uint8))]
    wl = S.Workload("edge_batch", specs)
    bd = BatchOnDevice(wl)
    new = S.uniform_f32(13, 0, 299, 0.0, 2.0)
    out = pin(np.zeros(wl.n_tasks))
    bd.run_host(pin(new), out, **o)
    bd.sync()
    ref = np.concatenate([oracle.kahn(4, specs[0].src, specs[0].dst, specs[0].delay)[0],
                          oracle.kahn(300, specs[1].src, specs[1].dst, new)[0],
                          oracle.kahn(1, specs[2].src, specs[2].dst, specs[2].delay)[0]])
    np.testing.assert_array_equal(bits(out.numpy()), bits(ref))
    bd.close()


def test_arrivals_on_device():
    spec = S.layered(7, 5000, 20, 1, 4)
    gd = GraphOnDevice(spec)
    gd.run(mode=hf.HF_MODE_PERSISTENT)
    out = torch.empty(spec.n, dtype=torch.float32, device="cuda")
    hf.hf_get_arrivals(gd.g, spec.n, out, on_device=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(bits(out.cpu().numpy()), bits(oracle.run_spec(spec)["arr"]))
    gd.close()


@pytest.mark.parametrize("ring", [0, 256])
def test_stalled_task_times_out_and_context_survives(ring):
    """Failure path without a GPU fault: one task's counter starts one too high, so it never
    becomes ready; the persistent kernel's bounded waits end the run with HF_ETIMEDOUT and the
    next run on the same context is correct (global queue, and work stealing)."""
    spec = S.layered(8, 20000, 40, 1, 4)
    gd = GraphOnDevice(spec)
    gd.run(mode=hf.HF_MODE_PERSISTENT, stall_task=12345, spin_limit_ns=50_000_000, steal_ring=ring)
    assert gd.sync(check=False) == hf.HF_ETIMEDOUT
    gd.run(mode=hf.HF_MODE_PERSISTENT, steal_ring=ring)
    gd.sync()
    np.testing.assert_array_equal(bits(gd.arrivals()), bits(oracle.run_spec(spec)["arr"]))
    gd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal_small", "team_heur"])
def test_new_timing_view_through_set_delays(ex):
    """A second timing view of the same circuit: new delays in place, arrivals as the oracle
    computes them on the new delays; a non-finite delay is reported, then recovered from."""
    wl = S.batch(5, graphs=6, nmin=2000, nmax=20000)
    bd = BatchOnDevice(wl)
    bd.run(**EXECUTORS[ex])
    bd.sync()
    new = [S.uniform_f32(77, i, g.m, -0.5, 2.0) for i, g in enumerate(wl.graphs)]
    allnew = torch.from_numpy(np.concatenate(new)).pin_memory()
    hf.hf_batch_set_delays(bd.b, allnew, on_device=False)
    bd.run(**EXECUTORS[ex])
    bd.sync()
    for i, g in enumerate(wl.graphs):
        ref = oracle.kahn(g.n, g.src, g.dst, new[i])[0]
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(ref))
    bad = allnew.clone()
    bad[12345] = float("nan")
    hf.hf_batch_set_delays(bd.b, bad.cuda(), on_device=True)
    bd.run(**EXECUTORS[ex])
    assert bd.sync(check=False) == hf.HF_EINVAL
    hf.hf_batch_set_delays(bd.b, allnew.cuda(), on_device=True)
    bd.run(**EXECUTORS[ex])
    bd.sync()
    allarr = hf.hf_batch_get_arrivals(bd.b, -1, wl.n_tasks)
    ref_all = np.concatenate([oracle.kahn(g.n, g.src, g.dst, new[i])[0] for i, g in enumerate(wl.graphs)])
    np.testing.assert_array_equal(bits(allarr), bits(ref_all))
    bd.close()


@pytest.mark.parametrize("ex", ["levelsync", "persistent", "steal", "team", "team_heur", "team_k2"])
def test_run_host_streams_timing_views(ex):
    """hf_batch_run_host: delays in from page-locked memory and arrivals out to it, in one call,
    for several timing views in a row (each the oracle's arrivals on its delays); payloads run as
    in hf_batch_run; NULL delays keep the current ones; unpinned buffers are rejected."""
    wl = S.batch(6, graphs=10, nmin=500, nmax=30000, frac_saxpy=0.1, sx_min=1, sx_max=3000)
    bd = BatchOnDevice(wl)
    N = wl.n_tasks
    views = [[S.uniform_f32(91 + v, i, g.m, -0.5, 2.0) for i, g in enumerate(wl.graphs)] for v in range(3)]
    outs = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in views]
    for v, new in enumerate(views):
        dl = torch.from_numpy(np.concatenate(new)).pin_memory()
        bd.run_host(dl, outs[v], chunk_elems=256, **EXECUTORS[ex])
        bd.sync()
        ref = np.concatenate([oracle.kahn(g.n, g.src, g.dst, new[i])[0] for i, g in enumerate(wl.graphs)])
        np.testing.assert_array_equal(bits(outs[v].numpy()), bits(ref), err_msg="view %d" % v)
    # the device keeps the last view: a plain run and a run_host without delays agree with it
    bd.run(chunk_elems=256, **EXECUTORS[ex])
    bd.sync()
    np.testing.assert_array_equal(bits(hf.hf_batch_get_arrivals(bd.b, -1, N)), bits(outs[-1].numpy()))
    again = torch.empty(N, dtype=torch.float32).pin_memory()
    bd.run_host(None, again, **EXECUTORS[ex])
    bd.sync()
    np.testing.assert_array_equal(bits(again.numpy()), bits(outs[-1].numpy()))
    # the other executors see the last view too (the level-sorted in-edges and the persistent
    # executor's edge records both follow it)
    for other in ("persistent", "levelsync", "team"):
        bd.run(chunk_elems=256, **EXECUTORS[other])
        bd.sync()
        np.testing.assert_array_equal(bits(hf.hf_batch_get_arrivals(bd.b, -1, N)), bits(outs[-1].numpy()), err_msg=other)
    with pytest.raises(hf.HfError):
        bd.run_host(np.zeros(wl.n_edges, np.float32), again, **EXECUTORS[ex])  # not page-locked
    with pytest.raises(hf.HfError):
        bd.run_host(None, np.zeros(N, np.float32), **EXECUTORS[ex])
    bd.close()


def test_run_host_pipelined_views_across_executors():
    """Eight timing views enqueued back to back without synchronising (each with its own
    page-locked delay and arrival buffers), the executor changing between views: the copies,
    gathers and runs of consecutive views overlap, and every view's arrivals are the oracle's
    on its own delays."""
    wl = S.batch(8, graphs=12, nmin=500, nmax=40000)
    bd = BatchOnDevice(wl)
    N = wl.n_tasks
    order = ["team", "team", "levelsync", "team", "persistent", "team", "levelsync", "persistent"]
    views = [[S.uniform_f32(131 + v, i, g.m, 0.0, 3.0) for i, g in enumerate(wl.graphs)] for v in range(len(order))]
    ins = [torch.from_numpy(np.concatenate(new)).pin_memory() for new in views]
    outs = [torch.full((N,), float("nan"), dtype=torch.float32).pin_memory() for _ in views]
    stream = torch.cuda.current_stream()
    for v, ex in enumerate(order):
        bd.run_host(ins[v], outs[v], stream, **EXECUTORS[ex])
    bd.sync()
    for v, new in enumerate(views):
        ref = np.concatenate([oracle.kahn(g.n, g.src, g.dst, new[i])[0] for i, g in enumerate(wl.graphs)])
        np.testing.assert_array_equal(bits(outs[v].numpy()), bits(ref), err_msg="view %d (%s)" % (v, order[v]))
    bd.close()


def test_run_host_payloads_and_bad_delay():
    """Payload results through hf_batch_run_host equal the oracle's; a non-finite delay is
    reported by the next synchronisation, as with hf_batch_set_delays."""
    wl = S.batch(7, graphs=8, nmin=500, nmax=20000, frac_saxpy=0.1, sx_min=1, sx_max=3000)
    bd = BatchOnDevice(wl)
    N = wl.n_tasks
    dl = torch.from_numpy(np.concatenate([g.delay for g in wl.graphs])).pin_memory()
    out = torch.empty(N, dtype=torch.float32).pin_memory()
    bd.run_host(dl, out, mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC)
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        ref = oracle.run_spec(spec)
        _check_payloads(bd.graphs[i], ref)
    ref = np.concatenate([oracle.run_spec(g)["arr"] for g in wl.graphs])
    np.testing.assert_array_equal(bits(out.numpy()), bits(ref))
    bad = dl.clone().pin_memory()
    bad[777] = float("inf")
    bd.run_host(bad, out, mode=hf.HF_MODE_TEAM)
    assert bd.sync(check=False) == hf.HF_EINVAL
    bd.close()


def test_unpinned_pull_buffer_rejected():
    g = hf.hf_graph_create()
    buf = np.zeros(16, np.float32)  # pageable host memory
    hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=buf.ctypes.data, bytes=64))
    with pytest.raises(hf.HfError) as ei:
        hf.hf_run(g, None, hf.hf_run_opts_default())
    assert ei.value.status == hf.HF_EINVAL
    hf.hf_graph_destroy(g)


def test_work_stealing_counters():
    """Work stealing moves work between CTAs: with rings, ready tasks go to the owner's ring and
    idle CTAs steal; without, no ring is touched. Arrivals are the oracle's either way."""
    wl = S.batch(5, graphs=8, nmin=2000, nmax=30000)
    ref = [oracle.run_spec(g)["arr"] for g in wl.graphs]
    bd = BatchOnDevice(wl)
    seen = {}
    for ring in (0, 64, 4096):
        bd.run(mode=hf.HF_MODE_PERSISTENT, steal_ring=ring, ctas=8, instrument=2)
        bd.sync()
        st = hf.hf_batch_get_stats(bd.b)
        seen[ring] = st
        for i in range(len(wl.graphs)):
            np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(ref[i]), err_msg="ring %d graph %d" % (ring, i))
        n = sum(g.n for g in wl.graphs)
        assert st["items"] == n
    assert seen[0]["push_ring"] == 0 and seen[0]["steals"] == 0
    for ring in (64, 4096):
        assert seen[ring]["push_ring"] > 0 and seen[ring]["steals"] > 0, seen[ring]
    # a 64-slot ring overflows into the global queue more than a 4096-slot one
    assert seen[64]["push_global"] >= seen[4096]["push_global"]
    bd.close()
