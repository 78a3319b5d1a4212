"""Repeated runs (Section III-B's run_n / run_until) through the C ABI: payloads apply once per
run and arrivals stay the oracle's, the plan is reused, a sequence reports its first failure,
and run_until stops when its predicate says so."""
import numpy as np
import pytest

import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S
from paper_2203_08395_b300.workload import BatchOnDevice, GraphOnDevice

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = {"levelsync": dict(mode=hf.HF_MODE_LEVELSYNC), "persistent": dict(mode=hf.HF_MODE_PERSISTENT),
         "steal": dict(mode=hf.HF_MODE_PERSISTENT, steal_ring=128), "team": dict(mode=hf.HF_MODE_TEAM)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    hf.install_torch_allocator()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _saxpy_chain(n_elems, a):
    """max-plus source -> saxpy (y += a x) -> max-plus sink, on caller device buffers."""
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(-1, 1, n_elems).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.uniform(-1, 1, n_elems).astype(np.float32)).cuda()
    g = hf.hf_graph_create()
    s = hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_maxplus_payload(op=hf.HF_K_MAXPLUS, arr0=1.25))
    k = hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=a, n=n_elems, x_pull=-1,
                                                           y_pull=-1, x_dev=x.data_ptr(), y_dev=y.data_ptr()))
    t = hf.hf_add_task(g, hf.HF_KERNEL, None)
    hf.hf_precede_w(g, s, k, 0.5)
    hf.hf_precede_w(g, k, t, 0.25)
    return g, x, y


@pytest.mark.parametrize("mode", sorted(MODES))
def test_run_n_applies_payloads_n_times(mode):
    g, x, y = _saxpy_chain(5000, 0.5)
    x0, y0 = x.cpu().numpy(), y.cpu().numpy()
    hf.hf_run_n(g, 3, opts=hf.hf_run_opts_default(**MODES[mode]))
    hf.hf_sync_status(g)
    want = y0
    for _ in range(3):
        want = oracle.saxpy_f32(0.5, x0, want)
    np.testing.assert_array_equal(bits(y.cpu().numpy()), bits(want))
    np.testing.assert_array_equal(bits(hf.hf_get_arrivals(g, 3)), bits(np.array([1.25, 1.75, 2.0], np.float32)))
    hf.hf_graph_destroy(g)


def test_run_n_reports_a_failure_and_recovers():
    """A stalled task (bounded waits, no GPU fault) in a sequence of three runs: the sequence's
    status is HF_ETIMEDOUT; a clean sequence on the same plan afterwards is exact."""
    spec = S.layered(8, 20000, 40, 1, 4)
    gd = GraphOnDevice(spec)
    hf.hf_run_n(gd.g, 3, opts=hf.hf_run_opts_default(mode=hf.HF_MODE_PERSISTENT, stall_task=12345,
                                                    spin_limit_ns=50_000_000))
    assert gd.sync(check=False) == hf.HF_ETIMEDOUT
    hf.hf_run_n(gd.g, 3, opts=hf.hf_run_opts_default(mode=hf.HF_MODE_PERSISTENT))
    gd.sync()
    np.testing.assert_array_equal(bits(gd.arrivals()), bits(oracle.run_spec(spec)["arr"]))
    gd.close()


@pytest.mark.parametrize("mode", sorted(MODES))
def test_run_until_stops_on_the_predicate(mode):
    g, x, y = _saxpy_chain(3000, 2.0)
    x0, y0 = x.cpu().numpy(), y.cpu().numpy()
    calls = []

    def pred():
        calls.append(1)
        return len(calls) == 4

    runs = hf.hf_run_until(g, pred, 10, opts=hf.hf_run_opts_default(**MODES[mode]))
    assert runs == 4 and len(calls) == 4
    want = y0
    for _ in range(4):
        want = oracle.saxpy_f32(2.0, x0, want)
    np.testing.assert_array_equal(bits(y.cpu().numpy()), bits(want))
    assert hf.hf_run_until(g, lambda: False, 2, opts=hf.hf_run_opts_default(**MODES[mode])) == 2
    hf.hf_graph_destroy(g)


def test_batch_run_n_and_until():
    wl = S.batch(4, graphs=5, nmin=1000, nmax=8000)
    bd = BatchOnDevice(wl)
    hf.hf_batch_run_n(bd.b, 2, opts=hf.hf_run_opts_default(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC))
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(oracle.run_spec(spec)["arr"]))
    n = [0]

    def pred():
        n[0] += 1
        return n[0] >= 3

    assert hf.hf_batch_run_until(bd.b, pred, 5) == 3
    bd.close()
