"""Parity of the benchmarked configuration at full size, in the plan the benchmark times.

The benchmark's headline runs the 256-graph mixed batch (9.95 M tasks, 34.6 M edges, 1.38 G
saxpy elements) with learned costs (a model trained on recordings of two other seeds), the
executor the cost model picks, autotuned launch options and, for the team executor, its
concurrent team classes up to 8-CTA clusters. This test builds that plan with the benchmark's
own code (bench.headline_plan) and checks one run of it against the CPU oracle:

* every arrival, bit for bit (max-plus arrivals are schedule-independent: the dependency rule
  of Section III-A, "Add a Dependency Link", fixes every sum's inputs);
* >= 256 sampled saxpy tasks, bit for bit against the oracle's fused multiply-add (Listing 1's
  kernel in FP32), at least a quarter of them from graphs that ran on the largest clusters;
* the end-to-end call the benchmark also times (hf_batch_run_host: delays in, arrivals out
  through page-locked host memory), bit for bit.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S
from paper_2203_08395_b300.workload import BatchOnDevice

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    hf.load()
    hf.install_torch_allocator()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def test_headline_batch256_mixed_full_size_in_the_benchmarked_plan():
    name = bench.DEFAULT_WORKLOAD
    assert name == "batch256_mixed"
    wl = S.config(name, seed=0)
    bd = BatchOnDevice(wl)
    stream = torch.cuda.current_stream()
    hp = bench.headline_plan(bd, wl, stream, name)
    try:
        assert hp["prio"] == hf.HF_PRIO_LEARNED
        G, N = len(wl.graphs), wl.n_tasks
        ref = np.concatenate([oracle.run_spec(g, with_data=False)["arr"] for g in wl.graphs])
        # one timed-step run on fresh payload data
        bd.reset_y()
        bd.run(stream, **hp["opts"])
        assert bd.sync(check=False) == hf.HF_OK
        np.testing.assert_array_equal(bits(hf.hf_batch_get_arrivals(bd.b, -1, N)), bits(ref))
        # sampled saxpy tasks, weighted towards the graphs on the largest teams
        rng = np.random.default_rng(2024)
        if hp["chosen"] == hf.HF_MODE_TEAM:
            team = hf.hf_batch_team_plan(bd.b, G)
            print("team sizes:", {int(k): int((team == k).sum()) for k in np.unique(team)})
        else:
            team = np.ones(G, np.int32)
        big = np.flatnonzero(team == team.max())
        cand = [(g, j) for g in range(G) for j in range(wl.graphs[g].sx_task.size)]
        cand_big = [(g, j) for g, j in cand if g in set(big.tolist())]
        pick = [cand_big[i] for i in rng.choice(len(cand_big), min(96, len(cand_big)), replace=False)]
        pick += [cand[i] for i in rng.choice(len(cand), 192, replace=False)]
        for g, j in pick:
            spec = wl.graphs[g]
            want = oracle.saxpy_f32(spec.sx_a[j], spec.init_x(j), spec.init_y(j))
            got = bd.graphs[g].y_of(j).cpu().numpy()
            np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32), err_msg="graph %d saxpy %d" % (g, j))
        assert len(pick) >= 256
        # the end-to-end call of the benchmark, with the same delays
        delays = torch.cat([torch.from_numpy(g.delay) for g in wl.graphs]).pin_memory()
        out = torch.full((N,), float("nan"), dtype=torch.float32).pin_memory()
        bd.run_host(delays, out, stream, **hp["opts"])
        assert bd.sync(check=False) == hf.HF_OK
        np.testing.assert_array_equal(bits(out.numpy()), bits(ref))
    finally:
        bd.close()
        if hp["cm"] is not None:
            hf.hf_costmodel_destroy(hp["cm"])
