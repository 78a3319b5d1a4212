"""Team executor with the arrival keys of cluster jobs in distributed shared memory: bit-exact
against the oracle, the same as with every key in global memory, and used exactly where a
graph's keys fit (its task count / cluster size entries per CTA, every CTA of its class still
resident); single-CTA jobs, non-power-of-two clusters and payload batches keep global keys."""
import numpy as np
import pytest

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


def _check(bd, wl):
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(bits(bd.arrivals(i)), bits(oracle.run_spec(spec)["arr"]), err_msg=spec.name)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_shared_keys_bit_exact(k):
    # sizes with ragged shares (n_g not a multiple of k), fan-in up to 8 across far levels
    wl = S.Workload("sk", [S.layered(700 + i, n, max(4, n // 120), 1, 8, name="g%d" % i)
                           for i, n in enumerate([997, 4093, 12_289, 30_011])])
    bd = BatchOnDevice(wl)
    G = len(wl.graphs)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=k)
    bd.sync()
    assert (hf.hf_batch_team_plan(bd.b, G) == k).all()
    assert hf.hf_batch_team_keys(bd.b, G).all()
    _check(bd, wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=k, team_global_keys=1)
    bd.sync()
    assert not hf.hf_batch_team_keys(bd.b, G).any()
    _check(bd, wl)
    bd.close()


def test_graph_too_large_for_shared_memory_runs_from_global():
    # 2-CTA clusters: 150,000 keys (300 KB per CTA) never fit; the small graphs' do
    wl = S.Workload("sk2", [S.layered(800 + i, n, max(4, n // 250), 1, 6, name="h%d" % i)
                            for i, n in enumerate([1500, 150_000, 6000])])
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=2)
    bd.sync()
    np.testing.assert_array_equal(hf.hf_batch_team_keys(bd.b, 3), [1, 0, 1])
    _check(bd, wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=1)  # single CTAs: global keys
    bd.sync()
    assert not hf.hf_batch_team_keys(bd.b, 3).any()
    _check(bd, wl)
    bd.close()


def test_non_power_of_two_team_keeps_global_keys():
    wl = S.Workload("sk3", [S.layered(900 + i, n, max(4, n // 200), 1, 5, name="q%d" % i)
                            for i, n in enumerate([3000, 9000])])
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=3)
    bd.sync()
    assert not hf.hf_batch_team_keys(bd.b, 2).any()
    _check(bd, wl)
    bd.close()


def test_payload_batch_keeps_global_keys():
    # the payload kernel keeps every key in global memory
    wl = S.batch(5, graphs=4, nmin=1000, nmax=8000, frac_saxpy=0.1)
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=2)
    bd.sync()
    assert not hf.hf_batch_team_keys(bd.b, 4).any()
    _check(bd, wl)
    bd.close()


def test_whole_class_kernel_and_per_graph_tables():
    # every graph of the 4-CTA class fits: the class runs the kernel with shared keys only; with
    # one graph too large the class runs the general kernel, shared keys for the graphs that fit
    small = [S.layered(950 + i, n, max(4, n // 150), 1, 6, name="w%d" % i) for i, n in enumerate([2500, 7000, 11_000])]
    wl = S.Workload("sk5", small)
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=4)
    bd.sync()
    assert hf.hf_batch_team_keys(bd.b, 3).all()
    _check(bd, wl)
    bd.close()
    wl = S.Workload("sk6", small + [S.layered(960, 600_000, 2400, 1, 4, name="big")])
    bd = BatchOnDevice(wl)
    bd.run(mode=hf.HF_MODE_TEAM, team_size=4)
    bd.sync()
    np.testing.assert_array_equal(hf.hf_batch_team_keys(bd.b, 4), [1, 1, 1, 0])
    _check(bd, wl)
    bd.close()


def test_planned_batch_keys_only_in_clusters():
    wl = S.batch(9, graphs=24, nmin=1000, nmax=60_000)
    bd = BatchOnDevice(wl)
    G = len(wl.graphs)
    bd.run(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_HEURISTIC)
    bd.sync()
    k = hf.hf_batch_team_plan(bd.b, G)
    sk = hf.hf_batch_team_keys(bd.b, G)
    assert not sk[k <= 1].any()
    _check(bd, wl)
    with pytest.raises(hf.HfError):
        bd.run(mode=hf.HF_MODE_TEAM, team_global_keys=2)
    bd.close()
