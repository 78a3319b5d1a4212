"""Device placement (Section III-C, Algorithm 1) and batch sharding, host only: groups of a
kernel task and the pulls it uses never span devices, host tasks stay on the CPU, loads follow
the longest-processing-time rule (checked against brute force on small cases), and two gloo
ranks taking their shards cover every graph exactly once."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    hf.load()


def _pinned_free(nbytes):
    # host pointers are only stored by the builder; placement never dereferences them
    return 4096 * (1 + nbytes)


def test_kernel_and_its_pulls_share_a_device():
    g = hf.hf_graph_create()
    pulls = [hf.hf_add_task(g, hf.HF_PULL, hf.hf_pull_payload(host_ptr=_pinned_free(i), bytes=4096 * (i + 1)))
             for i in range(6)]
    ks = []
    for i in range(3):  # kernel i reads pull 2i and writes pull 2i+1
        ks.append(hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=2.0, n=1024 * (i + 1),
                                                                     x_pull=pulls[2 * i], y_pull=pulls[2 * i + 1])))
    push = hf.hf_add_task(g, hf.HF_PUSH, hf.hf_push_payload(src_pull=pulls[5], host_ptr=_pinned_free(9), bytes=64))
    h = hf.hf_add_task(g, hf.HF_HOST, hf.hf_host_payload(fn=hf.HOST_FN(lambda arg: None), arg=None))
    first = hf.hf_add_tasks_bulk(g, 4)
    dev = hf.hf_place(g, 11 + 4, 2)
    for i in range(3):
        assert dev[ks[i]] == dev[pulls[2 * i]] == dev[pulls[2 * i + 1]]
    assert dev[push] == dev[pulls[5]] and dev[h] == -1
    assert set(dev[first:first + 4]) <= {0, 1}
    # explicit costs: one heavy group goes alone on a device
    cost = np.ones(15, np.float32)
    cost[ks[0]] = 100.0
    dev = hf.hf_place(g, 15, 2, cost)
    heavy = dev[ks[0]]
    assert all(dev[v] != heavy for v in range(15) if v not in (ks[0], pulls[0], pulls[1], h))
    hf.hf_graph_destroy(g)


def _batch(sizes):
    b = hf.hf_batch_create()
    gs = []
    for n in sizes:
        g = hf.hf_graph_create()
        hf.hf_add_tasks_bulk(g, n)
        src = np.arange(n - 1, dtype=np.int32)
        hf.hf_precede_bulk(g, src, src + 1)
        hf.hf_batch_add(b, g)
        gs.append(g)
    return b, gs


def test_batch_partition_is_lpt_within_grahams_bound():
    rng = np.random.default_rng(2)
    for trial in range(20):
        sizes = rng.integers(10, 2000, int(rng.integers(2, 8)))
        ndev = int(rng.integers(2, 4))
        b, gs = _batch(sizes)
        dev, loads = hf.hf_batch_partition(b, len(sizes), ndev)
        cost = np.zeros(len(sizes))
        for d in range(ndev):
            assert loads[d] == pytest.approx(sum(300.0 * n + 30.0 * (n - 1) for n, x in zip(sizes, dev) if x == d))
        # brute-force optimum of the same costs
        per = 300.0 * sizes + 30.0 * (sizes - 1)
        best = min(max(np.bincount(np.array(a), weights=per, minlength=ndev))
                   for a in itertools.product(range(ndev), repeat=len(sizes)))
        assert loads.max() <= (4.0 / 3.0 - 1.0 / (3.0 * ndev)) * best + 1e-6
        hf.hf_batch_destroy(b)
        for g in gs:
            hf.hf_graph_destroy(g)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_rank(rank, port, sizes, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2203_08395_b300 import hf as H

    H.load()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    b = H.hf_batch_create()
    keep = []
    for n in sizes:
        g = H.hf_graph_create()
        H.hf_add_tasks_bulk(g, int(n))
        H.hf_batch_add(b, g)
        keep.append(g)
    dev, _ = H.hf_batch_partition(b, len(sizes), 2)
    mine = torch.tensor([1 if dev[i] == rank else 0 for i in range(len(sizes))], dtype=torch.int64)
    allv = [torch.empty_like(mine) for _ in range(2)]
    dist.all_gather(allv, mine)
    out.put((rank, (allv[0] + allv[1]).tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_every_graph_once():
    import torch.multiprocessing as mp

    sizes = [500, 40, 3000, 77, 1200, 9, 640]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, covered in got:
        assert covered == [1] * len(sizes)  # every graph on exactly one rank
