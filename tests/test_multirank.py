"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2): the step time is the
maximum over ranks, the units processed are summed over ranks (each rank runs its own batch),
the job rate divides the two, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 3.0 * rank)
    n = bench.sum_over_ranks(1000 + rank)
    out.put((rank, ms, n, bench.job_rate(n, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, n, rate in got:
        assert ms == 13.0 and n == 2001.0
        assert rate == pytest.approx(2001.0 / 13.0e-3)


def test_single_process_reductions_are_identities():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5) == 7.5 and bench.sum_over_ranks(42) == 42.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "layered10k", "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "layered10k", "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "layered10k"


def _shard_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_2203_08395_b300 import synth as S
    from paper_2203_08395_b300.workload import share

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    # the benchmark's strong-scaling path: the same batch on every rank, each taking its LPT share
    full = S.batch(5, graphs=14, nmin=200, nmax=6000, frac_saxpy=0.1, sx_min=16, sx_max=512)
    full.graphs.append(S.mixed(6, n=800, nmin=16, nmax=256, n_copy=20))  # pulls and pushes too
    mine, idx = share(full, rank, world)
    flags = torch.zeros(len(full.graphs), dtype=torch.int64)
    flags[idx] = 1
    gathered = [torch.empty_like(flags) for _ in range(world)]
    dist.all_gather(gathered, flags)
    n_all = bench.sum_over_ranks(mine.n_tasks)
    out.put((rank, [int(x) for x in sum(gathered)], n_all, full.n_tasks, [g.name for g in mine.graphs],
             [full.graphs[i].name for i in idx]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_batch_by_lpt():
    """bench.py --shard lpt on CPU ranks: each rank's share (workload.share, i.e.
    hf_batch_partition's balanced bin packing, the paper's Algorithm 1) is disjoint from the other's,
    together they cover the batch, and the tasks summed over ranks are the batch's."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, covered, n_all, n_full, names, want in got:
        assert covered == [1] * len(covered)
        assert n_all == n_full
        assert names == want and len(names) > 0
