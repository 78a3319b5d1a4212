#!/usr/bin/env python3
"""Benchmark of the task-graph executor on one B300 (one JSON line on stdout, rank 0).

A step is one execution of the whole workload through the C ABI (hf_batch_run): reset of
counters and queue, then the executor (persistent kernel, or the level-synchronous CUDA
graph), every task's payload included. Inputs (graph structure, delays, saxpy data) are
resident in HBM before the timed region and larger than L2 (126 MB), so no flush is needed.

Reported:
  value        tasks/s of the headline executor (whole job; weak scaling over ranks)
  edges_per_s  the same run in edges/s
  compare      the same workload under the level-synchronous executor
  e2e          per step through the public API with host buffers: new edge delays from
               page-locked host memory (hf_batch_set_delays), the run, all arrivals back to
               the host (hf_batch_get_arrivals index -1)
  roofline     algorithmic bytes of the dominant kernel / its CUDA-event time vs measured HBM
  cpu_baseline the CPU oracle (sequential Kahn, 1 thread) on a bounded sample of the workload

--impl reference times the CPU oracle alone on this workload (the method's plain definition).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "batch256"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2203_08395_b300", "csrc", "kernels.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--mode", default="persistent", choices=["persistent", "levelsync"])
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--claim", type=int, default=1)
    ap.add_argument("--local-keep", type=int, default=-1)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def traffic_for(kernel, workload):
    """Per-launch DRAM bytes from a committed ncu summary, if taken on the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
        e = t.get(kernel + "/" + workload)
        if e and e.get("kernels_sha256") == sha:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampler for SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(wl):
    """8E + 12N + 4 per graph (row pointers, successor ids+delays, counter reads, arrival writes)
    plus 12 bytes per saxpy element (read x, read y, write y) and 2x the bytes of each copy."""
    b = 0
    for g in wl.graphs:
        b += 8 * g.m + 12 * g.n + 4
        b += 12 * g.saxpy_elems
        for j in g.pl_saxpy:
            b += 2 * 4 * int(g.sx_n[j])
        for j in g.ps_saxpy:
            b += 2 * 4 * int(g.sx_n[j])
    return b


def cpu_oracle_rate(wl, budget_s=15.0, max_graphs=None):
    """Times the oracle (single thread) on whole graphs of the workload, in order, until about
    budget_s of oracle time. Returns (tasks/s, edges/s, description)."""
    import oracle

    tasks = edges = 0
    spent = 0.0
    used = 0
    for g in wl.graphs:
        prep = oracle.prepare(g)
        t0 = time.perf_counter()
        oracle.execute(prep)
        spent += time.perf_counter() - t0
        tasks += g.n
        edges += g.m
        used += 1
        del prep
        if spent >= budget_s or (max_graphs and used >= max_graphs):
            break
    desc = "%d of %d graphs (%d tasks, %d edges), %.1f s of oracle time" % (used, len(wl.graphs), tasks, edges, spent)
    return tasks / spent, edges / spent, desc


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2203_08395_b300 import synth as S

    wl = S.config(args.workload, seed=0)
    # each step: the oracle over a bounded prefix of the workload's graphs
    import oracle

    oracle.build()
    per_step_graphs = max(1, min(len(wl.graphs), 8))
    sample = S.Workload(wl.name, wl.graphs[:per_step_graphs])
    preps = None
    times = []
    for i in range(args.warmup + args.steps):
        preps = [oracle.prepare(g) for g in sample.graphs]
        t0 = time.perf_counter()
        for p in preps:
            oracle.execute(p)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
        if sum(times) > 120:
            break
    ms = 1e3 * float(np.mean(times))
    value = sample.n_tasks / (ms / 1e3)
    desc = "%d of %d graphs per step (%d tasks, %d edges)" % (per_step_graphs, len(wl.graphs), sample.n_tasks,
                                                                 sample.n_edges)
    line = {
        "impl": "reference", "metric": "DAG tasks/s", "value": value, "unit": "tasks/s", "n_gpus": 0,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2203_08395_b300 import hf
    from paper_2203_08395_b300 import synth as S
    from paper_2203_08395_b300.workload import BatchOnDevice

    hf.install_torch_allocator()
    t_gen = time.time()
    wl = S.config(args.workload, seed=rank)  # weak scaling: every rank runs its own instance
    bd = BatchOnDevice(wl)
    t_gen = time.time() - t_gen
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    mode = hf.HF_MODE_PERSISTENT if args.mode == "persistent" else hf.HF_MODE_LEVELSYNC
    opts = dict(mode=mode, ctas=args.ctas, claim=args.claim, local_keep=args.local_keep, chunk_elems=args.chunk)

    def timed(opts_, steps, warmup):
        for _ in range(warmup):
            bd.run(stream, **opts_)
        bd.sync()
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        kms = []
        evs[0].record(stream)
        for i in range(steps):
            bd.run(stream, time_kernel=1, **opts_)
            evs[i + 1].record(stream)
            kms.append(None)
        torch.cuda.synchronize()
        st = bd.sync(check=False)
        barrier()
        step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        kernel_ms = hf.hf_batch_kernel_ms(bd.b)  # last step's main kernel
        return float(np.mean(step_ms)), float(np.median(step_ms)), kernel_ms, st

    # kernel-only time per step: one more pass with time_kernel, averaged
    clocks = Clocks(local)
    clocks.start()
    ms_mean, ms_med, _, status = timed(opts, args.steps, args.warmup)
    clk = clocks.stop()
    kms = []
    for _ in range(min(args.steps, 20)):
        bd.run(stream, time_kernel=1, **opts)
        kms.append(hf.hf_batch_kernel_ms(bd.b))
    kernel_ms = float(np.mean(kms))
    if status != 0:
        raise SystemExit("run failed: %s" % hf.hf_status_string(status))

    ms = ms_mean
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    N, E = wl.n_tasks, wl.n_edges
    value = world * N / (ms / 1e3)

    compare = None
    if not args.no_compare:
        other = dict(opts, mode=hf.HF_MODE_LEVELSYNC if mode == hf.HF_MODE_PERSISTENT else hf.HF_MODE_PERSISTENT)
        c_mean, c_med, _, c_st = timed(other, max(5, args.steps // 4), 3)
        compare = {"executor": "levelsync" if other["mode"] == hf.HF_MODE_LEVELSYNC else "persistent",
                   "tasks_per_s": N / (c_mean / 1e3), "edges_per_s": E / (c_mean / 1e3), "ms_per_step": c_mean,
                   "status": hf.hf_status_string(c_st)}

    e2e = None
    if not args.no_e2e:
        delays = torch.cat([torch.from_numpy(g.delay) for g in wl.graphs]).pin_memory()
        arr_host = torch.empty(N, dtype=torch.float32, pin_memory=True)
        steps = max(3, args.steps // 4)
        for i in range(steps + 2):
            if i == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            hf.hf_batch_set_delays(bd.b, delays, on_device=False, stream=stream)
            bd.run(stream, **opts)
            hf.hf_batch_get_arrivals(bd.b, -1, N, out=arr_host.numpy())
        st = bd.sync(check=False)
        dt = (time.perf_counter() - t0) / steps
        e2e = {"value": world * N / dt, "unit": "tasks/s", "h2d_bytes_per_step": 4 * E,
               "d2h_bytes_per_step": 4 * N + 4, "ms_per_step": 1e3 * dt, "status": hf.hf_status_string(st)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, erate, desc = cpu_oracle_rate(wl)
        cpu = {"value": rate, "unit": "tasks/s", "cores": 1, "kind": "oracle", "sample": desc,
               "edges_per_s": erate, "host_nproc": os.cpu_count()}

    peak, peak_kind = peaks()
    b_alg = algorithmic_bytes(wl)
    kname = "k_persist" if mode == hf.HF_MODE_PERSISTENT else "k_level"
    achieved = b_alg / (kernel_ms / 1e3) / 1e9
    traffic = traffic_for(kname, args.workload)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": b_alg,
            "kernel_ms": kernel_ms, "peak_source": peak_kind}
    launches_per_step = 2 if mode == hf.HF_MODE_PERSISTENT else sum(1 for _ in range(max(g.levels for g in wl.graphs) or 1))
    line = {
        "metric": "DAG tasks/s", "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_median": ms_med, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "edges_per_s": world * E / (ms / 1e3),
        "config": {"workload": args.workload, "executor": args.mode, "tasks": N, "edges": E,
                   "graphs": len(wl.graphs), "saxpy_elems": wl.saxpy_elems, "ctas": args.ctas,
                   "claim": args.claim, "local_keep": args.local_keep, "chunk_elems": args.chunk,
                   "l2": "inputs larger than L2 (graph %.0f MB + payload %.0f MB)" % (
                       (8 * E + 16 * N) / 1e6, 8 * wl.saxpy_elems / 1e6),
                   "setup_s": t_gen},
        "compare": compare, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    bd.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
