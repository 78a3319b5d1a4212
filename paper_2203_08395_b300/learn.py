"""Training the cost model on timings the executor records (argument marshalling and data
plumbing only: features, timing, the MLP and its training all run in libhf.so kernels).

record()   runs a batch with the executor's cost recording on and returns, on the device, every
           task's 12 features and its log cost in ns. By default the team executor records (the
           executor whose planner consumes the costs): a task's cost is its thread's gather plus,
           for a payload task, the summed warp times of its pieces, under the run's real load
           (hf_batch_get_task_costs). executor="persistent" records the persistent executor's
           per-task time from pop to the end of its successors' release instead;
train()    trains a model on rows pooled from several recordings (hf_costmodel_train);
evaluate() compares the model's and the plain heuristic's cost predictions on a recording:
           MSE of log costs, median |log(predicted / actual)| and symmetric mean absolute
           percentage error (plain MAPE is not used: it caps under-prediction at 100%).
"""
from __future__ import annotations

import numpy as np

from . import hf

MIN_NS = 16.0  # costs below the timer's resolution are clamped (the timer ticks every 32 ns)


def record(bd, stream=None, executor="team", **opts):
    """Instrumented run of `bd` (a workload.BatchOnDevice) by `executor` ("team": the team
    executor under the heuristic plan, cost recording bit 2; "persistent": per-task timestamps);
    returns (X, t) CUDA tensors: X [N, 12] features, t [N] log ns."""
    import torch

    o = dict(opts)
    N = bd.n_tasks
    if executor == "team":
        o.setdefault("mode", hf.HF_MODE_TEAM)
        o.setdefault("priority", hf.HF_PRIO_HEURISTIC)
        bd.run(stream, instrument=4, **o)
        bd.sync()
        dt = np.maximum(hf.hf_batch_get_task_costs(bd.b, -1, N).astype(np.float64), MIN_NS)
    else:
        o.setdefault("mode", hf.HF_MODE_PERSISTENT)
        bd.run(stream, instrument=1, **o)
        bd.sync()
        t0 = np.empty(N, np.int64)
        t1 = np.empty(N, np.int64)
        off = 0
        for i, g in enumerate(bd.wl.graphs):
            a, b = hf.hf_batch_get_task_times(bd.b, i, g.n)
            t0[off:off + g.n] = a
            t1[off:off + g.n] = b
            off += g.n
        dt = np.maximum((t1 - t0).astype(np.float64), MIN_NS)
    X = torch.empty((N, hf.HF_FEATURES), dtype=torch.float32, device="cuda")
    hf.hf_batch_features(bd.b, X, stream)
    t = torch.from_numpy(np.log(dt).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    return X, t


def train(cm, recordings, rows=262144, epochs=12, batch=2048, lr=2e-3, seed=0):
    """Trains `cm` on up to `rows` rows drawn uniformly from the pooled recordings; returns
    the final MSE (log space) over the rows used."""
    import torch

    X = torch.cat([r[0] for r in recordings])
    t = torch.cat([r[1] for r in recordings])
    n = X.shape[0]
    if n > rows:
        g = torch.Generator(device="cpu").manual_seed(seed)
        idx = torch.randperm(n, generator=g)[:rows].cuda()
        X, t = X[idx].contiguous(), t[idx].contiguous()
        n = rows
    return hf.hf_costmodel_train(cm, X, t, n, epochs, batch, lr, seed)


def evaluate(bd, cm, recording, stream=None):
    """Prediction error of the learned model and of the heuristic on one recording."""
    import torch

    X, t = recording
    N = X.shape[0]
    y = torch.empty(N, device="cuda")
    hf.hf_costmodel_forward(cm, X, N, y, stream)
    cost = torch.empty(N, device="cuda")
    bot = torch.empty(N, device="cuda")
    hf.hf_batch_task_costs(bd.b, hf.HF_PRIO_HEURISTIC, cost, bot, stream)
    torch.cuda.synchronize()
    actual = torch.exp(t).double()
    learned = torch.exp(torch.clamp(y, 0, 30)).double()
    heur = cost.double()
    out = {}
    for name, pred in (("learned", learned), ("heuristic", heur)):
        lr = torch.log(pred) - t.double()
        out[name] = {
            "mse_log": float(torch.mean(lr ** 2)),
            "median_abs_log_ratio": float(torch.median(torch.abs(lr))),
            "smape": float(torch.mean(2 * torch.abs(pred - actual) / (pred + actual))),
        }
    return out
