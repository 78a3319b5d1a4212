"""FP64 oracle for the learned cost model. TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The model (the learned part of the executor; the paper itself has no learned component, its
scheduler is the heuristic prior art of Section III-C): an MLP 12 -> 64 -> 64 -> 1 that maps
per-task features to a predicted log task cost.

  x   : 12 features, stored as BF16
  z1  = W1 x + b1          (W1: 64x12 BF16, b1: 64 FP32, accumulate in FP32/FP64)
  h1  = bf16(relu(z1))
  z2  = W2 h1 + b2         (W2: 64x64 BF16)
  h2  = bf16(relu(z2))
  y   = w3 . h2 + b3       (w3: 64 BF16, b3: FP32 scalar)
  loss = mean_i (y_i - t_i)^2

Backward takes the BF16 weights as exact values (gradients flow to FP32 master weights; the
BF16 copies are re-rounded after every optimizer step). Adam: Kingma & Ba, "Adam: a method
for stochastic optimization", ICLR 2015, Algorithm 1 (bias-corrected moments).

Pins (tests/test_oracle_mlp.py): bf16 rounding against torch's conversion; gradients against
central finite differences and against torch autograd in FP64 with rounding switched off;
Adam against torch.optim.Adam; closed-form forward cases.
"""
from __future__ import annotations

import numpy as np

D_IN, D_H = 12, 64


def bf16(a):
    """Round to the nearest BF16 value (ties to even), through FP32. Returns float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, rounding=True):
    """p: dict W1 (64,12), b1 (64,), W2 (64,64), b2 (64,), w3 (64,), b3 (scalar).
    X: (n, 12). Returns (y (n,), cache)."""
    X = np.asarray(X, np.float64)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    W1, W2, w3 = r(p["W1"]), r(p["W2"]), r(p["w3"])
    xb = r(X)
    z1 = xb @ W1.T + np.asarray(p["b1"], np.float64)
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + np.asarray(p["b2"], np.float64)
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ w3 + float(p["b3"])
    return y, dict(x=xb, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, w3=w3)


def loss(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def backward(cache, y, t):
    """Gradients of mean squared error w.r.t. W1, b1, W2, b2, w3, b3."""
    n = y.shape[0]
    dy = 2.0 * (np.asarray(y, np.float64) - np.asarray(t, np.float64)) / n
    g = {}
    g["w3"] = cache["h2"].T @ dy
    g["b3"] = float(dy.sum())
    dh2 = np.outer(dy, cache["w3"])
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ cache["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["x"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter (step counts from 1). Returns new (p, m, v)."""
    p2, m2, v2 = {}, {}, {}
    for k in p:
        gk = np.asarray(g[k], np.float64)
        m2[k] = beta1 * np.asarray(m[k], np.float64) + (1.0 - beta1) * gk
        v2[k] = beta2 * np.asarray(v[k], np.float64) + (1.0 - beta2) * gk * gk
        mh = m2[k] / (1.0 - beta1 ** step)
        vh = v2[k] / (1.0 - beta2 ** step)
        p2[k] = np.asarray(p[k], np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def zeros_like(p):
    return {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in p.items()}


def init_params(seed=0):
    """He-uniform initialisation (limit sqrt(6 / fan_in)), biases zero; values pre-rounded to
    BF16 where the model stores BF16."""
    rng = np.random.default_rng(seed)
    lim1, lim2 = np.sqrt(6.0 / D_IN), np.sqrt(6.0 / D_H)
    return dict(
        W1=bf16(rng.uniform(-lim1, lim1, (D_H, D_IN))),
        b1=np.zeros(D_H),
        W2=bf16(rng.uniform(-lim2, lim2, (D_H, D_H))),
        b2=np.zeros(D_H),
        w3=bf16(rng.uniform(-lim2, lim2, D_H)),
        b3=0.0,
    )


def heuristic_cost(F):
    """The plain heuristic task cost (ns of warp time) the learned model is judged against:
    300 per task + 30 per out-edge + payload bytes / 8 (bytes per ns one warp moves).
    Computed from the features' fan-out and payload-bytes entries."""
    F = np.asarray(F, np.float64)
    return 300.0 + 30.0 * np.expm1(F[:, 5]) + np.expm1(F[:, 8]) / 8.0


# --------------------------------------------------------------------- per-task features

FEATURES = [
    "is_maxplus", "is_saxpy", "is_pull", "is_push",
    "log1p_fanin", "log1p_fanout", "level_frac", "log1p_level",
    "log1p_payload_bytes", "log1p_graph_tasks", "log1p_graph_edges", "log1p_mean_succ_fanout",
]


def features(n, src, dst, cat, payload_bytes):
    """The 12 per-task features of one graph, FP64.

    cat[v]: 0 max-plus kernel task, 1 saxpy kernel task, 2 pull, 3 push, other = none of
    these (all four one-hot entries zero). payload_bytes[v]: bytes the payload moves (saxpy:
    12 bytes per element; copies: the copy size; max-plus: 0).
    level(v) = longest hop count from any source (sources are level 0); level_frac divides by
    the number of levels of the graph (max level + 1).
    """
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    m = src.size
    fin = np.bincount(dst, minlength=n).astype(np.float64)
    fout = np.bincount(src, minlength=n).astype(np.float64)
    # levels by relaxation in topological order (own small Kahn pass, FP64 not needed: ints)
    level = np.zeros(n, np.int64)
    pend = fin.astype(np.int64).copy()
    order = list(np.nonzero(pend == 0)[0])
    succ = [[] for _ in range(n)]
    for e in range(m):
        succ[src[e]].append(dst[e])
    i = 0
    while i < len(order):
        u = order[i]
        i += 1
        for v in succ[u]:
            if level[u] + 1 > level[v]:
                level[v] = level[u] + 1
            pend[v] -= 1
            if pend[v] == 0:
                order.append(v)
    nlev = int(level.max()) + 1 if n else 1
    msf = np.zeros(n)
    for u in range(n):
        if succ[u]:
            msf[u] = np.mean([fout[s] for s in succ[u]])
    F = np.zeros((n, D_IN))
    cat = np.asarray(cat)
    for k in range(4):
        F[:, k] = (cat == k).astype(np.float64)
    F[:, 4] = np.log1p(fin)
    F[:, 5] = np.log1p(fout)
    F[:, 6] = level / nlev
    F[:, 7] = np.log1p(level.astype(np.float64))
    F[:, 8] = np.log1p(np.asarray(payload_bytes, np.float64))
    F[:, 9] = np.log1p(float(n))
    F[:, 10] = np.log1p(float(m))
    F[:, 11] = np.log1p(msf)
    return F
