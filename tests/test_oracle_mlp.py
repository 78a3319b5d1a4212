"""Pins for the cost-model oracle (oracle/mlp.py) against things other than itself:
torch's BF16 conversion, central finite differences, torch autograd in FP64, torch's Adam,
and closed-form forward cases; the features against hand-derived values on the paper's
saxpy graph (Section I, Figure 1)."""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 10000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0 + 2 ** -8 + 2 ** -9, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def _rand_params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(0, scale, (64, 12)), b1=rng.normal(0, 0.1, 64), W2=rng.normal(0, scale / 4, (64, 64)),
                b2=rng.normal(0, 0.1, 64), w3=rng.normal(0, 0.3, 64), b3=0.3)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _rand_params(1)
    X = rng.normal(0, 1, (7, 12))
    t = rng.normal(0, 1, 7)
    y, cache = mlp.forward(p, X, rounding=False)
    g = mlp.backward(cache, y, t)
    h = 1e-6
    for k in ["W1", "b1", "W2", "b2", "w3", "b3"]:
        base = np.asarray(p[k], np.float64)
        flat = base.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False) if flat.size > 1 else [0]
        for i in idx:
            pp = {kk: np.array(vv, np.float64, copy=True) for kk, vv in p.items()}
            pm = {kk: np.array(vv, np.float64, copy=True) for kk, vv in p.items()}
            pp[k].reshape(-1)[i] += h
            pm[k].reshape(-1)[i] -= h
            fd = (mlp.loss(mlp.forward(pp, X, False)[0], t) - mlp.loss(mlp.forward(pm, X, False)[0], t)) / (2 * h)
            an = np.asarray(g[k], np.float64).reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (k, i, fd, an)


def test_backward_matches_torch_autograd_fp64():
    rng = np.random.default_rng(2)
    p = _rand_params(2)
    X = rng.normal(0, 1, (33, 12))
    t = rng.normal(0, 1, 33)
    y, cache = mlp.forward(p, X, rounding=False)
    g = mlp.backward(cache, y, t)
    tp = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()}
    Xt = torch.tensor(X)
    h1 = torch.relu(Xt @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    yt = h2 @ tp["w3"] + tp["b3"]
    L = torch.mean((yt - torch.tensor(t)) ** 2)
    L.backward()
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    for k in p:
        np.testing.assert_allclose(np.asarray(g[k], np.float64), tp[k].grad.numpy(), rtol=1e-10, atol=1e-12)


def test_forward_closed_forms():
    X = np.random.default_rng(3).normal(0, 1, (5, 12))
    p = dict(W1=np.zeros((64, 12)), b1=np.zeros(64), W2=np.zeros((64, 64)), b2=np.zeros(64), w3=np.zeros(64),
             b3=1.25)
    y, _ = mlp.forward(p, X)
    assert np.all(y == 1.25)
    # one active path: x0 -> h1[0] -> h2[0] -> y with unit weights and biases 0: y = relu(x0)
    p = dict(W1=np.zeros((64, 12)), b1=np.zeros(64), W2=np.zeros((64, 64)), b2=np.zeros(64), w3=np.zeros(64),
             b3=0.0)
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["w3"][0] = 1.0
    X = np.array([[0.5] + [0.0] * 11, [-0.5] + [0.0] * 11, [3.0] + [9.0] * 11])
    y, _ = mlp.forward(p, X)
    np.testing.assert_array_equal(y, [0.5, 0.0, 3.0])


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    p = _rand_params(4)
    tp = [torch.tensor(np.atleast_1d(np.asarray(v, np.float64)), requires_grad=True) for v in p.values()]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m, v = mlp.zeros_like(p), mlp.zeros_like(p)
    cur = {k: np.asarray(val, np.float64) for k, val in p.items()}
    for step in range(1, 6):
        g = {k: rng.normal(0, 1, np.shape(val)) for k, val in p.items()}
        for tt, k in zip(tp, p):
            tt.grad = torch.tensor(np.atleast_1d(g[k]))
        opt.step()
        cur, m, v = mlp.adam_step(cur, g, m, v, step, 1e-2)
    for tt, k in zip(tp, p):
        np.testing.assert_allclose(np.atleast_1d(cur[k]), tt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_heuristic_cost_by_hand():
    F = np.zeros((2, 12))
    F[0, 5], F[0, 8] = np.log1p(3), np.log1p(1200)  # fan-out 3, 1200 payload bytes
    np.testing.assert_allclose(mlp.heuristic_cost(F), [300 + 90 + 150, 300.0])


def test_features_on_paper_saxpy_graph():
    # Figure 1: host_x(0) host_y(1) pull_x(2) pull_y(3) kernel(4) push_x(5) push_y(6)
    src = [0, 1, 2, 3, 4, 4]
    dst = [2, 3, 4, 4, 5, 6]
    cat = [9, 9, 2, 2, 1, 3, 3]  # host tasks fall in none of the four one-hot classes
    N = 65536
    pb = [0, 0, 4 * N, 4 * N, 12 * N, 4 * N, 4 * N]
    F = mlp.features(7, src, dst, cat, pb)
    # kernel: fan-in 2, fan-out 2, level 2 of 4 levels, successors' mean fan-out 0
    np.testing.assert_allclose(F[4], [0, 1, 0, 0, np.log(3), np.log(3), 0.5, np.log(3), np.log1p(12 * N),
                                      np.log(8), np.log(7), 0.0])
    # host_x: source, fan-out 1, its successor pull_x has fan-out 1
    np.testing.assert_allclose(F[0], [0, 0, 0, 0, 0, np.log(2), 0, 0, 0, np.log(8), np.log(7), np.log(2)])
    # push_y: sink at level 3
    np.testing.assert_allclose(F[6, [3, 4, 5, 6, 7]], [1, np.log(2), 0, 0.75, np.log(4)])
