"""GPU parity of the learned cost model (MLP forward, gradients, Adam, training) and of the
feature, cost and bottom-level kernels against the FP64 oracle (oracle/mlp.py, oracle.kahn).

Tolerances: the GPU accumulates in FP32 and the oracle in FP64 with the same BF16 rounding
points; an FP32 rounding difference can move a hidden activation across a BF16 rounding
boundary (one BF16 ulp, 2^-8 relative), so outputs and gradients are compared at rtol 1e-2
with an absolute floor of 1e-2 of the largest magnitude, and most rows must agree to 1e-5.
Bottom levels are compared bit for bit (fixed inputs per add, monotone rounding)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
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
    hf.install_torch_allocator()


def flat(p):
    return np.concatenate([np.ravel(p["W1"]), p["b1"], np.ravel(p["W2"]), p["b2"], p["w3"], [p["b3"]]]).astype(np.float32)


def unflat(v):
    v = np.asarray(v, np.float64)
    return dict(W1=v[0:768].reshape(64, 12), b1=v[768:832], W2=v[832:4928].reshape(64, 64), b2=v[4928:4992],
                w3=v[4992:5056], b3=float(v[5056]))


def _params(seed):
    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed)
    p["b1"] = rng.normal(0, 0.1, 64)
    p["b2"] = rng.normal(0, 0.1, 64)
    p["b3"] = 0.5
    return unflat(flat(p))  # the FP32 master values the GPU holds


def _features(seed, n):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 12))
    X[np.arange(n), rng.integers(0, 4, n)] = 1
    X[:, 4:] = rng.uniform(0, 5, (n, 8))
    return X.astype(np.float32)


def test_forward_matches_oracle():
    p = _params(1)
    X = _features(2, 5000)
    cm = hf.hf_costmodel_create(0)
    hf.hf_costmodel_set_params(cm, flat(p))
    Xd = torch.from_numpy(X).cuda()
    yd = torch.empty(5000, device="cuda")
    hf.hf_costmodel_forward(cm, Xd, 5000, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref, _ = mlp.forward(p, X)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(y, ref, rtol=1e-2, atol=1e-2 * scale)
    assert np.mean(np.abs(y - ref) <= 1e-5 * np.maximum(np.abs(ref), 1)) > 0.99
    hf.hf_costmodel_destroy(cm)


def test_gradient_and_adam_match_oracle():
    p = _params(3)
    n = 3000
    X = _features(4, n)
    rng = np.random.default_rng(5)
    t = rng.normal(7, 2, n).astype(np.float32)
    cm = hf.hf_costmodel_create(0)
    hf.hf_costmodel_set_params(cm, flat(p))
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    g = torch.empty(hf.HF_COSTMODEL_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    hf.hf_costmodel_grad(cm, Xd, td, n, g, loss)
    torch.cuda.synchronize()
    y, cache = mlp.forward(p, X)
    gref = flat({k: v for k, v in mlp.backward(cache, y, t).items()})
    gg = g.cpu().numpy()
    np.testing.assert_allclose(loss.item(), mlp.loss(y, t), rtol=1e-4)
    np.testing.assert_allclose(gg, gref, rtol=1e-2, atol=1e-2 * np.abs(gref).max())
    # one Adam step from the GPU gradient, both sides from the same gradient values
    hf.hf_costmodel_adam_step(cm, g, 1e-3)
    torch.cuda.synchronize()
    after = hf.hf_costmodel_get_params(cm)
    zero = mlp.zeros_like(p)
    pref, _, _ = mlp.adam_step(p, unflat(gg), zero, zero, 1, 1e-3)
    np.testing.assert_allclose(after, flat(pref), rtol=1e-5, atol=1e-7)
    hf.hf_costmodel_destroy(cm)


def test_training_reduces_loss_and_save_load_roundtrip(tmp_path):
    rng = np.random.default_rng(6)
    n = 20000
    X = _features(7, n)
    # a target the model can represent: a smooth function of a few features
    t = (3.0 + 1.5 * X[:, 1] + 0.8 * X[:, 8] - 0.3 * X[:, 5] + 0.05 * rng.normal(size=n)).astype(np.float32)
    cm = hf.hf_costmodel_create(11)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    g = torch.empty(hf.HF_COSTMODEL_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    hf.hf_costmodel_grad(cm, Xd, td, n, g, loss)
    torch.cuda.synchronize()
    before = loss.item()
    after = hf.hf_costmodel_train(cm, Xd, td, n, epochs=20, batch=1024, lr=3e-3, seed=1)
    assert after < 0.05 * before and after < 0.05
    # the oracle's forward on the trained weights agrees with the GPU's loss
    params = hf.hf_costmodel_get_params(cm)
    y, _ = mlp.forward(unflat(params), X)
    assert abs(mlp.loss(y, t) - after) <= 1e-2 * max(after, 1e-3) + 1e-4
    path = str(tmp_path / "cm.bin")
    hf.hf_costmodel_save(cm, path)
    cm2 = hf.hf_costmodel_create(99)
    hf.hf_costmodel_load(cm2, path)
    np.testing.assert_array_equal(hf.hf_costmodel_get_params(cm2), params)
    hf.hf_costmodel_destroy(cm)
    hf.hf_costmodel_destroy(cm2)


def _cat_and_bytes(spec):
    cat = np.zeros(spec.n, np.int64)
    pb = np.zeros(spec.n, np.float64)
    for j, tsk in enumerate(spec.sx_task):
        cat[tsk] = 1
        pb[tsk] = 12.0 * spec.sx_n[j]
    for i, tsk in enumerate(spec.pl_task):
        cat[tsk] = 2
        pb[tsk] = 4.0 * spec.sx_n[spec.pl_saxpy[i]]
    for i, tsk in enumerate(spec.ps_task):
        cat[tsk] = 3
        pb[tsk] = 4.0 * spec.sx_n[spec.ps_saxpy[i]]
    return cat, pb


def test_features_costs_and_bottom_levels_match_oracle():
    wl = S.Workload("w", [S.mixed(2, n=3000, nmin=16, nmax=5000, n_copy=40),
                          S.batch(3, graphs=3, nmin=500, nmax=4000).graphs[1]])
    bd = BatchOnDevice(wl)
    N = wl.n_tasks
    Xd = torch.empty((N, 12), device="cuda")
    hf.hf_batch_features(bd.b, Xd)
    cost = torch.empty(N, device="cuda")
    bot = torch.empty(N, device="cuda")
    hf.hf_batch_task_costs(bd.b, hf.HF_PRIO_HEURISTIC, cost, bot)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy()
    off = 0
    for spec in wl.graphs:
        cat, pb = _cat_and_bytes(spec)
        F = mlp.features(spec.n, spec.src, spec.dst, cat, pb)
        np.testing.assert_allclose(X[off:off + spec.n], F, rtol=2e-6, atol=1e-6)
        np.testing.assert_allclose(cost.cpu().numpy()[off:off + spec.n], mlp.heuristic_cost(F), rtol=1e-5)
        off += spec.n
    # bottom levels bit for bit on seeded costs given to both sides
    c = S.uniform_f32(9, 1, N, 1.0, 5000.0)
    cd = torch.from_numpy(c).cuda()
    hf.hf_batch_bottom_levels(bd.b, cd, bot)
    torch.cuda.synchronize()
    b = bot.cpu().numpy()
    off = 0
    for spec in wl.graphs:
        ref = oracle.bottom_levels(spec.n, spec.src, spec.dst, c[off:off + spec.n])
        np.testing.assert_array_equal(b[off:off + spec.n].view(np.uint32), ref.view(np.uint32))
        off += spec.n
    # learned costs: exp of the oracle's forward on the oracle's features
    cm = hf.hf_costmodel_create(5)
    hf.hf_batch_set_costmodel(bd.b, cm)
    hf.hf_batch_task_costs(bd.b, hf.HF_PRIO_LEARNED, cost, bot)
    torch.cuda.synchronize()
    p = unflat(hf.hf_costmodel_get_params(cm))
    y, _ = mlp.forward(p, X)
    np.testing.assert_allclose(cost.cpu().numpy(), np.exp(np.clip(y, 0, 30)), rtol=3e-2)
    bd.close()
    hf.hf_costmodel_destroy(cm)


@pytest.mark.parametrize("prio", [hf.HF_PRIO_HEURISTIC, hf.HF_PRIO_LEARNED])
def test_priorities_never_change_results(prio):
    wl = S.batch(4, graphs=16, nmin=1000, nmax=30000)
    bd = BatchOnDevice(wl)
    cm = hf.hf_costmodel_create(3)
    hf.hf_batch_set_costmodel(bd.b, cm)
    bd.run(mode=hf.HF_MODE_PERSISTENT, priority=prio)
    bd.sync()
    for i, spec in enumerate(wl.graphs):
        np.testing.assert_array_equal(bd.arrivals(i).view(np.uint32), oracle.run_spec(spec)["arr"].view(np.uint32))
    bd.close()
    hf.hf_costmodel_destroy(cm)
