"""Network kernels against the float64 oracle."""
import numpy as np
import pytest

from oracle import mlp
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


def _params(seed):
    rng = gg.Rng(seed)
    return np.array([(rng.uniform() - 0.5) * 0.6 for _ in range(mlp.N_PARAMS)], dtype=np.float32)


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


@pytest.mark.parametrize("batch", [1, 7, 128, 1000, 4099])
def test_forward_and_grad(ctx, batch):
    rng = np.random.default_rng(batch)
    x = rng.random((batch, 12)).astype(np.float32)
    y = rng.random(batch).astype(np.float32)
    p = _params(batch)
    _, _, yhat = mlp.forward(p.astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(ctx.mlp_forward(p, x), yhat, rtol=1e-5, atol=1e-6)
    g_ref = mlp.grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    g = ctx.mlp_grad(p, x, y)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-5 * scale)


def test_adam_step(ctx):
    p = _params(3)
    g = _params(4)
    m = np.zeros_like(p); v = np.zeros_like(p)
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in (1, 2, 3):
        ctx.mlp_adam(p, g, m, v, t, lr=0.01)
        pr, mr, vr = mlp.adam_step(pr, g.astype(np.float64), mr, vr, t, lr=0.01)
    np.testing.assert_allclose(p, pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(m, mr, rtol=1e-5, atol=1e-7)


def test_train_matches_oracle_steps(ctx):
    rng = np.random.default_rng(5)
    B = 300
    x = rng.random((B, 12)).astype(np.float32)
    y = (x[:, :3].sum(axis=1) / 3).astype(np.float32)
    p0 = _params(6)
    epochs, mb = 3, 64
    perm = np.stack([rng.permutation(B) for _ in range(epochs)]).astype(np.int32)
    p = p0.copy()
    loss = ctx.mlp_train(p, x, y, mb, perm, lr=0.01)
    pr = p0.astype(np.float64)
    m = np.zeros_like(pr); v = np.zeros_like(pr)
    t = 0
    losses = []
    for e in range(epochs):
        tot = 0.0
        for s in range(0, B, mb):
            idx = perm[e, s: s + mb]
            _, _, yh = mlp.forward(pr, x[idx])
            tot += float(((yh - y[idx]) ** 2).sum())
            t += 1
            pr, m, v = mlp.adam_step(pr, mlp.grad(pr, x[idx], y[idx]), m, v, t, lr=0.01)
        losses.append(tot / B)
    np.testing.assert_allclose(p, pr, rtol=2e-3, atol=2e-4)
    np.testing.assert_allclose(loss, losses, rtol=1e-3)
