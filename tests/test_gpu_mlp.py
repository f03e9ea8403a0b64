"""GPU parity: the MLP cost-model kernels against the FP64 oracle (forward,
loss, per-tensor gradients within 1e-4 relative, Adam), determinism, and the
learned-schedule choice with its heuristic fallback."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

SLICES = {"W1": (0, 1024), "b1": (1024, 1088), "W2": (1088, 5184), "b2": (5184, 5248),
          "W3": (5248, 6016), "b3": (6016, 6028)}


def _data(B, seed):
    g = np.random.default_rng(seed)
    p = g.normal(0, 0.25, R.MLP_NPARAM).astype(np.float32)
    X = g.normal(size=(B, 16)).astype(np.float32)
    Y = g.normal(size=(B, 12)).astype(np.float32)
    return p, X, Y


@pytest.mark.parametrize("B", [1, 7, 256, 4099])
def test_forward_vs_oracle(rt, B):
    import torch
    p, X, _ = _data(B, 1)
    y = torch.zeros((B, 12), dtype=torch.float32, device="cuda")
    rt.mlp_forward(dev(p), dev(X), y)
    ref = O.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    got = host(y)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("B", [1, 33, 256, 2048])
def test_loss_and_gradients_vs_oracle(rt, B):
    import torch
    p, X, Y = _data(B, 2)
    g = torch.zeros(R.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    rt.mlp_loss_grad(dev(p), dev(X), dev(Y), g, loss)
    ref_loss, ref_g = O.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64),
                                      Y.astype(np.float64))
    assert abs(float(host(loss)[0]) - ref_loss) <= 1e-5 * abs(ref_loss)
    got = host(g)
    for name, (a, b) in SLICES.items():
        err = np.linalg.norm(got[a:b] - ref_g[a:b])
        assert err <= 1e-4 * np.linalg.norm(ref_g[a:b]) + 1e-12, name


def test_gradients_deterministic(rt):
    import torch
    p, X, Y = _data(512, 3)
    pd, Xd, Yd = dev(p), dev(X), dev(Y)
    outs = []
    for _ in range(3):
        g = torch.zeros(R.MLP_NPARAM, dtype=torch.float32, device="cuda")
        rt.mlp_loss_grad(pd, Xd, Yd, g)
        outs.append(host(g).tobytes())
    assert len(set(outs)) == 1


def test_adam_vs_oracle(rt):
    import torch
    g = np.random.default_rng(4)
    p0 = g.normal(size=R.MLP_NPARAM)
    grads = [g.normal(size=R.MLP_NPARAM) for _ in range(4)]
    p, m, v = dev(p0.astype(np.float32)), torch.zeros(R.MLP_NPARAM, device="cuda"), \
        torch.zeros(R.MLP_NPARAM, device="cuda")
    rp, rm, rv = p0.astype(np.float32).astype(np.float64), np.zeros(R.MLP_NPARAM), \
        np.zeros(R.MLP_NPARAM)
    for t, gr in enumerate(grads, start=1):
        gf = gr.astype(np.float32)
        rt.mlp_adam(p, dev(gf), m, v, t, lr=1e-3)
        O.adam_step(rp, gf.astype(np.float64), rm, rv, t, lr=1e-3)
    assert np.max(np.abs(host(p) - rp)) <= 1e-6 * (1 + np.max(np.abs(rp)))


def test_training_reduces_loss(rt):
    """A few hundred Adam steps on a smooth synthetic target lower the loss."""
    import torch
    from paper_2106_03219_gb300 import learned
    g = np.random.default_rng(5)
    X = g.normal(size=(2048, 16)).astype(np.float32)
    W = g.normal(size=(16, 12)).astype(np.float32)
    Y = np.tanh(X @ W).astype(np.float32)
    p = dev(learned.init_params(0))
    grad, m, v = (torch.zeros_like(p) for _ in range(3))
    loss = torch.zeros(1, device="cuda")
    Xd, Yd = dev(X), dev(Y)
    rt.mlp_loss_grad(p, Xd, Yd, grad, loss)
    first = float(host(loss)[0])
    for t in range(1, 301):
        rt.mlp_loss_grad(p, Xd, Yd, grad, loss)
        rt.mlp_adam(p, grad, m, v, t, lr=3e-3)
    rt.mlp_loss_grad(p, Xd, Yd, grad, loss)
    assert float(host(loss)[0]) < 0.3 * first


def test_choose_config_fallbacks(rt):
    import torch
    x = torch.zeros(1 << 16, device="cuda")
    d = R.loop_desc(R.BODY_AXPY, n=1 << 16, x=x, y=x.clone())
    rt.set_cost_model(None)
    assert rt.choose_config(d, False) == 9                       # heuristic
    p = np.zeros(R.MLP_NPARAM, np.float32)
    p[-12:] = np.arange(12)[::-1]                                # bias only: argmin = 11
    rt.set_cost_model(p, np.zeros(16), np.ones(16))
    assert rt.choose_config(d, False) == 11
    p[-12:] = np.nan                                             # invalid output: heuristic
    rt.set_cost_model(p, np.zeros(16), np.ones(16))
    assert rt.choose_config(d, False) == 9
    rt.set_cost_model(None)
    f = rt.loop_features(d, False)
    assert f[0] == 16.0 and f[1] == 12.0 and f[3] == 1.0 and f[8] == 0.0
