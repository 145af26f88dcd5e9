"""Pins of the oracle's FP64 surrogate network (no GPU): forward and backward
against torch autograd in float64 (a library routine), gradients against
central finite differences, and the optimizer against torch's AdamW."""
import numpy as np
import pytest
import torch

from oracle import mlp

WIDTHS = (4, 16, 16, 16, 1)


def _torch_net(params):
    layers = []
    for li, (W, b) in enumerate(params):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
        if li != len(params) - 1:
            layers.append(torch.nn.SiLU())
    return torch.nn.Sequential(*layers)


def _setup(seed=0, B=32):
    params = mlp.init_params(WIDTHS, seed)
    for W, b in params:
        b += np.random.default_rng(seed + 1).normal(0, 0.1, b.shape)
    rng = np.random.default_rng(seed + 2)
    return params, rng.standard_normal((B, 4)), rng.standard_normal(B)


def test_forward_backward_match_torch_float64():
    params, x, z = _setup()
    out, _ = mlp.forward(params, x)
    loss, grads = mlp.loss_and_grads(params, x, z)
    net = _torch_net(params)
    xt = torch.from_numpy(x)
    ot = net(xt)[:, 0]
    lt = ((ot - torch.from_numpy(z)) ** 2).mean()
    lt.backward()
    assert np.allclose(out, ot.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (gW, gb), lin in zip(grads, lins):
        assert np.allclose(gW, lin.weight.grad.numpy(), rtol=1e-11, atol=1e-13)
        assert np.allclose(gb, lin.bias.grad.numpy(), rtol=1e-11, atol=1e-13)


def test_gradients_central_differences():
    params, x, z = _setup(seed=3, B=8)
    _, grads = mlp.loss_and_grads(params, x, z)
    rng = np.random.default_rng(4)
    eps = 1e-6
    for li in range(len(params)):
        for j in range(2):
            P = params[li][j]
            for _ in range(3):
                idx = tuple(rng.integers(0, s) for s in P.shape)
                old = P[idx]
                P[idx] = old + eps
                lp, _ = mlp.loss_and_grads(params, x, z)
                P[idx] = old - eps
                lm, _ = mlp.loss_and_grads(params, x, z)
                P[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert grads[li][j][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_adam_matches_torch_adamw():
    params, x, z = _setup(seed=5)
    net = _torch_net(params)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    opt_t = torch.optim.AdamW([
        {"params": [l.weight for l in lins], "weight_decay": 0.01},
        {"params": [l.bias for l in lins], "weight_decay": 0.0}],
        lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
    opt = mlp.Adam(params, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8, wd=0.01)
    xt, zt = torch.from_numpy(x), torch.from_numpy(z)
    for _ in range(3):
        _, grads = mlp.loss_and_grads(params, x, z)
        opt.step(params, grads)
        opt_t.zero_grad()
        ((net(xt)[:, 0] - zt) ** 2).mean().backward()
        opt_t.step()
    for (W, b), lin in zip(params, lins):
        assert np.allclose(W, lin.weight.detach().numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(b, lin.bias.detach().numpy(), rtol=1e-10, atol=1e-12)


def test_training_reduces_loss():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((256, 4))
    z = np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2]
    params = mlp.init_params(WIDTHS, 1)
    opt = mlp.Adam(params, lr=3e-3)
    l0, _ = mlp.loss_and_grads(params, x, z)
    for _ in range(300):
        _, g = mlp.loss_and_grads(params, x, z)
        opt.step(params, g)
    l1, _ = mlp.loss_and_grads(params, x, z)
    assert l1 < 0.2 * l0


def test_bf16_round_matches_torch():
    x = np.random.default_rng(9).standard_normal(10000) * 10.0 ** np.random.default_rng(10).uniform(-5, 5, 10000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_bf16_emulation_reduces_to_fp64_network():
    """With the identity in place of BF16 rounding the emulated network is the
    FP64 network (pinned against torch above); with rounding it stays close."""
    rng = np.random.default_rng(11)
    W = 32
    params = mlp.init_params((mlp.N_IN, W, W, W, 1), 3)
    for layer in params:
        layer[1] += rng.normal(0, 0.1, layer[1].shape)
    x = np.zeros((64, mlp.N_IN))
    x[:, :4] = rng.standard_normal((64, 4))
    z = rng.standard_normal(64)
    l0, g0 = mlp.loss_and_grads(params, x, z)
    l1, g1, _ = mlp.loss_and_grads_bf16(params, x, z, rnd=mlp._ident)
    assert l1 == pytest.approx(l0, rel=1e-13)
    for (a, b), (c, d) in zip(g0, g1):
        assert np.allclose(a, c, rtol=1e-12, atol=1e-14) and np.allclose(b, d, rtol=1e-12, atol=1e-14)
    l2, g2, _ = mlp.loss_and_grads_bf16(params, x, z)
    assert l2 == pytest.approx(l0, rel=0.05)
    flat0, flat2 = mlp.flatten(g0), mlp.flatten(g2)
    assert np.linalg.norm(flat2 - flat0) < 0.05 * np.linalg.norm(flat0)


def test_flat_layout_roundtrip():
    W = 8
    _, n = mlp.flat_layout(W)
    flat = np.arange(n, dtype=np.float64)
    assert np.array_equal(mlp.flatten(mlp.unflatten(flat, W)), flat)
