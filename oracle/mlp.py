"""FP64 surrogate network: forward, backward, Adam (TEST INFRASTRUCTURE ONLY).

The surrogate of the delayed-acceptance sampler (not in the paper; it follows
Christen & Fox 2005) is a multilayer perceptron
    x -> SiLU(W1 x + b1) -> SiLU(W2 . + b2) -> SiLU(W3 . + b3) -> W4 . + b4,
SiLU(z) = z / (1 + exp(-z)), with inputs x_i = (log theta_i - mu_i) / s_i and
output mapped to a log-likelihood by
    Phi~(theta) = floor + exp(shift + scale * net(x)).
Training minimises the mean squared error (1/B) sum (net(x) - z)^2 on
z = (log(Phi - floor) - shift) / scale with Adam (Kingma & Ba 2015) and
decoupled weight decay (Loshchilov & Hutter 2019).

Parity: forward and backward are pinned against torch autograd in float64
(a library routine) and central finite differences; Adam against a hand-run
two-step example.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(widths, seed):
    """He-uniform initial weights for layer widths e.g. (4, 256, 256, 256, 1)."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        bound = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-bound, bound, size=(fan_out, fan_in))
        b = np.zeros(fan_out)
        params.append([W, b])
    params[-1][0] *= 0.1
    return params


def forward(params, x):
    """Returns (out [B], cache) for inputs x [B][in]."""
    pre, act = [], [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = z if li == len(params) - 1 else silu(z)
        act.append(h)
    return h[:, 0], (pre, act)


def loss_and_grads(params, x, target):
    """MSE loss (1/B) sum (out - target)^2 and its gradient for every W, b."""
    out, (pre, act) = forward(params, x)
    B = x.shape[0]
    err = out - target
    loss = float(np.mean(err * err))
    g = (2.0 / B) * err[:, None]
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li != len(params) - 1:
            g = g * silu_grad(pre[li])
        gW = g.T @ act[li]
        gb = g.sum(axis=0)
        grads[li] = [gW, gb]
        g = g @ W
    return loss, grads


class Adam:
    """Adam with bias correction and decoupled weight decay on the weights."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, beta1, beta2, eps, wd
        self.t = 0
        self.m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for li, (p, g) in enumerate(zip(params, grads)):
            for j in range(2):
                m = self.m[li][j] = self.b1 * self.m[li][j] + (1 - self.b1) * g[j]
                v = self.v[li][j] = self.b2 * self.v[li][j] + (1 - self.b2) * g[j] ** 2
                if j == 0 and self.wd:
                    p[j] -= self.lr * self.wd * p[j]
                p[j] -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)


def features(theta, in_mu, in_sd):
    return (np.log(theta) - in_mu) / in_sd


def surrogate_phi(params, theta, norm):
    """Phi~(theta) for theta [B][P]; norm = dict(in_mu, in_sd, floor, shift, scale)."""
    x = features(np.atleast_2d(theta), norm["in_mu"], norm["in_sd"])
    out, _ = forward(params, x)
    return norm["floor"] + np.exp(norm["shift"] + norm["scale"] * out)


# ---------------------------------------------------------------------------
# Flat parameter layout of the GPU library (width W, 16 padded inputs):
# W1 [W][16], b1 [W], W2 [W][W], b2 [W], W3 [W][W], b3 [W], W4 [W], b4 [1].
# ---------------------------------------------------------------------------
N_IN = 16


def flat_layout(W):
    sizes = [("W1", (W, N_IN)), ("b1", (W,)), ("W2", (W, W)), ("b2", (W,)),
             ("W3", (W, W)), ("b3", (W,)), ("W4", (1, W)), ("b4", (1,))]
    out, off = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


def unflatten(flat, W):
    lay, _ = flat_layout(W)
    get = lambda k: np.asarray(flat[lay[k][0]: lay[k][0] + int(np.prod(lay[k][1]))],
                               dtype=np.float64).reshape(lay[k][1])
    return [[get("W1"), get("b1")], [get("W2"), get("b2")], [get("W3"), get("b3")],
            [get("W4"), get("b4")]]


def flatten(params):
    return np.concatenate([np.ravel(a) for layer in params for a in layer])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even) via float32, as the GPU
    rounds its FP32 values; returned as float64."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grads_bf16(params, x, target, rnd=bf16_round):
    """MSE loss and gradients with the network evaluated at the precision the
    tensor-core kernels use: BF16 inputs, weights W1-W3, hidden activations
    and backpropagated dZ; FP32 (here FP64) accumulation, pre-activations
    and the last layer.  With rnd = identity this is loss_and_grads."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = params
    B = x.shape[0]
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64) if rnd is not _ident else a
    xb = rnd(x)
    W1b, W2b, W3b = rnd(W1), rnd(W2), rnd(W3)
    z1 = f32(xb @ W1b.T + b1)
    h1 = rnd(silu(z1))
    z2 = f32(h1 @ W2b.T + b2)
    h2 = rnd(silu(z2))
    z3 = f32(h2 @ W3b.T + b3)
    h3 = rnd(silu(z3))
    out = h3 @ W4[0] + b4[0]
    err = out - target
    loss = float(np.mean(err * err))
    dout = 2.0 * err / B
    dz3 = rnd(dout[:, None] * W4[0][None, :] * silu_grad(z3))
    g = {"W4": (dout @ h3)[None, :], "b4": np.array([dout.sum()]),
         "W3": dz3.T @ h2, "b3": dz3.sum(0)}
    dz2 = rnd((dz3 @ W3b) * silu_grad(z2))
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = rnd((dz2 @ W2b) * silu_grad(z1))
    g["W1"], g["b1"] = dz1.T @ xb, dz1.sum(0)
    grads = [[g["W1"], g["b1"]], [g["W2"], g["b2"]], [g["W3"], g["b3"]], [g["W4"], g["b4"]]]
    return loss, grads, out


def _ident(a):
    return np.asarray(a, dtype=np.float64)
