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
