"""The rounding model behind the tensor-core kernels' MMA order and output
scaling, checked on the CPU (numpy only; no GPU, no library code).

One transform stage 8C x (256 R)^T with split-FP16 operands is accumulated
as the tensor core does it: each MMA adds the exact sum of 16 products to an
FP32 accumulator and rounds the result toward zero.  Issuing the products of
every K block as hi*hi, hi*lo, lo*hi in turn shrinks the result by several
2^-24; issuing the small hi*lo and lo*hi products of all blocks first, then
the hi*hi ones, leaves fewer truncations at the accumulator's full size and a
smaller shrink; scaling the output by 1 + 2^-22 (what the kernels do at
N = 128) brings the remaining bias closer to zero."""
import numpy as np

F16, F32, F64 = np.float16, np.float32, np.float64
N = 128


def _split(x):
    x = x.astype(F32)
    hi = x.astype(F16)
    lo = (x - hi.astype(F32)).astype(F16)
    return hi.astype(F64), lo.astype(F64)


def _round_toward_zero(x):
    y = x.astype(F32)
    over = np.abs(y.astype(F64)) > np.abs(x)
    y[over] = np.nextafter(y[over], F32(0))
    return y.astype(F64)


def _dct():
    c = np.zeros((N, N))
    for k in range(N):
        c[k] = (np.sqrt(1 / N) if k == 0 else np.sqrt(2 / N)) * np.cos(
            np.pi * k * (np.arange(N) + 0.5) / N)
    return c


def _field(rng):
    x = np.arange(N) + 0.5
    r = sum(rng.normal() * np.cos(np.pi * kx * x[None, :] / N) * np.cos(np.pi * ky * x[:, None] / N)
            for kx, ky in rng.integers(0, 12, (6, 2)))
    return 0.3 * r / np.abs(r).max() + 0.01 * rng.standard_normal((N, N))


def _stage(ah, al, bh, bl, corrections_first):
    d = np.zeros((N, N))
    blocks = [slice(16 * k, 16 * k + 16) for k in range(N // 16)]
    if not corrections_first:
        for s in blocks:
            for a, b in ((ah, bh), (ah, bl), (al, bh)):
                d = _round_toward_zero(d + a[:, s] @ b[:, s].T)
        return d
    for s in blocks:
        for a, b in ((ah, bl), (al, bh)):
            d = _round_toward_zero(d + a[:, s] @ b[:, s].T)
    for s in blocks:
        d = _round_toward_zero(d + ah[:, s] @ bh[:, s].T)
    return d


def test_corrections_first_and_compensation_reduce_the_shrink():
    ah, al = _split(8 * _dct().astype(F32))
    rng = np.random.default_rng(0)
    for _ in range(3):
        bh, bl = _split(256 * _field(rng))
        exact = ah @ bh.T + ah @ bl.T + al @ bh.T  # exact products, exact sum

        def scale_error(d):
            return ((d * exact).sum() / (exact * exact).sum() - 1.0) / 2.0**-24

        mixed = scale_error(_stage(ah, al, bh, bl, False))
        first = scale_error(_stage(ah, al, bh, bl, True))
        comp = scale_error(_stage(ah, al, bh, bl, True) * (1.0 + 2.0**-22))
        assert mixed < -5.0                     # a shrink of several 2^-24
        assert mixed < first < 0.0 and abs(first) < 0.5 * abs(mixed)
        assert abs(comp) < abs(first)           # the 1 + 2^-22 scaling helps
