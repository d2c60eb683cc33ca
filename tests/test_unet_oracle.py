"""Pins of the numpy U-Net oracle: central finite differences of its own forward pass
check its backward pass (weights, biases and input), and bf16 rounding is checked
against its definition on exactly representable values."""
import numpy as np

from oracle import unet_oracle as U


def test_bf16_rounding_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0], dtype=np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-8 ties to 1 + 2^-6
    want = [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0]
    assert np.array_equal(U.bf16_round(vals), np.array(want))


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    in_ch, out_ch, base, levels = 2, 2, 2, 2
    shapes = U.layer_shapes(in_ch, out_ch, base, levels)
    npar = sum(co * ci * 27 + co for ci, co in shapes)
    params = rng.standard_normal(npar) * 0.4
    x = rng.standard_normal((2, in_ch, 4, 4, 4))
    wout = rng.standard_normal((2, out_ch, 4, 4, 4))

    def f(par, xx):
        net = U.UNetOracle(par, in_ch, out_ch, base, levels, round_weights=False)
        return float((net.forward(xx) * wout).sum())

    net = U.UNetOracle(params, in_ch, out_ch, base, levels, round_weights=False)
    net.forward(x)
    gin, gpar = net.backward(wout)
    eps = 1e-6
    for k in rng.choice(npar, 40, replace=False):
        d = np.zeros(npar)
        d[k] = eps
        fd = (f(params + d, x) - f(params - d, x)) / (2 * eps)
        assert abs(fd - gpar[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gpar[k])
    for idx in [(0, 0, 1, 2, 3), (1, 1, 0, 0, 0), (0, 1, 3, 3, 1)]:
        d = np.zeros_like(x)
        d[idx] = eps
        fd = (f(params, x + d) - f(params, x - d)) / (2 * eps)
        assert abs(fd - gin[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_pool_and_upsample_are_adjoint_pairs():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((1, 2, 4, 4, 4))
    b = rng.standard_normal((1, 2, 2, 2, 2))
    # <pool(a), b> = <a, pool^T(b)> and <up(b), a> = <b, up^T(a)>
    assert np.isclose((U.pool(a) * b).sum(), (a * U.pool_backward(b)).sum())
    assert np.isclose((U.up(b) * a).sum(), (b * U.up_backward(a)).sum())
