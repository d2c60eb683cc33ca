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


def _direct_conv3(x, w, b):
    """out[n, o, z, y, x] = b[o] + sum over i and the 27 neighbours (z+dz, y+dy, x+dx) inside the
    grid of w[o, i, (dz+1)*9 + (dy+1)*3 + (dx+1)] * x[n, i, z+dz, y+dy, x+dx]: the definition, point by
    point, with the zero padding written as a bounds test."""
    N, C, Z, Y, X = x.shape
    O = w.shape[0]
    out = np.zeros((N, O, Z, Y, X))
    for n in range(N):
        for o in range(O):
            for z in range(Z):
                for y in range(Y):
                    for xx in range(X):
                        s = b[o]
                        for i in range(C):
                            for dz in (-1, 0, 1):
                                for dy in (-1, 0, 1):
                                    for dx in (-1, 0, 1):
                                        zz, yy, x2 = z + dz, y + dy, xx + dx
                                        if 0 <= zz < Z and 0 <= yy < Y and 0 <= x2 < X:
                                            s += w[o, i, (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] * x[n, i, zz, yy, x2]
                        out[n, o, z, y, xx] = s
    return out


def test_conv3_equals_the_direct_27_tap_sum():
    # a 3x4x5 grid (every voxel touches the boundary on some axis) with 2 -> 3 channels
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    assert np.abs(U.conv3(x, w, b) - _direct_conv3(x, w, b)).max() < 1e-12


def test_conv3_backward_equals_the_adjoint_of_the_direct_sum():
    # the direct sum is linear in x and in w: its gradients are the columns of the linear maps
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, 2, 3, 3, 4))
    w = rng.standard_normal((2, 2, 27))
    g = rng.standard_normal((1, 2, 3, 3, 4))
    gx, gw, gb = U.conv3_backward(x, w, g)
    zero_b = np.zeros(2)
    for idx in [(0, 0, 0, 0, 0), (0, 1, 2, 1, 3), (0, 0, 1, 2, 0)]:
        e = np.zeros_like(x)
        e[idx] = 1.0
        assert abs((_direct_conv3(e, w, zero_b) * g).sum() - gx[idx]) < 1e-12
    for o, i, t in [(0, 0, 0), (1, 1, 13), (0, 1, 26), (1, 0, 5)]:
        e = np.zeros_like(w)
        e[o, i, t] = 1.0
        assert abs((_direct_conv3(x, e, zero_b) * g).sum() - gw[o, i, t]) < 1e-12
    assert np.allclose(gb, g.sum(axis=(0, 2, 3, 4)))
