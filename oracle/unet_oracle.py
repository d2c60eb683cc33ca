"""Plain numpy (FP64) oracle of the learned coarse correction's U-Net.

TEST INFRASTRUCTURE ONLY (imported by the tests).  Not in the paper: the
network gives the paper's Additive-Schwarz preconditioner a coarse space.

Architecture (same definition as the library's): `levels` resolution levels
with channels ch(l) = min(base * 2^l, 4 * base); per encoder level two 3x3x3
convolutions (zero padding) each followed by ReLU; 2x average pooling between
levels; per decoder level nearest 2x upsampling of the level below,
concatenation [upsampled, skip] along channels, two convolutions + ReLU; a
final 3x3x3 convolution to out_ch channels without ReLU.  The forward pass
uses the weights rounded to bfloat16 (round to nearest even).

Parameter vector layout, layer by layer (encoder a, b per level top-down;
decoder a, b per level from the second-lowest up; output layer): the layer's
weights [cout][cin][27] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) then its biases.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(in_ch, out_ch, base, levels):
    ch = lambda l: min(base << l, 4 * base)
    shapes = []
    for l in range(levels):
        shapes.append((in_ch if l == 0 else ch(l - 1), ch(l)))
        shapes.append((ch(l), ch(l)))
    for l in range(levels - 2, -1, -1):
        shapes.append((ch(l + 1) + ch(l), ch(l)))
        shapes.append((ch(l), ch(l)))
    shapes.append((ch(0), out_ch))
    return shapes


def unpack(params, shapes):
    layers = []
    off = 0
    for cin, cout in shapes:
        w = params[off: off + cout * cin * 27].reshape(cout, cin, 27)
        off += cout * cin * 27
        b = params[off: off + cout]
        off += cout
        layers.append((w, b))
    assert off == len(params)
    return layers


def _shift(x, dz, dy, dx):
    """y[..., z, y, x] = x[..., z+dz, y+dy, x+dx] with zeros outside."""
    out = np.zeros_like(x)
    Z, Y, X = x.shape[-3:]
    zs, ze = max(0, -dz), min(Z, Z - dz)
    ys, ye = max(0, -dy), min(Y, Y - dy)
    xs, xe = max(0, -dx), min(X, X - dx)
    out[..., zs:ze, ys:ye, xs:xe] = x[..., zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(x, w, b):
    """x: [B, Cin, Z, Y, X]; w: [Cout, Cin, 27]; b: [Cout]."""
    out = np.zeros((x.shape[0], w.shape[0]) + x.shape[2:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += np.einsum("oi,bizyx->bozyx", w[:, :, t], _shift(x, dz, dy, dx))
    return out + b[None, :, None, None, None]


def conv3_backward(x, w, gout):
    """Gradients of conv3 with respect to x, w and b."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        gw[:, :, t] = np.einsum("bozyx,bizyx->oi", gout, xs)
        # out[p] gets w * x[p + d]  =>  x[q] receives w * gout[q - d]
        gx += _shift(np.einsum("oi,bozyx->bizyx", w[:, :, t], gout), -dz, -dy, -dx)
    gb = gout.sum(axis=(0, 2, 3, 4))
    return gx, gw, gb


def pool(x):
    B, C, Z, Y, X = x.shape
    return x.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(3, 5, 7))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=2), 2, axis=3), 2, axis=4) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=2), 2, axis=3), 2, axis=4)


def up_backward(g):
    B, C, Z, Y, X = g.shape
    return g.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(3, 5, 7))


class UNetOracle:
    def __init__(self, params, in_ch, out_ch, base, levels, round_weights=True):
        self.L = levels
        self.shapes = layer_shapes(in_ch, out_ch, base, levels)
        if round_weights:
            # forward weights in bfloat16, biases in FP32 (what the GPU forward pass uses)
            raw = unpack(np.asarray(params, dtype=np.float32), self.shapes)
            self.layers = [(bf16_round(w), b.astype(np.float64)) for w, b in raw]
        else:
            self.layers = unpack(np.asarray(params, dtype=np.float64), self.shapes)

    def _enc(self, l, k):
        return 2 * l + k

    def _dec(self, l, k):
        return 2 * self.L + 2 * (self.L - 2 - l) + k

    def forward(self, x):
        L = self.L
        c = {}
        c["in"] = x
        h = x
        for l in range(L):
            if l > 0:
                h = pool(c[("eB", l - 1)])
            c[("xin", l)] = h
            wa, ba = self.layers[self._enc(l, 0)]
            c[("ea", l)] = conv3(h, wa, ba)
            c[("eA", l)] = np.maximum(c[("ea", l)], 0)
            wb, bb = self.layers[self._enc(l, 1)]
            c[("eb", l)] = conv3(c[("eA", l)], wb, bb)
            c[("eB", l)] = np.maximum(c[("eb", l)], 0)
        prev = c[("eB", L - 1)]
        for l in range(L - 2, -1, -1):
            c[("cat", l)] = np.concatenate([up(prev), c[("eB", l)]], axis=1)
            wa, ba = self.layers[self._dec(l, 0)]
            c[("da", l)] = conv3(c[("cat", l)], wa, ba)
            c[("dA", l)] = np.maximum(c[("da", l)], 0)
            wb, bb = self.layers[self._dec(l, 1)]
            c[("db", l)] = conv3(c[("dA", l)], wb, bb)
            c[("dB", l)] = np.maximum(c[("db", l)], 0)
            prev = c[("dB", l)]
        c["top"] = prev
        w, b = self.layers[-1]
        out = conv3(prev, w, b)
        self.cache = c
        return out

    def backward(self, gout):
        """Returns (d input, d params in the packed layout)."""
        L = self.L
        c = self.cache
        grads = [None] * len(self.layers)
        w, _ = self.layers[-1]
        gtop, gw, gb = conv3_backward(c["top"], w, gout)
        grads[-1] = (gw, gb)
        geB = {l: np.zeros_like(c[("eB", l)]) for l in range(L)}
        g_prev = gtop
        if L == 1:
            geB[0] += gtop
        for l in range(0, L - 1):
            cu = c[("eB", l + 1)].shape[1] if l + 1 == L - 1 else c[("dB", l + 1)].shape[1]
            gdb = g_prev * (c[("db", l)] > 0)
            wb, _ = self.layers[self._dec(l, 1)]
            gdA, gw, gb = conv3_backward(c[("dA", l)], wb, gdb)
            grads[self._dec(l, 1)] = (gw, gb)
            gda = gdA * (c[("da", l)] > 0)
            wa, _ = self.layers[self._dec(l, 0)]
            gcat, gw, gb = conv3_backward(c[("cat", l)], wa, gda)
            grads[self._dec(l, 0)] = (gw, gb)
            geB[l] += gcat[:, cu:]
            g_below = up_backward(gcat[:, :cu])
            if l + 1 == L - 1:
                geB[L - 1] += g_below
            else:
                g_prev = g_below
        gin = None
        for l in range(L - 1, -1, -1):
            geb = geB[l] * (c[("eb", l)] > 0)
            wb, _ = self.layers[self._enc(l, 1)]
            geA, gw, gb = conv3_backward(c[("eA", l)], wb, geb)
            grads[self._enc(l, 1)] = (gw, gb)
            gea = geA * (c[("ea", l)] > 0)
            wa, _ = self.layers[self._enc(l, 0)]
            gx, gw, gb = conv3_backward(c[("xin", l)], wa, gea)
            grads[self._enc(l, 0)] = (gw, gb)
            if l > 0:
                geB[l - 1] += pool_backward(gx)
            else:
                gin = gx
        flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
        return gin, flat
