"""FP64 numpy reference of the surrogate network (test infrastructure only).

A plain 3-D U-Net in channels-last layout x[b, z, y, x, c]: per level two
3x3x3 convolutions with ReLU, 2x2x2 average pooling down, nearest x2
upsampling concatenated after the skip tensor up, and a 1x1x1 head without
activation.  Convolutions wrap periodic axes and pad the others with zeros.
The backward pass is written out by hand; tests pin it with finite
differences and compare the GPU kernels' gradients with it.  It shares no
code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

TAPS27 = [((t % 3) - 1, ((t // 3) % 3) - 1, t // 9 - 1) for t in range(27)]


def _shift(x, d, axis, periodic):
    """y[..., i, ...] = x[..., i + d, ...] along axis (wrap or zero pad)."""
    if d == 0:
        return x
    y = np.roll(x, -d, axis=axis)
    if not periodic:
        sl = [slice(None)] * x.ndim
        sl[axis] = slice(-1, None) if d > 0 else slice(0, 1)
        y[tuple(sl)] = 0.0
    return y


def conv3d(x, w, b, periodic, taps):
    """y[v, co] = b[co] + sum_t sum_ci w[co, t, ci] x[v + off_t, ci]."""
    offs = TAPS27 if taps == 27 else [(0, 0, 0)]
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for t, (dx, dy, dz) in enumerate(offs):
        xs = _shift(_shift(_shift(x, dx, 3, periodic[0]), dy, 2, periodic[1]), dz, 1, periodic[2])
        y += np.einsum("bzyxc,oc->bzyxo", xs, w[:, t, :])
    if b is not None:
        y += b
    return y


def conv3d_backward(x, w, gpre, periodic, taps):
    """Gradients of conv3d w.r.t. x, w, b given dL/dy (pre-activation)."""
    offs = TAPS27 if taps == 27 else [(0, 0, 0)]
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (ox, oy, oz) in enumerate(offs):
        xs = _shift(_shift(_shift(x, ox, 3, periodic[0]), oy, 2, periodic[1]), oz, 1, periodic[2])
        dw[:, t, :] = np.einsum("bzyxo,bzyxc->oc", gpre, xs)
        # x[v + off] receives w^T g[v]: shift back by -off
        contrib = np.einsum("bzyxo,oc->bzyxc", gpre, w[:, t, :])
        dx += _shift(_shift(_shift(contrib, -ox, 3, periodic[0]), -oy, 2, periodic[1]), -oz, 1, periodic[2])
    db = gpre.sum(axis=(0, 1, 2, 3))
    return dx, dw, db


def avgpool2(x):
    b, z, y, xx, c = x.shape
    return x.reshape(b, z // 2, 2, y // 2, 2, xx // 2, 2, c).mean(axis=(2, 4, 6))


def avgpool2_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up_concat(skip, low):
    up = np.repeat(np.repeat(np.repeat(low, 2, axis=1), 2, axis=2), 2, axis=3)
    return np.concatenate([skip, up], axis=-1)


def up_concat_backward(g, cs):
    gs = g[..., :cs]
    gu = g[..., cs:]
    b, z, y, x, c = gu.shape
    gl = gu.reshape(b, z // 2, 2, y // 2, 2, x // 2, 2, c).sum(axis=(2, 4, 6))
    return gs, gl


def layer_specs(cin=16, base=32, cout=16):
    """(name, cin, cout, taps, relu) of every convolution, in forward order."""
    c1, c2, c3, c4 = base, 2 * base, 4 * base, 8 * base
    return [("c1a", cin, c1, 27, True), ("c1b", c1, c1, 27, True),
            ("c2a", c1, c2, 27, True), ("c2b", c2, c2, 27, True),
            ("c3a", c2, c3, 27, True), ("c3b", c3, c3, 27, True),
            ("c4a", c3, c4, 27, True), ("c4b", c4, c4, 27, True),
            ("c5a", c3 + c4, c3, 27, True), ("c5b", c3, c3, 27, True),
            ("c6a", c2 + c3, c2, 27, True), ("c6b", c2, c2, 27, True),
            ("c7a", c1 + c2, c1, 27, True), ("c7b", c1, c1, 27, True),
            ("head", c1, cout, 1, False)]


def init_params(rng, cin=16, base=32, cout=16, head_scale=0.1):
    params = {}
    for name, ci, co, taps, relu in layer_specs(cin, base, cout):
        std = np.sqrt(2.0 / (taps * ci)) * (head_scale if name == "head" else 1.0)
        params[name] = (rng.standard_normal((co, taps, ci)) * std, np.zeros(co))
    return params


def forward(params, x, periodic, specs):
    """Returns (y, cache) with every layer's input and output."""
    sp = {s[0]: s for s in specs}
    cache = {}

    def conv(name, inp):
        _, ci, co, taps, relu = sp[name]
        w, b = params[name]
        pre = conv3d(inp, w, b, periodic, taps)
        out = np.maximum(pre, 0.0) if relu else pre
        cache[name] = (inp, out)
        return out

    s1 = conv("c1b", conv("c1a", x))
    s2 = conv("c2b", conv("c2a", avgpool2(s1)))
    s3 = conv("c3b", conv("c3a", avgpool2(s2)))
    b4 = conv("c4b", conv("c4a", avgpool2(s3)))
    d3 = conv("c5b", conv("c5a", up_concat(s3, b4)))
    d2 = conv("c6b", conv("c6a", up_concat(s2, d3)))
    d1 = conv("c7b", conv("c7a", up_concat(s1, d2)))
    y = conv("head", d1)
    cache["skips"] = (s1, s2, s3)
    return y, cache


def backward(params, cache, gy, periodic, specs):
    """Gradients {name: (dW, db)} for dL/dy = gy."""
    sp = {s[0]: s for s in specs}
    grads = {}

    def conv_b(name, g):
        _, ci, co, taps, relu = sp[name]
        inp, out = cache[name]
        gpre = g * (out > 0) if relu else g
        dx, dw, db = conv3d_backward(inp, params[name][0], gpre, periodic, taps)
        grads[name] = (dw, db)
        return dx

    s1, s2, s3 = cache["skips"]
    g_d1 = conv_b("head", gy)
    g_u1 = conv_b("c7a", conv_b("c7b", g_d1))
    g_s1, g_d2 = up_concat_backward(g_u1, s1.shape[-1])
    g_u2 = conv_b("c6a", conv_b("c6b", g_d2))
    g_s2, g_d3 = up_concat_backward(g_u2, s2.shape[-1])
    g_u3 = conv_b("c5a", conv_b("c5b", g_d3))
    g_s3, g_b4 = up_concat_backward(g_u3, s3.shape[-1])
    g_p3 = conv_b("c4a", conv_b("c4b", g_b4))
    g_s3 = g_s3 + avgpool2_backward(g_p3)
    g_p2 = conv_b("c3a", conv_b("c3b", g_s3))
    g_s2 = g_s2 + avgpool2_backward(g_p2)
    g_p1 = conv_b("c2a", conv_b("c2b", g_s2))
    g_s1 = g_s1 + avgpool2_backward(g_p1)
    conv_b("c1a", conv_b("c1b", g_s1))
    return grads


def mse(y, t, nch, wch):
    """Weighted MSE over the first nch channels and its gradient."""
    n = y[..., 0].size * nch
    d = (y - t)[..., :nch]
    loss = float((wch[:nch] * d * d).sum() / n)
    g = np.zeros_like(y)
    g[..., :nch] = 2.0 * wch[:nch] * d / n
    return loss, g
