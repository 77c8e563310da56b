"""Pins of the FP64 numpy U-Net reference: its hand-written backward pass
against central finite differences of its own forward pass, on a tiny
network (8^3 voxels, base width 16), and the conv against a direct loop."""
import numpy as np
import pytest

from oracle import unet_ref as U


def test_conv3d_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 3, 4, 5, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    per = (1, 0, 1)
    y = U.conv3d(x, w, b, per, 27)
    nz, ny, nx = 3, 4, 5
    for (z, yy, xx, co) in [(0, 0, 0, 0), (2, 3, 4, 2), (1, 0, 2, 1), (0, 3, 0, 0)]:
        s = b[co]
        for t, (dx, dy, dz) in enumerate(U.TAPS27):
            X, Y, Z = xx + dx, yy + dy, z + dz
            X %= nx
            Z %= nz
            if not (0 <= Y < ny):
                continue
            s += w[co, t] @ x[0, Z, Y, X]
        assert abs(y[0, z, yy, xx, co] - s) < 1e-12


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(1)
    specs = U.layer_specs(cin=16, base=16, cout=16)
    params = U.init_params(rng, cin=16, base=16, cout=16, head_scale=1.0)
    # non-zero biases so that ReLU kinks are exercised away from zero
    for k in params:
        w, b = params[k]
        params[k] = (w, 0.05 * rng.standard_normal(b.shape))
    x = rng.standard_normal((1, 8, 8, 8, 16))
    t = rng.standard_normal((1, 8, 8, 8, 16))
    return specs, params, x, t


def _loss(specs, params, x, t, per):
    y, _ = U.forward(params, x, per, specs)
    return U.mse(y, t, 5, np.ones(16))[0]


@pytest.mark.parametrize("name,idx", [("c1a", (3, 13, 5)), ("c4b", (7, 0, 100)), ("c5a", (2, 26, 130)),
                                      ("c7b", (1, 4, 9)), ("head", (4, 0, 11))])
def test_backward_matches_finite_differences(tiny, name, idx):
    specs, params, x, t = tiny
    per = (1, 0, 1)
    y, cache = U.forward(params, x, per, specs)
    loss, gy = U.mse(y, t, 5, np.ones(16))
    grads = U.backward(params, cache, gy, per, specs)
    w, b = params[name]
    eps = 1e-6
    wp, wm = w.copy(), w.copy()
    wp[idx] += eps
    wm[idx] -= eps
    pp = dict(params)
    pp[name] = (wp, b)
    lp = _loss(specs, pp, x, t, per)
    pp[name] = (wm, b)
    lm = _loss(specs, pp, x, t, per)
    fd = (lp - lm) / (2 * eps)
    an = grads[name][0][idx]
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (fd, an)
    # bias of the same layer
    co = idx[0]
    bp, bm = b.copy(), b.copy()
    bp[co] += eps
    bm[co] -= eps
    pp[name] = (w, bp)
    lp = _loss(specs, pp, x, t, per)
    pp[name] = (w, bm)
    lm = _loss(specs, pp, x, t, per)
    assert abs((lp - lm) / (2 * eps) - grads[name][1][co]) <= 1e-6 * max(1.0, abs(grads[name][1][co])) + 1e-9
