"""The surrogate's tensor-core kernels and network against the FP64 numpy
reference (oracle/unet_ref.py).

* conv forward (3x3x3 and 1x1x1, periodic and zero padding, channel counts up
  to 384 in and 256 out) and weight gradient vs numpy on BF16-rounded
  inputs: FP32 accumulation, so the error is summation order (rel 1e-5);
* the whole U-Net (base width 16 on 16^3 voxels): output and every weight
  gradient vs the FP64 reference evaluated with the same BF16 weights and
  input; activations pass through BF16 between layers, so the bound is a
  relative L2 error of 4e-2 (BF16 carries 8 significant bits);
* 40 Adam steps on one pair lower the loss by at least a quarter.
"""
import ctypes

import numpy as np
import pytest

from oracle import unet_ref as U

pytestmark = pytest.mark.gpu


def _bf(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("dims,cin,cout,taps,per,relu", [
    ((8, 4, 4, 1), 16, 16, 1, 7, 0), ((8, 4, 4, 1), 16, 16, 27, 7, 0), ((8, 8, 4, 2), 32, 32, 27, 2, 1),
    ((16, 8, 4, 1), 64, 64, 27, 5, 1), ((8, 4, 8, 1), 96, 32, 27, 7, 0), ((8, 4, 4, 1), 384, 128, 27, 5, 1),
    ((8, 4, 4, 1), 128, 256, 27, 0, 1), ((9, 5, 3, 1), 32, 48, 27, 7, 0)])
def test_conv_forward(dims, cin, cout, taps, per, relu):
    import torch
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    rng = np.random.default_rng(cin * 7 + cout)
    nx, ny, nz, nb = dims
    X = _bf(rng.standard_normal((nb, nz, ny, nx, cin)))
    W = _bf(rng.standard_normal((cout, taps, cin)) / np.sqrt(taps * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).to(dev)
    Wd = torch.from_numpy(W.astype(np.float32)).to(torch.bfloat16).to(dev)
    bd = torch.from_numpy(b).to(dev)
    Yf = torch.zeros((nb, nz, ny, nx, cout), dtype=torch.float32, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    rc = lib.lbnn_conv3d_fwd(Xd.data_ptr(), cin, Wd.data_ptr(), taps, bd.data_ptr(), None, Yf.data_ptr(), cout, 0,
                             nx, ny, nz, nb, per, relu, st.data_ptr(), None)
    assert rc == 0, lib.lb_last_error()
    torch.cuda.synchronize()
    ref = U.conv3d(X, W, b.astype(np.float64), (per & 1, (per >> 1) & 1, (per >> 2) & 1), taps)
    if relu:
        ref = np.maximum(ref, 0)
    assert int(st[0].item()) == 0
    assert np.abs(Yf.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dims,cin,cout,per,relu,ldy", [
    ((8, 16, 4, 1), 16, 32, 7, 0, 0), ((16, 16, 4, 2), 32, 64, 5, 1, 0), ((8, 32, 2, 1), 96, 32, 2, 0, 0),
    ((8, 16, 3, 1), 64, 128, 0, 1, 0), ((8, 16, 4, 1), 384, 128, 5, 1, 0), ((16, 16, 4, 1), 128, 256, 7, 0, 0),
    ((8, 16, 8, 1), 32, 16, 7, 1, 0), ((8, 16, 4, 1), 32, 32, 5, 0, 64), ((8, 16, 2, 1), 128, 64, 7, 1, 0),
    ((16, 16, 2, 1), 192, 64, 5, 0, 0), ((32, 32, 320, 1), 16, 32, 5, 1, 0), ((32, 32, 320, 1), 48, 32, 2, 0, 0),
    ((32, 32, 160, 1), 64, 64, 7, 1, 0), ((16, 32, 24, 1), 256, 128, 5, 1, 0),
    ((32, 32, 48, 1), 64, 128, 7, 1, 0)])
def test_conv_forward_tiled(dims, cin, cout, per, relu, ldy):
    """Grids with nx % 8 == 0 and ny % 16 == 0 take the pipelined tiled kernel
    (input block staged once per channel chunk, TZ planes per work item, z
    taps merged into one UMMA when 3 Cout <= 256, Cout split in two slices
    when the grid is small); the same comparison as above, including a
    strided output (ldy > cout).  The 32 x 32 x 320 and 32 x 32 x 160 grids
    have more than twice as many work items as the GPU has SMs, so the
    persistent CTAs reuse both accumulator and both input buffers."""
    import torch
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    rng = np.random.default_rng(cin * 5 + cout + dims[2])
    nx, ny, nz, nb = dims
    X = _bf(rng.standard_normal((nb, nz, ny, nx, cin)))
    W = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).to(dev)
    Wd = torch.from_numpy(W.astype(np.float32)).to(torch.bfloat16).to(dev)
    bd = torch.from_numpy(b).to(dev)
    ld = ldy or cout
    Yf = torch.full((nb, nz, ny, nx, ld), 7.0, dtype=torch.float32, device=dev)
    Yb = torch.zeros((nb, nz, ny, nx, ld), dtype=torch.bfloat16, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    rc = lib.lbnn_conv3d_fwd(Xd.data_ptr(), cin, Wd.data_ptr(), 27, bd.data_ptr(), Yb.data_ptr(), Yf.data_ptr(), cout,
                             ldy, nx, ny, nz, nb, per, relu, st.data_ptr(), None)
    assert rc == 0, lib.lb_last_error()
    torch.cuda.synchronize()
    ref = U.conv3d(X, W, b.astype(np.float64), (per & 1, (per >> 1) & 1, (per >> 2) & 1), 27)
    if relu:
        ref = np.maximum(ref, 0)
    assert int(st[0].item()) == 0
    got = Yf.cpu().numpy()
    assert np.abs(got[..., :cout] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    if ld > cout:
        assert np.all(got[..., cout:] == 7.0)  # columns beyond cout untouched
    gb = Yb.float().cpu().numpy()[..., :cout]
    assert np.abs(gb - ref).max() <= 1e-2 * max(1.0, np.abs(ref).max())  # BF16 copy of the same values


@pytest.mark.parametrize("dims,cs,cl,cout,per", [
    ((16, 16, 4, 1), 32, 64, 32, 5), ((16, 32, 8, 1), 64, 128, 64, 7), ((8, 16, 4, 1), 128, 256, 128, 5),
    ((32, 32, 48, 2), 32, 64, 32, 2)])
def test_conv_forward_upcat(dims, cs, cl, cout, per):
    """The decoder convolution reading the skip tensor and the half-resolution
    tensor in place equals the convolution of their concatenation (nearest x2
    upsampling), against the FP64 reference."""
    import torch
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    rng = np.random.default_rng(cs + cl + cout + dims[2])
    nx, ny, nz, nb = dims
    skip = _bf(rng.standard_normal((nb, nz, ny, nx, cs)))
    low = _bf(rng.standard_normal((nb, nz // 2, ny // 2, nx // 2, cl)))
    up = low.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)
    X = np.concatenate([skip, up], axis=-1)
    W = _bf(rng.standard_normal((cout, 27, cs + cl)) / np.sqrt(27 * (cs + cl)))
    b = rng.standard_normal(cout).astype(np.float32)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(dev)
    Sd, Ld, Wd = t(skip), t(low), t(W)
    bd = torch.from_numpy(b).to(dev)
    Yf = torch.zeros((nb, nz, ny, nx, cout), dtype=torch.float32, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    rc = lib.lbnn_conv3d_fwd_upcat(Sd.data_ptr(), cs, Ld.data_ptr(), cl, Wd.data_ptr(), bd.data_ptr(), None,
                                   Yf.data_ptr(), cout, 0, nx, ny, nz, nb, per, 1, st.data_ptr(), None)
    assert rc == 0, lib.lb_last_error()
    torch.cuda.synchronize()
    ref = np.maximum(U.conv3d(X, W, b.astype(np.float64), (per & 1, (per >> 1) & 1, (per >> 2) & 1), 27), 0)
    assert int(st[0].item()) == 0
    assert np.abs(Yf.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dims,cin,cout,taps,per,vpc", [
    ((8, 4, 4, 1), 16, 16, 1, 7, 64), ((8, 4, 4, 1), 16, 32, 27, 7, 64), ((8, 8, 8, 1), 32, 64, 27, 5, 128),
    ((8, 4, 8, 2), 96, 32, 27, 2, 64), ((8, 4, 4, 1), 128, 256, 27, 5, 64),
    # nx % 8 == 0 and ny % 16 == 0: the pipelined kernel (x or dy as the halo operand,
    # channel slices and tap groups), including runs of many blocks per CTA
    ((16, 16, 4, 1), 32, 64, 27, 7, 64), ((8, 16, 6, 2), 96, 32, 27, 5, 64), ((8, 16, 4, 1), 384, 128, 27, 5, 64),
    ((16, 16, 2, 1), 128, 256, 27, 2, 64), ((8, 16, 4, 1), 16, 32, 27, 0, 64), ((32, 32, 64, 1), 32, 32, 27, 5, 64)])
def test_conv_weight_gradient(dims, cin, cout, taps, per, vpc):
    import torch
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    rng = np.random.default_rng(cin + 3 * cout)
    nx, ny, nz, nb = dims
    X = _bf(rng.standard_normal((nb, nz, ny, nx, cin)))
    G = _bf(rng.standard_normal((nb, nz, ny, nx, cout)))
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).to(dev)
    Gd = torch.from_numpy(G.astype(np.float32)).to(torch.bfloat16).to(dev)
    dW = torch.zeros((cout, taps, cin), dtype=torch.float32, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    rc = lib.lbnn_conv3d_wgrad(Gd.data_ptr(), cout, Xd.data_ptr(), cin, taps, dW.data_ptr(), nx, ny, nz, nb, per, vpc,
                               st.data_ptr(), None)
    assert rc == 0, lib.lb_last_error()
    torch.cuda.synchronize()
    _, ref, _ = U.conv3d_backward(X, np.zeros((cout, taps, cin)), G, (per & 1, (per >> 1) & 1, (per >> 2) & 1), taps)
    assert int(st[0].item()) == 0
    assert np.abs(dW.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(1e-30, np.linalg.norm(np.ravel(b))))


def test_unet_forward_and_gradients_match_reference():
    import torch
    from paper_2405_14551_gb300 import surrogate as S
    rng = np.random.default_rng(5)
    net = S.UNet(base=16, seed=3)
    specs = U.layer_specs(cin=16, base=16, cout=16)
    params = {}
    for name, ci, co, taps, relu in specs:
        w = _bf(rng.standard_normal((co, taps, ci)) * np.sqrt(2.0 / (taps * ci)))
        b = 0.05 * rng.standard_normal(co)
        params[name] = (w, b)
    net.load_parameters(params)
    shape = (16, 16, 16, 1)
    x = _bf(rng.standard_normal((1, 16, 16, 16, 16)))
    t = rng.standard_normal((1, 16, 16, 16, 16))
    dev = torch.device("cuda")
    xd = torch.from_numpy(x.reshape(-1, 16).astype(np.float32)).to(torch.bfloat16).to(dev)
    y = net.forward(xd, shape)
    per = (1, 0, 1)
    yr, cache = U.forward(params, x, per, specs)
    yg = y.cpu().numpy().reshape(yr.shape)
    assert _rel(yg, yr) < 4e-2
    loss, gy = U.mse(yr, t, 5, np.ones(16))
    gyd = torch.from_numpy(gy.reshape(-1, 16).astype(np.float32)).to(dev)
    net.backward(gyd)
    torch.cuda.synchronize()
    net.check_status()
    grads = U.backward(params, cache, gy, per, specs)
    for name in grads:
        gw = net.gw[name].cpu().numpy()
        gb = net.gb[name].cpu().numpy()
        assert _rel(gw, grads[name][0]) < 4e-2, name
        assert _rel(gb, grads[name][1]) < 4e-2, name


def test_training_lowers_the_loss():
    import torch
    from paper_2405_14551_gb300 import surrogate as S
    torch.manual_seed(0)
    shape = (32, 32, 32)
    rng = np.random.default_rng(0)
    dev = torch.device("cuda")
    f0 = torch.zeros((5, 32 * 32 * 32), dtype=torch.float32, device=dev)
    z, yy, xx = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
    phi0 = np.tanh((8 - np.sqrt((xx - 16) ** 2 + (yy - 16) ** 2 + (z - 14) ** 2)) / 1.5)
    phi1 = np.tanh((8 - np.sqrt((xx - 16) ** 2 + (yy - 16) ** 2 + (z - 16) ** 2)) / 1.5)
    f0[0] = torch.from_numpy(phi0.reshape(-1).astype(np.float32))
    f0[1] = 1.0
    f1 = f0.clone()
    f1[0] = torch.from_numpy(phi1.reshape(-1).astype(np.float32))
    net = S.UNet(base=16, seed=1)
    hist = S.train(net, [[f0, f1]], shape, iters=40, lr=2e-3, log_every=39)
    assert hist[-1][1] < 0.75 * hist[0][1], hist



def test_native_surrogate_matches_python_driver():
    """The native runtime (lb_surrogate_load / _predict / _cycle) runs the same
    kernels in the same order as the Python driver: bitwise equal candidate,
    accepted jumps rebuild the candidate by regularised reconstruction, a
    rejected judged jump leaves the plain-LB result, and the judged error is
    the mean |phi_candidate - phi_LB|."""
    import os
    import tempfile
    import torch
    import paper_2405_14551_gb300.lbcg as L
    from paper_2405_14551_gb300 import surrogate as S
    from paper_2405_14551_gb300 import workloads as W
    n, K = 32, 5
    p = dict(W.BASE, A_h=0.1, g=(0.0, 0.0, 1e-5), g_mode=1)
    stream = torch.cuda.current_stream()

    def make():
        s = L.Sim(n, n, n, walls=0b010, **p)
        s.init_droplets([[15.3, 14.2, 10.1], [16.2, 17.1, 23.4]], [6.0, 5.5])
        return s

    sim = make()
    sim.step(20)
    net = S.UNet(base=16, seed=4)  # untrained: small increments, the droplet count is kept
    f0 = sim.fields_device(S.FIELD_MASK).reshape(5, -1)
    x = torch.empty((n ** 3, S.CIN), dtype=torch.bfloat16, device="cuda")
    out_py = torch.empty((5, n ** 3), dtype=torch.float32, device="cuda")
    S.pack_input(f0, x, stream)
    y = net.forward(x, (n, n, n, 1))
    S.unpack_output(f0, y, out_py, stream)
    fd, path = tempfile.mkstemp(suffix=".lbnn")
    os.close(fd)
    try:
        net.save(path)
        L.lb_surrogate_load(sim.h, path)
        with pytest.raises(L.LBError):
            L.lb_surrogate_load(sim.h, path)  # one network per handle
    finally:
        os.remove(path)
    out_c = torch.empty((5, n ** 3), dtype=torch.float32, device="cuda")
    L.lb_surrogate_predict(sim.h, out_c)
    torch.cuda.synchronize()
    assert torch.equal(out_c, out_py)
    # rejected judged jump: the handle holds the plain-LB state K steps on
    judge = make()
    twin = make()
    L.lb_copy_state(twin.h, sim.h)
    twin.step(K)
    ok, err = L.lb_surrogate_cycle(sim.h, judge.h, K, 0.02, 0.0)
    assert not ok and err > 0
    phi_lb = twin.fields_device(1).reshape(-1)
    assert abs(err - float((out_py[0] - phi_lb).double().abs().mean())) < 1e-9
    ft, fs = twin.fields(), sim.fields()
    for k in ft:
        np.testing.assert_array_equal(fs[k], ft[k])
    # accepted jump (tolerances wide open): regularised reconstruction of the candidate
    L.lb_surrogate_predict(sim.h, out_c)
    torch.cuda.synchronize()
    ok, err = L.lb_surrogate_cycle(sim.h, judge.h, K, 1e9, 1e9)
    assert ok and err >= 0
    rec = make()
    rec.init_fields(out_c[0], out_c[1], out_c[2:5], regularised=True)
    fr, fs = rec.fields(), sim.fields()
    for k in fr:
        np.testing.assert_array_equal(fs[k], fr[k])
    assert sim.t == 0


@pytest.mark.parametrize("kind,dims", [("fwd", (12, 12, 4, 1)), ("fwd", (16, 16, 4, 1)),
                                       ("wgrad", (12, 12, 4, 1)), ("wgrad", (16, 16, 4, 1))])
def test_conv_bounded_wait_gives_up_cleanly(kind, dims):
    """With a wait limit of 0 every handshake wait of the convolutions gives
    up at its first poll (12 x 12 grids take the two-buffer kernels, whose
    third channel chunk waits for the first one's UMMAs; 16 x 16 grids take
    the warp-specialised kernels, whose UMMA and epilogue roles wait for the
    copies).  The kernel must then drain what it committed, free its tensor
    memory and return: the status word carries bit 4, lbnn_check_status maps
    it to LB_ETIMEOUT and clears it, the output is left unwritten, and the
    same call with the default limit right after gives the reference result
    on the same context."""
    import torch
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    rng = np.random.default_rng(11)
    nx, ny, nz, nb = dims
    cin, cout = 32, 32
    X = _bf(rng.standard_normal((nb, nz, ny, nx, cin)))
    W = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    G = _bf(rng.standard_normal((nb, nz, ny, nx, cout)))
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).to(dev)
    Wd = torch.from_numpy(W.astype(np.float32)).to(torch.bfloat16).to(dev)
    Gd = torch.from_numpy(G.astype(np.float32)).to(torch.bfloat16).to(dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    out = (torch.full((nb, nz, ny, nx, cout), 7.0, dtype=torch.float32, device=dev) if kind == "fwd"
           else torch.zeros((cout, 27, cin), dtype=torch.float32, device=dev))

    def call():
        if kind == "fwd":
            return lib.lbnn_conv3d_fwd(Xd.data_ptr(), cin, Wd.data_ptr(), 27, None, None, out.data_ptr(), cout, 0,
                                       nx, ny, nz, nb, 7, 0, st.data_ptr(), None)
        # 192 voxels per CTA: three chunks of 64, so the third one waits
        return lib.lbnn_conv3d_wgrad(Gd.data_ptr(), cout, Xd.data_ptr(), cin, 27, out.data_ptr(), nx, ny, nz, nb, 7,
                                     192, st.data_ptr(), None)

    prev = L.lbnn_set_wait_limit(0)
    try:
        assert call() == 0, lib.lb_last_error()
        torch.cuda.synchronize()
        assert int(st[0].item()) & 16
        with pytest.raises(L.LBError) as e:
            L.lbnn_check_status(st.data_ptr())
        assert e.value.code == L.LB_ETIMEOUT
        assert int(st[0].item()) == 0  # cleared by the check
    finally:
        L.lbnn_set_wait_limit(prev)
    before = out.cpu().numpy()
    assert np.all(before == (7.0 if kind == "fwd" else 0.0))  # nothing written after the give-up
    assert call() == 0, lib.lb_last_error()
    L.lbnn_check_status(st.data_ptr())
    got = out.cpu().numpy()
    if kind == "fwd":
        ref = U.conv3d(X, W, np.zeros(cout), (1, 1, 1), 27)
    else:
        _, ref, _ = U.conv3d_backward(X, np.zeros((cout, 27, cin)), G, (1, 1, 1), 27)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
