"""Learned surrogate: a 3-D U-Net that advances (phi, rho, u) by K lattice
Boltzmann steps, trained and run with the library's own kernels.

Every tensor operation is a call into liblbcg.so (include/lbnn.h): tcgen05
implicit-GEMM convolutions for the forward pass and the input gradient
(with flipped weights), tcgen05 weight gradients, and element-wise kernels
for pooling, upsampling with skip concatenation, ReLU masks, bias
gradients, the MSE loss and Adam.  PyTorch only provides device memory and
the stream.  After a jump, the populations are rebuilt by the library's
regularised reconstruction (lb_init_fields with regularised = 1).

Network: 4 levels (base, 2 base, 4 base, 8 base channels), two 3x3x3
convolutions with ReLU per level and side, 2x2x2 average pooling, nearest x2
upsampling concatenated after the skip tensor, and a 1x1x1 head predicting
the scaled increments of (phi, rho, ux, uy, uz).  Weights: BF16 for the
kernels, FP32 master copies for Adam.  Convolutions wrap x and z (periodic)
and zero-pad y (walls).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import lbcg as L

CIN = 16          # input channels (5 fields, zero padded to a multiple of 16)
COUT = 16         # head channels (first 5 used)
S_RHO = 100.0     # scale of rho - 1 and its increments
S_U = 100.0       # scale of u and its increments
PERIODIC = 0b101  # x and z periodic, y walls


def layer_table(base=32, cin=CIN, cout=COUT):
    """(name, cin, cout, taps, relu) of every convolution, in forward order."""
    c1, c2, c3, c4 = base, 2 * base, 4 * base, 8 * base
    return [("c1a", cin, c1, 27, 1), ("c1b", c1, c1, 27, 1),
            ("c2a", c1, c2, 27, 1), ("c2b", c2, c2, 27, 1),
            ("c3a", c2, c3, 27, 1), ("c3b", c3, c3, 27, 1),
            ("c4a", c3, c4, 27, 1), ("c4b", c4, c4, 27, 1),
            ("c5a", c3 + c4, c3, 27, 1), ("c5b", c3, c3, 27, 1),
            ("c6a", c2 + c3, c2, 27, 1), ("c6b", c2, c2, 27, 1),
            ("c7a", c1 + c2, c1, 27, 1), ("c7b", c1, c1, 27, 1),
            ("head", c1, cout, 1, 0)]


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class UNet:
    def __init__(self, base=32, seed=0, stream=None, periodic=PERIODIC):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.sp = ctypes.c_void_p(self.stream.cuda_stream)
        self.lib = L.load_library()
        self.periodic = periodic
        self.layers = layer_table(base)
        self.spec = {l[0]: l for l in self.layers}
        self.status = torch.zeros(4, dtype=torch.int32, device=self.dev)
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.w32, self.b32, self.wbf, self.wflip, self.gw, self.gb, self.mw, self.vw, self.mb, self.vb = (
            {}, {}, {}, {}, {}, {}, {}, {}, {}, {})
        for name, ci, co, taps, relu in self.layers:
            std = math.sqrt(2.0 / (taps * ci)) * (0.1 if name == "head" else 1.0)
            w = (torch.randn((co, taps, ci), generator=g) * std).float().to(self.dev)
            self.w32[name] = w
            self.b32[name] = torch.zeros(co, dtype=torch.float32, device=self.dev)
            self.wbf[name] = w.to(torch.bfloat16).contiguous()
            self.wflip[name] = torch.empty((ci, taps, co), dtype=torch.bfloat16, device=self.dev)
            for d in (self.gw, self.mw, self.vw):
                d[name] = torch.zeros_like(w)
            for d in (self.gb, self.mb, self.vb):
                d[name] = torch.zeros(co, dtype=torch.float32, device=self.dev)
        self.step_count = 0
        self.acts = {}

    # ------------------------------------------------------------------ utils
    def _check(self, rc, what):
        L._check(rc, what)

    def _dims(self, level, shape):
        nx, ny, nz, nb = shape
        f = 1 << level
        return nx // f, ny // f, nz // f, nb

    def _buf(self, key, shape, dtype):
        t = self.acts.get(key)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = self.torch.empty(shape, dtype=dtype, device=self.dev)
            self.acts[key] = t
        return t

    def parameters(self):
        return {k: (self.w32[k], self.b32[k]) for k in self.w32}

    def load_parameters(self, params):
        for k, (w, b) in params.items():
            self.w32[k].copy_(self.torch.as_tensor(np.asarray(w), dtype=self.torch.float32))
            self.b32[k].copy_(self.torch.as_tensor(np.asarray(b), dtype=self.torch.float32))
            self.wbf[k].copy_(self.w32[k].to(self.torch.bfloat16))

    def save(self, path):
        """Write the network in the weight-file format lb_surrogate_load reads:
        magic, version, base, input and head channels, scales, periodic axes,
        then (ci, co, taps, relu, FP32 weights [co][taps][ci], FP32 bias) per
        convolution in forward order."""
        import struct
        base = self.layers[0][2]
        with open(path, "wb") as fh:
            fh.write(struct.pack("<Ii3iffIi", 0x4E4E424C, 1, base, CIN, COUT, S_RHO, S_U, self.periodic,
                                 len(self.layers)))
            for name, ci, co, taps, relu in self.layers:
                fh.write(struct.pack("<4i", ci, co, taps, relu))
                fh.write(self.w32[name].detach().float().cpu().numpy().astype("<f4").tobytes())
                fh.write(self.b32[name].detach().float().cpu().numpy().astype("<f4").tobytes())

    # ---------------------------------------------------------------- forward
    def _conv(self, name, x, level, shape, out_bf=None, out_f32=None):
        _, ci, co, taps, relu = self.spec[name]
        nx, ny, nz, nb = self._dims(level, shape)
        nv = nx * ny * nz * nb
        if out_bf is None and out_f32 is None:
            out_bf = self._buf(("act", name), (nv, co), self.torch.bfloat16)
        rc = self.lib.lbnn_conv3d_fwd(_p(x), ci, _p(self.wbf[name]), taps, _p(self.b32[name]),
                                      _p(out_bf) if out_bf is not None else None,
                                      _p(out_f32) if out_f32 is not None else None, co, 0, nx, ny, nz, nb,
                                      self.periodic, relu, _p(self.status), self.sp)
        self._check(rc, f"conv {name}")
        self.acts[("in", name)] = x
        return out_bf if out_bf is not None else out_f32

    def _pool(self, key, x, c, level, shape):
        nx, ny, nz, nb = self._dims(level, shape)
        y = self._buf(("pool", key), (nx * ny * nz * nb // 8, c), self.torch.bfloat16)
        self._check(self.lib.lbnn_avgpool2(_p(x), c, nx, ny, nz, nb, _p(y), self.sp), "avgpool2")
        return y

    def _upcat(self, key, skip, cs, low, cl, level, shape):
        nx, ny, nz, nb = self._dims(level, shape)
        y = self._buf(("cat", key), (nx * ny * nz * nb, cs + cl), self.torch.bfloat16)
        self._check(self.lib.lbnn_up_concat(_p(skip), cs, _p(low), cl, nx, ny, nz, nb, _p(y), self.sp), "up_concat")
        return y

    def _conv_cat(self, name, key, skip, cs, low, cl, level, shape):
        """Decoder convolution of concat(skip, up2(low)).  Where the grid allows
        it, the kernel reads both sources in place; the concatenated copy the
        weight gradient needs is then built in backward()."""
        nx, ny, nz, nb = self._dims(level, shape)
        if nx % 8 or ny % 16 or nz % 2:
            return self._conv(name, self._upcat(key, skip, cs, low, cl, level, shape), level, shape)
        _, ci, co, taps, relu = self.spec[name]
        out = self._buf(("act", name), (nx * ny * nz * nb, co), self.torch.bfloat16)
        rc = self.lib.lbnn_conv3d_fwd_upcat(_p(skip), cs, _p(low), cl, _p(self.wbf[name]), _p(self.b32[name]),
                                            _p(out), None, co, 0, nx, ny, nz, nb, self.periodic, relu,
                                            _p(self.status), self.sp)
        self._check(rc, f"conv {name}")
        self.acts[("in", name)] = (key, skip, cs, low, cl, level)
        return out

    def forward(self, x, shape):
        """x: BF16 [nvox][CIN] on the device; shape = (nx, ny, nz, nb).
        Returns the FP32 head output [nvox][COUT]."""
        for d in shape[:3]:
            if d % 8:
                raise ValueError("every extent must be a multiple of 8")
        sp = self.spec
        self.shape = shape
        a = self._conv("c1a", x, 0, shape)
        s1 = self._conv("c1b", a, 0, shape)
        a = self._conv("c2a", self._pool("p1", s1, sp["c1b"][2], 0, shape), 1, shape)
        s2 = self._conv("c2b", a, 1, shape)
        a = self._conv("c3a", self._pool("p2", s2, sp["c2b"][2], 1, shape), 2, shape)
        s3 = self._conv("c3b", a, 2, shape)
        a = self._conv("c4a", self._pool("p3", s3, sp["c3b"][2], 2, shape), 3, shape)
        b4 = self._conv("c4b", a, 3, shape)
        a = self._conv_cat("c5a", "u3", s3, sp["c3b"][2], b4, sp["c4b"][2], 2, shape)
        d3 = self._conv("c5b", a, 2, shape)
        a = self._conv_cat("c6a", "u2", s2, sp["c2b"][2], d3, sp["c5b"][2], 1, shape)
        d2 = self._conv("c6b", a, 1, shape)
        a = self._conv_cat("c7a", "u1", s1, sp["c1b"][2], d2, sp["c6b"][2], 0, shape)
        d1 = self._conv("c7b", a, 0, shape)
        nx, ny, nz, nb = shape
        y = self._buf(("act", "head32"), (nx * ny * nz * nb, COUT), self.torch.float32)
        self._conv("head", d1, 0, shape, out_bf=None, out_f32=y)
        self.acts["s"] = (s1, s2, s3, b4, d3, d2, d1)
        return y

    # --------------------------------------------------------------- backward
    def _conv_back(self, name, g, level, need_dx=True):
        """g: FP32 dL/d(output) [nv][co].  Accumulates dW, db; returns FP32 dL/d(input)."""
        _, ci, co, taps, relu = self.spec[name]
        nx, ny, nz, nb = self._dims(level, self.shape)
        nv = nx * ny * nz * nb
        T = self.torch
        y = self.acts[("act", name)] if name != "head" else None
        gpre_b = self._buf(("gpre_b", name), (nv, co), T.bfloat16)
        gpre_f = self._buf(("gpre_f", name), (nv, co), T.float32)
        self._check(self.lib.lbnn_relu_bwd(_p(g), _p(y) if y is not None else None, nv * co, relu if name != "head" else 0,
                                           _p(gpre_b), _p(gpre_f), self.sp), "relu_bwd")
        self._check(self.lib.lbnn_bias_grad(_p(gpre_f), nv, co, _p(self.gb[name]), self.sp), "bias_grad")
        x = self.acts[("in", name)]
        if isinstance(x, tuple):  # fused up-concat in forward: build the concatenated input now
            key, skip, cs, low, cl, lev = x
            x = self._upcat(key, skip, cs, low, cl, lev, self.shape)
        vpc = max(64, min(8192, (nv // 256 + 63) // 64 * 64))
        self._check(self.lib.lbnn_conv3d_wgrad(_p(gpre_b), co, _p(x), ci, taps, _p(self.gw[name]), nx, ny, nz, nb,
                                               self.periodic, vpc, _p(self.status), self.sp),
                    "conv wgrad")
        if not need_dx:
            return None
        dx = self._buf(("gin", name), (nv, ci), T.float32)
        self._check(self.lib.lbnn_flip_weights(_p(self.wbf[name]), co, taps, ci, _p(self.wflip[name]), self.sp),
                    "flip_weights")
        for c0 in range(0, ci, 256):  # the accumulator holds at most 256 output channels
            cc = min(256, ci - c0)
            wpart = self.wflip[name][c0:c0 + cc]
            self._check(self.lib.lbnn_conv3d_fwd(_p(gpre_b), co, _p(wpart), taps, None, None,
                                                 ctypes.c_void_p(dx.data_ptr() + 4 * c0), cc, ci, nx, ny, nz, nb,
                                                 self.periodic, 0, _p(self.status), self.sp), "conv dgrad")
        return dx

    def _zeros(self, key, shape):
        t = self._buf(("gz", key), shape, self.torch.float32)
        t.zero_()
        return t

    def backward(self, gy):
        """gy: FP32 dL/dy [nvox][COUT]; fills the parameter gradients."""
        sp = self.spec
        for k in self.gw:
            self.gw[k].zero_()
            self.gb[k].zero_()
        shape = self.shape
        nx, ny, nz, nb = shape
        c1, c2, c3, c4 = sp["c1b"][2], sp["c2b"][2], sp["c3b"][2], sp["c4b"][2]
        vol = lambda lev: (nx >> lev) * (ny >> lev) * (nz >> lev) * nb
        g = self._conv_back("head", gy, 0)
        g = self._conv_back("c7a", self._conv_back("c7b", g, 0), 0)        # dL/du1 [v][c1 + c2]
        gs1 = self._zeros("s1", (vol(0), c1))
        gd2 = self._zeros("d2", (vol(1), c2))
        self._check(self.lib.lbnn_up_concat_bwd(_p(g), c1, c2, nx, ny, nz, nb, _p(gs1), _p(gd2), self.sp), "upcat bwd")
        g = self._conv_back("c6a", self._conv_back("c6b", gd2, 1), 1)
        gs2 = self._zeros("s2", (vol(1), c2))
        gd3 = self._zeros("d3", (vol(2), c3))
        self._check(self.lib.lbnn_up_concat_bwd(_p(g), c2, c3, nx >> 1, ny >> 1, nz >> 1, nb, _p(gs2), _p(gd3),
                                                self.sp), "upcat bwd")
        g = self._conv_back("c5a", self._conv_back("c5b", gd3, 2), 2)
        gs3 = self._zeros("s3", (vol(2), c3))
        gb4 = self._zeros("b4", (vol(3), c4))
        self._check(self.lib.lbnn_up_concat_bwd(_p(g), c3, c4, nx >> 2, ny >> 2, nz >> 2, nb, _p(gs3), _p(gb4),
                                                self.sp), "upcat bwd")
        g = self._conv_back("c4a", self._conv_back("c4b", gb4, 3), 3)      # dL/dp3
        self._check(self.lib.lbnn_avgpool2_bwd(_p(g), c3, nx >> 2, ny >> 2, nz >> 2, nb, _p(gs3), self.sp), "pool bwd")
        g = self._conv_back("c3a", self._conv_back("c3b", gs3, 2), 2)      # dL/dp2
        self._check(self.lib.lbnn_avgpool2_bwd(_p(g), c2, nx >> 1, ny >> 1, nz >> 1, nb, _p(gs2), self.sp), "pool bwd")
        g = self._conv_back("c2a", self._conv_back("c2b", gs2, 1), 1)      # dL/dp1
        self._check(self.lib.lbnn_avgpool2_bwd(_p(g), c1, nx, ny, nz, nb, _p(gs1), self.sp), "pool bwd")
        self._conv_back("c1a", self._conv_back("c1b", gs1, 0), 0, need_dx=False)

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
        self.step_count += 1
        for k in self.w32:
            self._check(self.lib.lbnn_adam(_p(self.w32[k]), _p(self.gw[k]), _p(self.mw[k]), _p(self.vw[k]),
                                           self.w32[k].numel(), ctypes.c_float(lr), ctypes.c_float(b1),
                                           ctypes.c_float(b2), ctypes.c_float(eps), self.step_count,
                                           ctypes.c_float(wd), _p(self.wbf[k]), self.sp), "adam w")
            self._check(self.lib.lbnn_adam(_p(self.b32[k]), _p(self.gb[k]), _p(self.mb[k]), _p(self.vb[k]),
                                           self.b32[k].numel(), ctypes.c_float(lr), ctypes.c_float(b1),
                                           ctypes.c_float(b2), ctypes.c_float(eps), self.step_count,
                                           ctypes.c_float(0.0), None, self.sp), "adam b")

    def check_status(self):
        st = int(self.status[0].item())
        if st:
            raise RuntimeError(f"a tensor-core kernel gave up a bounded wait (status {st})")


# ---------------------------------------------------------------------------
# fields <-> network tensors
# ---------------------------------------------------------------------------
def pack_input(fields, x, stream):
    """fields: FP32 device tensor [5][N]; x: BF16 [N][CIN]."""
    lib = L.load_library()
    n = fields.shape[-1]
    L._check(lib.lbnn_pack_input(_p(fields), n, CIN, ctypes.c_float(S_RHO), ctypes.c_float(S_U), _p(x),
                                 ctypes.c_void_p(stream.cuda_stream)), "pack_input")


def pack_target(f0, f1, t, stream):
    lib = L.load_library()
    n = f0.shape[-1]
    L._check(lib.lbnn_pack_target(_p(f0), _p(f1), n, COUT, ctypes.c_float(S_RHO), ctypes.c_float(S_U), _p(t),
                                  ctypes.c_void_p(stream.cuda_stream)), "pack_target")


def unpack_output(fields, y, out, stream, rho_min=0.5):
    lib = L.load_library()
    n = fields.shape[-1]
    L._check(lib.lbnn_unpack_output(_p(fields), _p(y), n, COUT, ctypes.c_float(S_RHO), ctypes.c_float(S_U),
                                    ctypes.c_float(rho_min), _p(out), ctypes.c_void_p(stream.cuda_stream)),
             "unpack_output")


def mse(y, t, wch, grad, loss, stream, nch=5):
    lib = L.load_library()
    n = y.shape[0]
    L._check(lib.lbnn_mse(_p(y), _p(t), n, COUT, nch, _p(wch), _p(grad), _p(loss), ctypes.c_void_p(stream.cuda_stream)),
             "mse")


# ---------------------------------------------------------------------------
# training data, training, and the surrogate + LB controller
# ---------------------------------------------------------------------------
FIELD_MASK = 0b11111  # phi, rho, ux, uy, uz


def workload_params():
    """Parameters of the dense-emulsion trajectories the surrogate learns."""
    from . import workloads as W
    return dict(W.BASE, A_h=0.1, h_min=3.0, h_max=3.0, g=(0.0, 0.0, 1e-6), g_mode=1)


def generate_pairs(seeds, shape=(128, 128, 256), K=50, spinup=200, snaps=6, storage="twoset_f32", stream=None):
    """Run the LB from dense emulsions (one per seed) and keep field snapshots
    every K steps after a spin-up: returns a list of FP32 [5][N] device tensors
    per trajectory."""
    import torch
    from . import workloads as W
    stream = stream if stream is not None else torch.cuda.current_stream()
    trajs = []
    p = workload_params()
    sim = L.Sim(*shape, walls=0b010, stream=stream, storage=storage, **p)
    for seed in seeds:
        phi, _ = W.dense_emulsion_phi(shape, 0b010, int(seed), device=torch.device("cuda", torch.cuda.current_device()),
                                      film=W.DENSE_FILM)
        sim.init_fields(phi)
        sim.step(spinup)
        snaps_t = []
        for k in range(snaps):
            snaps_t.append(sim.fields_device(FIELD_MASK).reshape(5, -1).clone())
            if k + 1 < snaps:
                sim.step(K)
        sim.check()
        trajs.append(snaps_t)
    sim.close()
    return trajs


def train(net, trajs, shape, iters=300, lr=1e-3, seed=0, stream=None, wch=(4.0, 1.0, 1.0, 1.0, 1.0), log_every=50):
    """Adam on the MSE of the scaled K-step increments; returns the loss history."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    nx, ny, nz = shape
    N = nx * ny * nz
    x = torch.empty((N, CIN), dtype=torch.bfloat16, device=net.dev)
    t = torch.empty((N, COUT), dtype=torch.float32, device=net.dev)
    g = torch.empty((N, COUT), dtype=torch.float32, device=net.dev)
    w = torch.zeros(COUT, dtype=torch.float32, device=net.dev)
    w[:5] = torch.tensor(wch, dtype=torch.float32)
    loss = torch.zeros(1, dtype=torch.float64, device=net.dev)
    rng = np.random.default_rng(seed)
    pairs = [(a, b) for tr in trajs for a, b in zip(tr[:-1], tr[1:])]
    hist = []
    with torch.cuda.stream(stream):
        for it in range(iters):
            f0, f1 = pairs[int(rng.integers(len(pairs)))]
            pack_input(f0, x, stream)
            pack_target(f0, f1, t, stream)
            y = net.forward(x, (nx, ny, nz, 1))
            loss.zero_()
            mse(y, t, w, g, loss, stream)
            net.backward(g)
            net.adam(lr=lr * (0.5 * (1 + math.cos(math.pi * it / iters))))
            if it % log_every == 0 or it == iters - 1:
                hist.append((it, float(loss.item())))
        net.check_status()
    return hist


class Controller:
    """Alternate K plain LB steps with one surrogate jump of K steps.

    The jump itself is lb_surrogate_cycle (native): candidate from the network
    loaded on the handle, drift monitors (droplet count unchanged, dispersed
    volume within vol_tol), optional judgement by the plain LB on a shadow
    handle from the exact same state (mean |phi_sur - phi_LB| <= phi_tol),
    acceptance by regularised reconstruction or the LB result.  This class
    holds the policy: every jump is judged until one passes, then every
    judge_every-th; a judgement that passes with a margin (error <= margin x
    phi_tol) doubles the interval up to judge_max, one that passes without it
    keeps the interval, and a failed judgement withdraws the trust, resets
    the interval and suspends the surrogate for backoff cycles (2K plain
    steps per cycle)."""

    def __init__(self, sim, net, shape, K=50, vol_tol=0.02, phi_tol=1e-2, judge_every=4, backoff=8,
                 judge_max=16, margin=0.75, stream=None):
        import os
        import tempfile
        import torch
        self.torch = torch
        self.sim, self.net, self.K = sim, net, K
        self.shape = shape
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nx, ny, nz = shape
        p = workload_params()
        self.shadow = L.Sim(nx, ny, nz, walls=0b010, stream=self.stream, storage=sim.storage, **p)
        fd, path = tempfile.mkstemp(suffix=".lbnn")
        os.close(fd)
        try:
            net.save(path)
            L.lb_surrogate_load(sim.h, path)
        finally:
            os.remove(path)
        self.vol_tol, self.phi_tol = vol_tol, phi_tol
        self.judge_every, self.backoff = judge_every, backoff
        self.judge_max, self.margin = judge_max, margin
        self.interval = judge_every
        self.since = 0         # jumps since the last judgement
        self.accepted = 0
        self.rejected = 0
        self.judged = []       # (cycle, mean |phi_sur - phi_LB|)
        self.suspended = 0
        self.cycle = 0
        self.jumps = 0
        self.trusted = False   # set by a passing judgement

    def reset(self):
        """Forget the counters and the trust (the network and lattices stay)."""
        self.accepted = self.rejected = self.suspended = self.cycle = self.jumps = self.since = 0
        self.judged = []
        self.trusted = False
        self.interval = self.judge_every

    def jump(self):
        """One surrogate jump (or its LB replacement); returns (accepted, info)."""
        self.since += 1
        judge = (not self.trusted) or self.since >= self.interval
        if judge:
            self.since = 0
        self.jumps += 1
        ok, err = L.lb_surrogate_cycle(self.sim.h, self.shadow.h if judge else None, self.K, self.vol_tol,
                                       self.phi_tol)
        info = {"judged": judge, "phi_err": err}
        if judge:
            self.judged.append((self.cycle, err))
            if ok:
                if self.trusted and err <= self.margin * self.phi_tol:
                    self.interval = min(2 * self.interval, self.judge_max)
                self.trusted = True
            else:
                self.trusted = False
                self.interval = self.judge_every
                self.suspended = self.backoff
        if ok:
            self.accepted += 1
        else:
            self.rejected += 1
        return ok, info

    def run(self, cycles):
        """cycles x (K LB steps + one jump of K steps, or 2K LB steps while the
        surrogate is suspended)."""
        infos = []
        for _ in range(cycles):
            self.sim.step(self.K)
            if self.suspended > 0:
                self.sim.step(self.K)
                self.suspended -= 1
                infos.append((None, {"suspended": True}))
            else:
                infos.append(self.jump())
            self.cycle += 1
        return infos

    def close(self):
        self.shadow.close()
