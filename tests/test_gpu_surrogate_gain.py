"""What the trained network gains over the method without it.

The surrogate replaces K = 50 LB steps by one network jump; without the
network, a jump would leave the fields unchanged (the persistence forecast,
the only K-step prediction available without the learned part).  On a
128x128x128 dense emulsion (walls y, 6-node film seeding, near contact),
twelve LB trajectories after 2000 spin-up steps give 84 training pairs; the
BF16 U-Net (4 levels, 32 base channels) is trained by the library's tcgen05
kernels for 2000 Adam steps, and on six held-out pairs from two other seeds
its mean |phi_pred - phi_LB| per jump must be at most 0.8 of the
persistence error (measured: 0.71).  About 45 s on one GB300.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_network_beats_persistence_on_held_out_jumps():
    import torch

    from paper_2405_14551_gb300 import surrogate as S
    shape = (128, 128, 128)
    nx, ny, nz = shape
    n = nx * ny * nz
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        trajs = S.generate_pairs(range(12), shape=shape, spinup=2000, snaps=8, stream=st)
        test = S.generate_pairs([1000, 1001], shape=shape, spinup=2000, snaps=4, stream=st)
        net = S.UNet(base=32, seed=0, stream=st)
        S.train(net, trajs, shape, iters=2000, lr=1e-3, stream=st, log_every=1000)
        x = torch.empty((n, S.CIN), dtype=torch.bfloat16, device="cuda")
        out = torch.empty((5, n), dtype=torch.float32, device="cuda")
        err, pers = [], []
        for tr in test:
            for f0, f1 in zip(tr[:-1], tr[1:]):
                S.pack_input(f0, x, st)
                y = net.forward(x, (nx, ny, nz, 1))
                S.unpack_output(f0, y, out, st)
                err.append(float((out[0] - f1[0]).abs().mean()))
                pers.append(float((f0[0] - f1[0]).abs().mean()))
        net.check_status()
    err, pers = np.array(err), np.array(pers)
    print("held-out mean |dphi| per jump: network", err.round(5), "persistence", pers.round(5))
    assert len(err) == 6
    assert err.mean() <= 0.8 * pers.mean(), (err.mean(), pers.mean())
    assert np.all(err < pers)
