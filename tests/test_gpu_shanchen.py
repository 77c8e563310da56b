"""Parity of the Shan-Chen step (Sec. III.C.3, lattice pseudo-potential
model; LB_MODEL_SHAN_CHEN) with the FP64 oracle, through the C ABI.

Same tolerances as the colour-gradient path: FP32 two-set storage <= 1e-5
per field, FP64 <= 1e-11.  Cases: an off-axis droplet pair in a periodic box
with unequal relaxation times and a body force on each component's density;
a ragged walled channel (solid layers y = 0, ny - 1, the mirror force on
A); a single droplet over 200 steps; conservation of each component's mass
and of the total momentum (the force is pairwise) in FP64 on the GPU.
"""
import numpy as np
import pytest

from paper_2405_14551_gb300 import workloads as W

from _helpers import CMP_FIELDS, field_errors, make_gpu, make_oracle

pytestmark = pytest.mark.gpu

SC = dict(model=1, G=7.5, psi0=1.0, A_a=0.0, A_b=0.0, beta=0.0)
FIELDS = CMP_FIELDS + ("Frx", "Fry", "Frz")


def _pair():
    p = dict(W.BASE, tau_a=0.8, tau_b=1.3, g=(1e-5, 0.0, -2e-5), g_mode=1, **SC)
    return W.Workload("sc_pair", (26, 22, 30), 0, p, 40,
                      centres=np.array([[9.3, 10.6, 9.8], [15.1, 11.4, 20.7]]), radii=np.array([5.1, 4.4]))


def _channel():
    p = dict(W.BASE, tau_a=1.0, tau_b=0.7, g=(0.0, 0.0, 3e-5), g_mode=2, **SC)
    return W.Workload("sc_channel", (21, 18, 33), 0b010, p, 40,
                      centres=np.array([[10.0, 9.0, 10.0], [10.5, 8.6, 22.5]]), radii=np.array([4.6, 4.8]))


@pytest.mark.parametrize("wl_fn", [_pair, _channel])
@pytest.mark.parametrize("storage,tol", [("twoset_f32", 1e-5), ("twoset_f64", 1e-11)])
def test_shan_chen_matches_oracle(wl_fn, storage, tol):
    wl = wl_fn()
    o = make_oracle(wl)
    s = make_gpu(wl, storage=storage)
    e0 = field_errors(s.fields(f64=True), o.fields(), FIELDS)
    assert max(e0.values()) <= tol, e0
    o.step(wl.steps)
    s.step(wl.steps)
    s.check()
    fo, fg = o.fields(), s.fields(f64=True)
    e = field_errors(fg, fo, FIELDS)
    print(wl.name, storage, e)
    assert np.abs(fo["Frz"]).max() > 1e-3  # the pseudo-potential force is active
    assert max(e.values()) <= tol, e
    assert np.all(fg["h"] == 0)


def test_shan_chen_single_droplet_200_steps():
    wl = W.Workload("sc_droplet", (32, 32, 32), 0, dict(W.BASE, **SC), 200,
                    centres=np.array([[16.0, 16.0, 16.0]]), radii=np.array([8.0]))
    o = make_oracle(wl)
    s = make_gpu(wl)
    o.step(200)
    s.step(200)
    e = field_errors(s.fields(f64=True), o.fields(), FIELDS)
    print("sc droplet 200 steps", e)
    assert max(e.values()) <= 1e-5, e


def test_shan_chen_conserves_mass_and_momentum_fp64():
    wl = _pair()
    wl.params["g_mode"] = 0
    s = make_gpu(wl, storage="twoset_f64")
    r0 = s.reduce()
    s.step(120)
    r1 = s.reduce()
    assert abs(r1[0] - r0[0]) / r0[0] < 1e-13 and abs(r1[1] - r0[1]) / r0[1] < 1e-13
    assert np.all(np.abs(r1[2:5]) < 1e-11), r1[2:5]
