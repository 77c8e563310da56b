"""The allocation-free reduction entry point.

lb_reduce_fields_f64_static serves callers that cannot allocate device
memory when they need the global sums; it keeps its partial sums in a static
device array of the library.  Here it must give the same sums as
lb_reduce_f64 (which uses memory its handle allocated) on two calls in a row,
reusing the same static array, and reject grids beyond its limit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device_fields(sim):
    import paper_2405_14551_gb300.lbcg as L
    return sim.fields_device(L.ALL_FIELDS)


def test_static_reduction_matches_handle_reduction():
    import torch

    import paper_2405_14551_gb300.lbcg as L
    from paper_2405_14551_gb300 import workloads as W

    stream = torch.cuda.Stream()
    cases = [(W.small_droplet(), 60), (W.droplet_pair(48, 40, 56, R=8.0, sep=20.0), 25)]
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for wl, steps in cases:  # two calls in a row share the static array
        nx, ny, nz = wl.shape
        s = L.Sim(nx, ny, nz, walls=wl.walls, stream=stream, **wl.params)
        s.init_droplets(wl.centres, wl.radii)
        s.step(steps)
        ref = s.reduce()
        fields = _device_fields(s)
        torch.cuda.synchronize()
        L.lb_reduce_fields_f64_static(fields.data_ptr(), False, nx, ny, nz, wl.walls, out.data_ptr(),
                                      stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        s.close()


def test_static_reduction_walls_and_fp64_fields():
    """The two paths the periodic FP32 case does not reach: solid wall layers
    excluded from the sums (a channel walled in y, and one walled on every
    axis), and double-precision fields (fields_are_f64) of an FP64 handle."""
    import torch

    import paper_2405_14551_gb300.lbcg as L
    from paper_2405_14551_gb300 import workloads as W

    def channel(walls):
        p = dict(W.BASE, A_h=0.1, h_min=2.0, h_max=3.0, g=(0.0, 0.0, 1e-4), g_mode=2)
        return W.Workload("channel", (21, 18, 33), walls, p, 30,
                          centres=np.array([[10.0, 9.0, 10.0], [10.5, 9.0, 22.5]]), radii=np.array([5.0, 5.2]))

    stream = torch.cuda.Stream()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    cases = [(channel(0b010), "twoset_f32", False, 30),
             (channel(0b111), "twoset_f32", False, 12),
             (channel(0b010), "twoset_f64", True, 30)]
    for wl, storage, f64, steps in cases:
        nx, ny, nz = wl.shape
        s = L.Sim(nx, ny, nz, walls=wl.walls, stream=stream, storage=storage, **wl.params)
        s.init_droplets(wl.centres, wl.radii)
        s.step(steps)
        ref = s.reduce()
        dt = torch.float64 if f64 else torch.float32
        fields = torch.empty((len(L.FIELD_NAMES),) + s.shape, dtype=dt, device="cuda")
        L.lb_fields(s.h, L.ALL_FIELDS, fields, True, f64=f64)
        torch.cuda.synchronize()
        L.lb_reduce_fields_f64_static(fields.data_ptr(), f64, nx, ny, nz, wl.walls, out.data_ptr(),
                                      stream.cuda_stream)
        stream.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
        s.close()


def test_static_reduction_rejects_bad_sizes():
    import torch

    import paper_2405_14551_gb300.lbcg as L
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    for dims in ((0, 4, 4), (1 << 11, 1 << 11, 1 << 10)):
        with pytest.raises(L.LBError) as ei:
            L.lb_reduce_fields_f64_static(buf.data_ptr(), False, *dims, 0, buf.data_ptr(), 0)
        assert ei.value.code == L.LB_EINVAL
