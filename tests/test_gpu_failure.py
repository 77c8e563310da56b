"""Failure detection on the host side of the C ABI, without a GPU fault.

An lb_alloc callback that returns NULL on chosen calls (host-side
injection): lb_create reports LB_ENOMEM for every n among the allocations
it makes and returns every buffer it had obtained through the callback's
free; allocations made later (the droplet buffer of lb_init_droplets, the
fields buffer of the first lb_fields) report LB_ENOMEM without disturbing
the handle, which then initialises, steps, reads its fields and is destroyed
normally.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """Device memory from PyTorch; the allocations numbered in fail_at
    (0-based, an int or a set) return NULL.  Records every pointer handed
    out and every one freed."""

    def __init__(self, fail_at):
        import torch

        import paper_2405_14551_gb300.lbcg as L
        self.torch = torch
        self.fail_at = {fail_at} if isinstance(fail_at, int) else set(fail_at)
        self.calls = 0
        self.live = {}
        self.freed = 0
        self._a = L.ALLOC_FN(self._alloc)
        self._f = L.FREE_FN(self._free)
        self.struct = L.lb_alloc(self._a, self._f, None)

    def _alloc(self, ctx, nbytes):
        k = self.calls
        self.calls += 1
        if k in self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ctx, ptr):
        self.live.pop(ptr, None)
        self.freed += 1


def _create(alloc, shape=(12, 10, 14), **params):
    import paper_2405_14551_gb300.lbcg as L
    lib = L.load_library()
    h = ctypes.c_void_p()
    rc = lib.lb_create(ctypes.byref(L.make_grid(*shape, walls=0b010)), ctypes.byref(L.make_params(**params)),
                       ctypes.byref(alloc.struct), ctypes.byref(h))
    return rc, h


def test_create_reports_enomem_at_every_allocation_and_frees_the_rest():
    import paper_2405_14551_gb300.lbcg as L
    probe = FailingAllocator(fail_at=-1)
    rc, h = _create(probe, A_h=0.1)
    assert rc == L.LB_OK
    n_create = probe.calls
    assert n_create >= 8  # two lattices, phi, three accumulators, initial phi, scratch
    L.lb_destroy(h)
    assert not probe.live
    for n in range(n_create):
        a = FailingAllocator(fail_at=n)
        rc, h = _create(a, A_h=0.1)
        assert rc == L.LB_ENOMEM, (n, rc)
        assert not h.value
        assert a.calls == n + 1  # nothing allocated after the failure
        assert not a.live and a.freed == n, (n, a.freed)  # everything obtained was returned
        assert "alloc" in L.load_library().lb_last_error().decode()


def test_later_allocation_failure_leaves_the_handle_usable():
    import paper_2405_14551_gb300.lbcg as L
    probe = FailingAllocator(fail_at=-1)
    rc, h = _create(probe)
    n_create = probe.calls
    L.lb_destroy(h)
    # allocation n_create: the droplet buffer of the first lb_init_droplets;
    # n_create + 2: the fields buffer of the first lb_fields
    a = FailingAllocator(fail_at={n_create, n_create + 2})
    rc, h = _create(a)
    assert rc == L.LB_OK
    with pytest.raises(L.LBError) as ei:
        L.lb_init_droplets(h, [[6.0, 5.0, 7.0]], [3.0])
    assert ei.value.code == L.LB_ENOMEM
    with pytest.raises(L.LBError) as ei:
        L.lb_step(h, 1)  # nothing initialised yet
    assert ei.value.code == L.LB_ESTATE
    L.lb_init_droplets(h, [[6.0, 5.0, 7.0]], [3.0])
    L.lb_step(h, 3)
    nz, ny, nx = 14, 10, 12
    out = np.zeros((1, nz, ny, nx), dtype=np.float32)
    with pytest.raises(L.LBError) as ei:
        L.lb_fields(h, L.FIELD_BIT["phi"], out, False)
    assert ei.value.code == L.LB_ENOMEM
    L.lb_step(h, 2)
    L.lb_fields(h, L.FIELD_BIT["phi"], out, False)  # the next allocation succeeds
    assert L.lb_time(h) == 5
    assert np.abs(out).max() <= 1.0 + 1e-5 and out.max() > 0.5
    L.lb_check(h)
    L.lb_destroy(h)
    assert not a.live
