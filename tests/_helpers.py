"""Shared helpers of the test suite: build a GPU simulation and the FP64
oracle from the same seeded workload, and compare their fields."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2405_14551_gb300 import workloads as W

CMP_FIELDS = ("phi", "rho", "ux", "uy", "uz", "rhoA", "rhoB")


def oracle_params(wl: W.Workload, **over):
    p = dict(wl.params)
    p.update(over)
    nx, ny, nz = wl.shape
    return oracle.make_params(nx, ny, nz, walls=wl.walls, **p)


def make_oracle(wl: W.Workload, **over) -> oracle.OracleSim:
    o = oracle.OracleSim(oracle_params(wl, **over))
    if wl.phi is not None:
        o.init_fields(wl.phi.astype(np.float64))
    else:
        o.init_droplets(wl.centres, wl.radii)
    return o


def make_gpu(wl: W.Workload, storage="twoset_f32", **over):
    import paper_2405_14551_gb300.lbcg as L
    p = dict(wl.params)
    p.update(over)
    nx, ny, nz = wl.shape
    s = L.Sim(nx, ny, nz, walls=wl.walls, storage=storage, **p)
    if wl.phi is not None:
        s.init_fields(wl.phi.astype(np.float32))
    else:
        s.init_droplets(wl.centres, wl.radii)
    return s


def field_errors(gpu: dict, orc: dict, names=CMP_FIELDS, mask=None) -> dict:
    out = {}
    for k in names:
        d = np.abs(gpu[k].astype(np.float64) - orc[k])
        if mask is not None:
            d = d[mask]
        out[k] = float(d.max()) if d.size else 0.0
    return out
