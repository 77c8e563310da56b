"""Write tests/golden/droplet_pair_4000.json from the FP64 oracle alone.

The approaching droplet pair (64x64x128 periodic box, R = 10, centres at
z = 52 and z = 76, mirror body force +-1e-5 on the A component, near contact
A_h = 0.1, h_min = h_max = 3), and the same run without near contact, every
100 steps up to 4000: the droplet count (6-connected phi > 0), the centroids
z1, z2 of the dispersed phase (weight (1 + phi)/2) below and above the
mirror plane z = 64 (the mirror planes z = 0 and z = 64 excluded), and the
total momentum.  Run: python tests/golden/make_droplet_pair_trajectory.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2405_14551_gb300 import workloads as W  # noqa: E402


def centroids(phi):
    nz = phi.shape[0]
    w = 0.5 * (1.0 + phi)
    wz = w.sum(axis=(1, 2))
    z = np.arange(nz, dtype=np.float64)
    lo, hi = slice(1, nz // 2), slice(nz // 2 + 1, nz)
    return float((z[lo] * wz[lo]).sum() / wz[lo].sum()), float((z[hi] * wz[hi]).sum() / wz[hi].sum())


def trajectory(A_h, steps=4000, every=100):
    wl = W.droplet_pair()
    nx, ny, nz = wl.shape
    p = dict(wl.params, A_h=A_h)
    o = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=wl.walls, **p))
    o.init_droplets(wl.centres, wl.radii)
    rows = []
    for t in range(every, steps + 1, every):
        o.step(every)
        z1, z2 = centroids(o.fields()["phi"])
        r = o.reduce()
        rows.append({"t": t, "count": o.droplet_count(), "z1": z1, "z2": z2,
                     "momentum": [float(v) for v in r[2:5]]})
        print(A_h, rows[-1], flush=True)
    o.close()
    return rows


def main():
    out = {"source": "FP64 oracle (oracle/cglb_oracle.c), written by tests/golden/make_droplet_pair_trajectory.py",
           "workload": "droplet_pair 64x64x128, R = 10, centres z = 52, 76, g = +-1e-5 (g_mode 2), h_min = h_max = 3",
           "near_contact": trajectory(0.1), "no_near_contact": trajectory(0.0)}
    with open(os.path.join(HERE, "droplet_pair_4000.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
