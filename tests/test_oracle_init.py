"""Pin of the oracle's droplet initialiser (reading C14: sharp droplets,
periodic minimum-image distance on open axes, union of overlapping droplets)
against a hand-counted fixture, tests/golden/init_droplets.json."""
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _case():
    with open(os.path.join(GOLDEN, "init_droplets.json")) as fh:
        return json.load(fh)


def test_periodic_cut_and_overlapping_pair():
    c = _case()
    nx, ny, nz = c["box"]
    s = oracle.OracleSim(oracle.make_params(nx, ny, nz))
    s.init_droplets(c["centres"], c["radii"])
    f = s.fields()
    phi = f["phi"]
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for x, y, z in c["periodic"]["inside"]:
        inside[z, y, x] = True
    assert inside.sum() == c["periodic"]["count_plus"]
    np.testing.assert_array_equal(phi[inside], 1.0)
    np.testing.assert_array_equal(phi[~inside], -1.0)
    # rho = 1 and the component densities split as (1 +- phi)/2
    np.testing.assert_allclose(f["rho"], 1.0, atol=1e-15)
    np.testing.assert_allclose(f["rhoA"], (1.0 + phi) / 2, atol=1e-15)


def test_walled_axis_has_no_periodic_image():
    c = _case()
    nx, ny, nz = c["box"]
    s = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=0b001))
    s.init_droplets(c["centres"][:1], c["radii"][:1])
    phi = s.fields()["phi"]
    fluid = np.ones((nz, ny, nx), dtype=bool)
    fluid[:, :, 0] = fluid[:, :, nx - 1] = False
    assert int((phi[fluid] > 0).sum()) == c["walled_x"]["count_plus_fluid_droplet0"]
    assert phi[0, 0, 1] == 1.0 and phi[0, 0, 2] == 1.0 and phi[0, 0, 3] == -1.0
