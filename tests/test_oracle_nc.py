"""Pins of the oracle's colour gradient and near-contact scan.

* The isotropic gradient stencil is exact on linear phi (reading of
  n = grad phi/|grad phi|, Sec. III.C.1, with the D3Q27 stencil).
* Hand-counted near-contact distances h for planar films
  (tests/golden/nc_planar_film.json; near-contact paragraph of Sec. III.C.1,
  Eqs. stress_jump and near_cont_force), including the h^-3 tail.
* An isolated droplet and a far-apart pair feel no repulsion; walls stop the
  scan; the force field of a mirror-symmetric pair is mirror-antisymmetric.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _film_sim(case, A_h=0.1):
    nz = case["nz"]
    p = oracle.make_params(4, 4, nz, A_h=case.get("A_h", A_h), h_min=case["h_min"], h_max=case["h_max"])
    s = oracle.OracleSim(p)
    phi = np.broadcast_to(np.asarray(case["phi"], dtype=np.float64)[:, None, None], (nz, 4, 4)).copy()
    s.init_fields(phi)
    return s


def test_gradient_exact_on_linear_phi():
    nx, ny, nz = 12, 10, 14
    p = oracle.make_params(nx, ny, nz)
    s = oracle.OracleSim(p)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a = np.array([0.011, -0.007, 0.013])
    phi = -0.2 + a[0] * x + a[1] * y + a[2] * z
    s.init_fields(phi)
    f = s.fields()
    inner = (slice(1, nz - 1), slice(1, ny - 1), slice(1, nx - 1))
    for k, comp in enumerate(("gx", "gy", "gz")):
        np.testing.assert_allclose(f[comp][inner], a[k], atol=1e-14)
    np.testing.assert_allclose(f["phi"], phi, atol=1e-15)


def test_gradient_neutral_wall():
    """A solid neighbour contributes the node's own phi: a phi that varies only
    along the wall normal gives a one-sided difference at the first fluid layer."""
    ny = 8
    p = oracle.make_params(4, ny, 4, walls=0b010)
    s = oracle.OracleSim(p)
    prof = np.array([0, 0.1, 0.3, 0.5, 0.7, 0.9, 0.95, 0], dtype=np.float64)
    phi = np.broadcast_to(prof[None, :, None], (4, ny, 4)).copy()
    s.init_fields(phi)
    f = s.fields()
    gy = f["gy"][0, :, 0]
    # y=1 sees a solid at y=0 -> (phi(2) - phi(1))/2 ; interior central differences
    assert abs(gy[1] - (0.3 - 0.1) / 2) < 1e-15
    assert abs(gy[3] - (0.7 - 0.3) / 2) < 1e-15
    assert abs(gy[6] - (0.95 - 0.95) / 2 - (0.95 - 0.9) / 2) < 1e-15
    assert gy[0] == 0.0 and gy[7] == 0.0


@pytest.mark.parametrize("name", ["film_3_interface_pairs", "film_3_hmax_2", "thin_film_touching",
                                  "wide_film_beyond_reach", "tail_decay"])
def test_planar_film_hand_counted(name):
    with open(os.path.join(GOLDEN, "nc_planar_film.json")) as fh:
        cases = {c["name"]: c for c in json.load(fh)["cases"]}
    case = cases[name]
    s = _film_sim(case)
    f = s.fields()
    h = f["h"][:, 0, 0]
    np.testing.assert_array_equal(h, np.asarray(case["h"], dtype=np.float64))
    # h and the force are uniform over each z-plane
    assert np.all(f["h"] == f["h"][:, :1, :1])
    if "grad_z" in case:
        np.testing.assert_allclose(f["gz"][:, 0, 0], case["grad_z"], atol=1e-15)
    A_h = case.get("A_h", 0.1)
    frz = f["Frz"][:, 0, 0]
    for z in range(case["nz"]):
        hz = int(case["h"][z])
        if hz == 0:
            assert frz[z] == 0.0
            continue
        if "A_of_h" in case:
            Aeff = case["A_of_h"][str(hz)]
        else:
            Aeff = A_h
        # F_rep = -A_h n_out delta_I = (A_h/2) grad phi  (Eq. near_cont_force)
        assert abs(frz[z] - 0.5 * Aeff * f["gz"][z, 0, 0]) < 1e-16
    # the repulsion pushes each interface back towards its own droplet: below
    # the film centre (A underneath) the force points to -z, above it to +z
    centre = int(np.argmin(case["phi"]))
    assert np.all(frz[:centre] <= 0) and np.all(frz[centre + 1:] >= 0)


def test_isolated_droplet_feels_no_repulsion():
    p = oracle.make_params(24, 24, 24, A_h=0.1)
    s = oracle.OracleSim(p)
    s.init_droplets([[12, 12, 12]], [7.0], width=1.5)
    f = s.fields()
    assert np.all(f["h"] == 0)
    assert np.all(f["Frx"] == 0) and np.all(f["Fry"] == 0) and np.all(f["Frz"] == 0)
    s.step(20)
    f = s.fields()
    assert np.all(f["h"] == 0)


def test_far_pair_feels_no_repulsion_near_pair_does():
    p = oracle.make_params(20, 20, 48, A_h=0.1)
    far = oracle.OracleSim(p)
    far.init_droplets([[10, 10, 12], [10, 10, 36]], [6.0, 6.0], width=1.0)
    assert np.all(far.fields()["h"] == 0)
    near = oracle.OracleSim(p)
    near.init_droplets([[10, 10, 17], [10, 10, 31]], [6.0, 6.0], width=1.0)
    fn = near.fields()
    assert np.any(fn["h"] > 0)
    # mirror z -> 48 - z maps the pair onto itself: h symmetric, F_z antisymmetric
    h = fn["h"]
    hm = np.roll(h[::-1], 1, axis=0)
    np.testing.assert_array_equal(h, hm)
    fz = fn["Frz"]
    np.testing.assert_allclose(fz, -np.roll(fz[::-1], 1, axis=0), atol=1e-15)
    # net repulsion pushes the lower droplet down and the upper one up
    assert fz[:24].sum() < 0 and fz[24:].sum() > 0


def test_wall_stops_scan():
    """A film against a wall: the scan from the droplet interface towards the
    wall hits the solid layer and produces no force (no droplet-wall repulsion)."""
    ny = 10
    p = oracle.make_params(4, ny, 4, walls=0b010, A_h=0.1)
    s = oracle.OracleSim(p)
    prof = np.array([0, -0.5, 0.5, 1, 1, 1, 1, 1, 1, 0], dtype=np.float64)
    phi = np.broadcast_to(prof[None, :, None], (4, ny, 4)).copy()
    s.init_fields(phi)
    f = s.fields()
    assert np.all(f["h"] == 0)


@pytest.mark.parametrize("name", ["diagonal_film", "two_to_one_film"])
def test_oblique_film_hand_counted(name):
    """Films whose normal is off the lattice axes (tests/golden/nc_oblique_film.json):
    the scan's targets are x + lround(k n_out) with a non-axis normal, so the
    rounding decides which nodes are visited (a diagonal ray visits s + 2
    twice; a (2, 1) ray steps over the opposite interface of the outer layer)."""
    with open(os.path.join(GOLDEN, "nc_oblique_film.json")) as fh:
        case = {c["name"]: c for c in json.load(fh)["cases"]}[name]
    nx, ny, a, b, nz = case["nx"], case["ny"], case["a"], case["b"], 2
    prof = np.array([1, 1, 0.5, -0.5, -1, -0.5, 0.5, 1], dtype=np.float64)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    s_of = (a * x + b * y) % 8
    phi = np.broadcast_to(prof[s_of][None], (nz, ny, nx)).copy()
    p = oracle.make_params(nx, ny, nz, A_h=0.1, h_min=3.0, h_max=3.0)
    sim = oracle.OracleSim(p)
    sim.init_fields(phi)
    f = sim.fields()
    for s in range(8):
        m = np.broadcast_to(s_of == s, (nz, ny, nx))
        assert np.all(f["h"][m] == case["h_s"][str(s)]), (s, np.unique(f["h"][m]))
        np.testing.assert_allclose(f["gz"][m], 0.0, atol=1e-15)
        if "g_s" in case:
            np.testing.assert_allclose(f["gx"][m], case["g_s"][str(s)], atol=1e-15)
            np.testing.assert_allclose(f["gy"][m], case["g_s"][str(s)], atol=1e-15)
        if str(s) in case.get("gx_s", {}):
            np.testing.assert_allclose(f["gx"][m], case["gx_s"][str(s)], atol=1e-15)
            np.testing.assert_allclose(f["gy"][m], case["gy_s"][str(s)], atol=1e-15)
        # F_rep = (A_h/2) grad phi where h > 0, else 0 (Eq. near_cont_force, reading C9)
        on = case["h_s"][str(s)] > 0
        np.testing.assert_allclose(f["Frx"][m], 0.05 * f["gx"][m] if on else 0.0, atol=1e-17)
        np.testing.assert_allclose(f["Fry"][m], 0.05 * f["gy"][m] if on else 0.0, atol=1e-17)
