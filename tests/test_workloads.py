"""The seeded input recipes (host logic, no GPU): what the readings of the
configurations fix about the synthetic inputs.

* random sequential addition: radii in range, surface gaps >= gap under the
  periodic minimum image, distance to the solid layers >= wall_gap,
  reproducible per seed (readings C15, C19);
* dense emulsion (reading C15): phi is +-1, +1 exactly on the fluid nodes of
  the grown and eroded power cells, dispersed fraction of the fluid nodes at
  the target, solid layers -1, reproducible per seed;
* batch sweep (reading C19): 64 periodic cubic runs drawn from the four
  sizes, A ~ U[0.005, 0.02], A_h ~ U[0.05, 0.2], 1..20 droplets of radius
  U[6, min(12, L/6)], reproducible per seed.
"""
import numpy as np
import pytest

from paper_2405_14551_gb300 import workloads as W


def _min_image(d, L, wall):
    d = d.copy()
    for a in range(3):
        if not wall[a]:
            d[..., a] -= L[a] * np.round(d[..., a] / L[a])
    return d


@pytest.mark.parametrize("shape,walls,rmin,rmax,gap", [((48, 40, 36), 0b010, 3.0, 6.0, 1.0),
                                                        ((64, 64, 64), 0, 6.0, 10.0, 2.0),
                                                        ((40, 30, 50), 0b111, 4.0, 5.0, 2.0)])
def test_rsa_spheres_gaps_walls_and_seed(shape, walls, rmin, rmax, gap):
    rng = np.random.default_rng(11)
    cen, rad = W.rsa_spheres(shape, walls, rng, rmin, rmax, gap=gap, wall_gap=2.0, max_fail=300)
    assert len(rad) >= 3
    assert rad.min() >= rmin and rad.max() <= rmax
    L = np.asarray(shape, dtype=float)
    wall = [(walls >> a) & 1 for a in range(3)]
    d = _min_image(cen[:, None, :] - cen[None, :, :], L, wall)
    dist = np.sqrt((d * d).sum(-1))
    need = rad[:, None] + rad[None, :] + gap
    off = ~np.eye(len(rad), dtype=bool)
    assert np.all(dist[off] >= need[off] - 1e-12)
    for a in range(3):
        if wall[a]:
            # solid layers are nodes 0 and L-1; the sphere keeps wall_gap off them
            assert np.all(cen[:, a] - rad >= 1.0 + 2.0 - 0.5 - 1e-12)
            assert np.all(cen[:, a] + rad <= L[a] - 2.0 - 2.0 + 0.5 + 1e-12)
    cen2, rad2 = W.rsa_spheres(shape, walls, np.random.default_rng(11), rmin, rmax, gap=gap, wall_gap=2.0,
                               max_fail=300)
    np.testing.assert_array_equal(cen, cen2)
    np.testing.assert_array_equal(rad, rad2)


def test_dense_emulsion_fraction_walls_and_seed():
    shape, walls = (64, 48, 80), 0b010
    phi, info = W.dense_emulsion_phi(shape, walls, seed=5, phi_d=0.7)
    assert phi.shape == (shape[2], shape[1], shape[0]) and phi.dtype == np.float32
    assert set(np.unique(phi)) <= {-1.0, 1.0}
    fl = W.fluid_mask(shape, walls)
    assert np.all(phi[~fl] == -1.0)
    frac = float((phi[fl] > 0).mean())
    assert abs(frac - 0.7) < 5e-3 and abs(info["phi_d"] - frac) < 1e-12
    assert info["droplets"] >= 5 and info["film"] > 0
    # the spheres alone fill less than the target: the cells were grown
    assert info["rsa_fraction"] < frac
    phi2, _ = W.dense_emulsion_phi(shape, walls, seed=5, phi_d=0.7)
    np.testing.assert_array_equal(phi, phi2)
    phi3, _ = W.dense_emulsion_phi(shape, walls, seed=6, phi_d=0.7)
    assert np.any(phi3 != phi)


def test_dense_emulsion_film_seeding():
    """The bench's seeding: cells eroded by a film of DENSE_FILM nodes.  Every
    +1 node lies at least half a film from its cell's faces and from the
    walls, so two droplets are never closer than the film."""
    shape, walls = (64, 48, 80), 0b010
    phi, info = W.dense_emulsion_phi(shape, walls, seed=5, film=W.DENSE_FILM)
    rng = np.random.default_rng(5)
    cen, rad = W.rsa_spheres(shape, walls, rng, 8.0, 12.0, max_fail=400)
    owner, margin = W.power_cell_margin(shape, walls, cen, rad, 12.0)
    fl = W.fluid_mask(shape, walls)
    inside = phi > 0
    assert np.all(margin[inside] >= 0.5 * W.DENSE_FILM) and np.all(fl[inside])
    assert np.all(phi[fl & (margin < 0.5 * W.DENSE_FILM)] == -1.0)
    assert info["film"] == W.DENSE_FILM and abs(info["phi_d"] - float(inside[fl].mean())) < 1e-12
    # a thinner film reaches a larger fraction, bounded by the 0.7 of the fraction mode
    assert info["phi_d"] < W.dense_emulsion_phi(shape, walls, seed=5, phi_d=0.7)[1]["phi_d"]
    assert len(np.unique(owner[inside])) == info["droplets"] == len(rad)


def test_batch_sweep_ranges_and_seed():
    runs = W.batch_sweep()
    assert len(runs) == 64
    sizes = {r.shape[0] for r in runs}
    assert sizes <= {48, 64, 96, 128} and len(sizes) >= 3
    for r in runs:
        L = r.shape[0]
        assert r.shape == (L, L, L) and r.walls == 0 and r.steps == 1000
        p = r.params
        assert 0.005 <= p["A_a"] == p["A_b"] <= 0.02
        assert 0.05 <= p["A_h"] <= 0.2 and p["h_min"] == p["h_max"] == 3.0
        assert 1 <= len(r.radii) <= 20
        assert r.radii.min() >= 6.0 and r.radii.max() <= min(12.0, L / 6.0)
    again = W.batch_sweep()
    for a, b in zip(runs, again):
        assert a.shape == b.shape and a.params == b.params
        np.testing.assert_array_equal(a.centres, b.centres)
