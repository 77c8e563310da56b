"""Pins of the oracle's regularised collision (the regularised colour-gradient
scheme that Sec. III.C.1 cites for filtering the non-hydrodynamic modes; the
paper gives no formula, the reading is the Hermite projection of the
non-equilibrium part on orders 1 and 2).

What fixes it, independently of how the projection is coded:
  * Hermite algebra: the projection keeps the non-equilibrium moments of
    orders 0, 1 and 2, its third- and fourth-order Hermite moments vanish, and
    projecting twice changes nothing;
  * at tau = 1 the relaxed part is multiplied by 1 - 1/tau = 0, so the
    collision equals BGK exactly;
  * the post-collision moments up to order 2 (mass, momentum, momentum flux)
    equal BGK's, so the hydrodynamics (and the Poiseuille profile with the
    same viscosity) are unchanged; per-component mass is still conserved;
  * a state whose non-equilibrium part already lies in orders 1-2 collides
    exactly as under BGK.
"""
import numpy as np
import pytest

import oracle
from oracle import OracleSim, make_params

RNG = np.random.default_rng(7)
CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat():
    c, w, _, _ = oracle.lattice()
    return c.astype(np.float64), w


def _state(rho, u, amp):
    return oracle.feq(rho, u) * (1.0 + amp * RNG.normal(size=27))


@pytest.mark.parametrize("trial", range(4))
def test_projection_keeps_low_moments_and_drops_high_ones(lat, trial):
    c, w = lat
    f = _state(1.1, 0.03 * RNG.normal(size=3), 0.05)
    rho = f.sum()
    # equilibrium at the state's own density and a shifted velocity, as with
    # the half-force shift: the non-equilibrium part then has zero mass and a
    # non-zero first moment
    feq = oracle.feq(rho, (f @ c) / rho + 1e-3 * RNG.normal(size=3))
    r = oracle.regularise(f, feq)
    d = f - feq
    assert abs(r.sum() - d.sum()) < 1e-15
    np.testing.assert_allclose(r @ c, d @ c, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", r, c, c), np.einsum("i,ia,ib->ab", d, c, c), atol=1e-15)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    for h3 in (x * y * z, (x * x - CS2) * y, (y * y - CS2) * z, (z * z - CS2) * x):
        assert abs(r @ h3) < 1e-15
        assert abs(d @ h3) > 1e-6  # the random state did carry third-order content
    assert abs(r @ ((x * x - CS2) * (y * y - CS2))) < 1e-15
    np.testing.assert_allclose(oracle.regularise(feq + r, feq), r, atol=1e-16)


def _collide(collision, tau, fA, fB, grad, F):
    p = make_params(8, 8, 8, tau_a=tau, tau_b=tau, A_a=0.01, A_b=0.02, beta=0.7, collision=collision)
    return oracle.node_collide(p, fA, fB, grad, F)


@pytest.mark.parametrize("trial", range(3))
def test_tau_one_equals_bgk(trial):
    u = 0.02 * RNG.normal(size=3)
    fA, fB = _state(0.3, u, 0.05), _state(0.7, u, 0.05)
    grad, F = 0.3 * RNG.normal(size=3), 1e-4 * RNG.normal(size=3)
    a = _collide(0, 1.0, fA, fB, grad, F)
    b = _collide(1, 1.0, fA, fB, grad, F)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=2e-16)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.7])
def test_moments_up_to_second_order_equal_bgk(lat, tau):
    c, _ = lat
    u = 0.02 * RNG.normal(size=3)
    fA, fB = _state(0.45, u, 0.08), _state(0.55, u, 0.08)
    grad, F = 0.2 * RNG.normal(size=3), 1e-4 * RNG.normal(size=3)
    oa0, ob0, _ = _collide(0, tau, fA, fB, grad, F)
    oa1, ob1, _ = _collide(1, tau, fA, fB, grad, F)
    assert abs(oa1.sum() - fA.sum()) < 1e-15 and abs(ob1.sum() - fB.sum()) < 1e-15
    t0, t1 = oa0 + ob0, oa1 + ob1
    np.testing.assert_allclose(t1 @ c, t0 @ c, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", t1, c, c), np.einsum("i,ia,ib->ab", t0, c, c), atol=1e-15)
    assert np.abs(t1 - t0).max() > 1e-6  # the ghost content was removed


def test_hermite_state_collides_as_bgk(lat):
    c, w = lat
    u = np.array([0.01, -0.02, 0.015])
    rho = 1.0
    J = 1e-3 * RNG.normal(size=3)
    P = 1e-3 * RNG.normal(size=(3, 3))
    P = P + P.T
    Qc = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)
    neq = w * (c @ J / CS2 + np.einsum("iab,ab->i", Qc, P) / (2 * CS2 * CS2))
    f = oracle.feq(rho, u) + neq
    fA, fB = 0.4 * f, 0.6 * f
    a = _collide(0, 0.8, fA, fB, np.zeros(3), np.zeros(3))
    b = _collide(1, 0.8, fA, fB, np.zeros(3), np.zeros(3))
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=1e-15)


def test_poiseuille_regularised_same_viscosity():
    ny, g, tau = 34, 1e-6, 0.8
    p = make_params(4, ny, 4, walls=0b010, tau_a=tau, tau_b=tau, g=(0, 0, g), g_mode=1, collision=1)
    s = OracleSim(p)
    s.init_fields(-np.ones((4, ny, 4)))
    s.step(20000)
    f = s.fields()
    u = f["uz"][0, :, 0]
    nu = (tau - 0.5) / 3.0
    sec = u[1:-3] - 2 * u[2:-2] + u[3:-1]
    np.testing.assert_allclose(sec, -g / nu, rtol=1e-6)
    y = np.arange(ny)
    ua = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    assert np.abs(u[1:-1] - ua[1:-1]).max() < 0.01 * ua.max()


def test_component_mass_conserved_with_droplets():
    p = make_params(24, 24, 24, tau_a=0.7, tau_b=1.2, A_h=0.1, g=(0, 0, 1e-5), g_mode=2, collision=1)
    s = OracleSim(p)
    s.init_droplets([[12.0, 12.0, 7.0], [12.0, 12.0, 17.5]], [4.5, 4.5])
    m0 = s.reduce()
    s.step(150)
    m1 = s.reduce()
    assert abs(m1[0] - m0[0]) < 1e-12 * m0[0] and abs(m1[1] - m0[1]) < 1e-12 * m0[1]
    assert np.isfinite(s.fields()["phi"]).all()


@pytest.mark.parametrize("tau", [0.6, 0.95, 1.6])
def test_regularised_post_collision_is_w_times_a_quadratic(lat, tau):
    """Reading of the population-free (moment) storage: after the regularised
    collision every post-collision total population is w_i times a
    polynomial of degree <= 2 in c_i (ten numbers per node), and the
    component split is s f*_i + w_i c_i.v/|c_i| with one vector v; under BGK
    a state with non-hydrodynamic content leaves a remainder that ten numbers
    cannot hold."""
    c, w = lat
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    basis = np.stack([np.ones(27), x, y, z, x * x, y * y, z * z, x * y, x * z, y * z], axis=1)
    u = 0.02 * RNG.normal(size=3)
    fA, fB = _state(0.35, u, 0.08), _state(0.65, u, 0.08)
    grad, F = 0.25 * RNG.normal(size=3), 1e-4 * RNG.normal(size=3)

    def remainder(t):
        coef, *_ = np.linalg.lstsq(basis, t / w, rcond=None)
        return np.abs(basis @ coef - t / w).max()

    oa, ob, _ = _collide(1, tau, fA, fB, grad, F)
    t = oa + ob
    assert remainder(t) < 1e-14
    s = fA.sum() / (fA.sum() + fB.sum())
    norm = np.sqrt((c * c).sum(axis=1))
    seg = oa - s * t
    moving = norm > 0
    v, *_ = np.linalg.lstsq(c[moving] * (w[moving] / norm[moving])[:, None], seg[moving], rcond=None)
    assert abs(seg[~moving]).max() < 1e-16
    np.testing.assert_allclose((c[moving] @ v) * w[moving] / norm[moving], seg[moving], atol=1e-16)
    assert np.linalg.norm(v) > 1e-4  # the recolouring term is present
    oa0, ob0, _ = _collide(0, tau, fA, fB, grad, F)
    assert remainder(oa0 + ob0) > 1e-5  # BGK keeps the ghost content
