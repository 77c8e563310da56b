"""Pins of the oracle's per-node building blocks against closed forms.

Each test checks a property the paper (or plain lattice algebra) fixes, not a
re-typing of the oracle's formula:
  * D3Q27 isotropy up to fourth order with c_s^2 = 1/3 (Sec. III.B, Eq. disteq
    needs it);
  * the equilibrium's moments rho, rho u, rho u u + c_s^2 rho I (Eqs. eq:rho,
    eq:u, eq:Pi applied to Eq. disteq);
  * the perturbation's conservation constraints (Eqs. consconstr,
    consconstr2) and its non-ideal stress Sigma = -tau sum Omega2 c c, which
    must equal sigma delta_I (I - n n) with sigma from Eq. sigmaA;
  * the isotropy constraints on B_i (Sec. III.C.1);
  * recolouring: component mass, f^A + f^B = f*, beta = 0 proportional split
    (Eqs. ome3_1, ome3_2);
  * Guo forcing moments (sum S = 0, sum S c = (1 - 1/2tau) F,
    sum S c c = (1 - 1/2tau)(u F + F u));
  * harmonic viscosity mixing (Eq. sigmaA's definition of nu_bar).
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20240523)


@pytest.fixture(scope="module")
def lat():
    return oracle.lattice()


def test_lattice_velocity_set(lat):
    c, w, opp, B = lat
    # all 27 distinct velocities of {-1,0,1}^3
    assert len({tuple(v) for v in c}) == 27
    assert np.all(np.abs(c) <= 1)
    for i in range(27):
        assert np.array_equal(c[opp[i]], -c[i])
    # rest first (the recolouring sets cos(theta_0) = 0 for it)
    assert np.array_equal(c[0], [0, 0, 0])


def test_lattice_isotropy(lat):
    c, w, _, _ = lat
    cf = c.astype(np.float64)
    I = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, cf), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, cf, cf), I / 3.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf), 0.0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9.0
    np.testing.assert_allclose(four, iso, atol=1e-15)


def test_B_isotropy_constraints(lat):
    """Sec. III.C.1: sum B = 1/3, sum B c = 0, sum B c c = I/3."""
    c, _, _, B = lat
    cf = c.astype(np.float64)
    assert abs(B.sum() - 1.0 / 3.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", B, cf), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", B, cf, cf), np.eye(3) / 3.0, atol=1e-15)


@pytest.mark.parametrize("trial", range(5))
def test_feq_moments(lat, trial):
    c, _, _, _ = lat
    cf = c.astype(np.float64)
    rho = 0.8 + 0.4 * RNG.random()
    u = 0.1 * (RNG.random(3) - 0.5)
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(f @ cf, rho * u, atol=1e-15)
    Pi = np.einsum("i,ia,ib->ab", f, cf, cf)
    np.testing.assert_allclose(Pi, rho * np.outer(u, u) + rho / 3.0 * np.eye(3), atol=1e-14)


@pytest.mark.parametrize("trial", range(5))
def test_omega2_conservation_and_surface_tension(lat, trial):
    """Eqs. consconstr/consconstr2 and the stress that yields Eq. sigmaA."""
    c, _, _, _ = lat
    cf = c.astype(np.float64)
    A_a, A_b = 0.005 + 0.02 * RNG.random(2)
    grad = RNG.normal(size=3) * (0.05 + RNG.random())
    om = oracle.omega2(A_a, A_b, grad)
    assert abs(om.sum()) < 1e-16
    np.testing.assert_allclose(om @ cf, 0.0, atol=1e-16)
    g = np.linalg.norm(grad)
    n = grad / g
    tau = 0.6 + 1.5 * RNG.random()
    Sigma = -tau * np.einsum("i,ia,ib->ab", om, cf, cf)
    omega_bar = 1.0 / tau
    sigma = 2.0 / 9.0 * (A_a + A_b) / omega_bar  # Eq. sigmaA
    delta_I = 0.5 * g  # delta_I = |grad phi| / 2 (text after Eq. force)
    np.testing.assert_allclose(Sigma, sigma * delta_I * (np.eye(3) - np.outer(n, n)), atol=1e-15)


def test_omega2_zero_gradient():
    np.testing.assert_array_equal(oracle.omega2(0.01, 0.01, np.zeros(3)), 0.0)


def test_surface_tension_golden():
    """The paper's equal-amplitude value sigma = (4/9) A / omega_bar for the
    small-droplet workload (A = 0.01, tau = 1)."""
    with open(os.path.join(GOLDEN, "sigma_eq_sigmaA.json")) as fh:
        gold = json.load(fh)
    c, _, _, _ = oracle.lattice()
    cf = c.astype(np.float64)
    grad = np.array([0.0, 0.0, 0.4])
    om = oracle.omega2(gold["A"], gold["A"], grad)
    Sigma = -gold["tau"] * np.einsum("i,ia,ib->ab", om, cf, cf)
    sigma_measured = Sigma[0, 0] / (0.5 * 0.4)
    assert abs(sigma_measured - gold["sigma"]) < 1e-15


@pytest.mark.parametrize("trial", range(5))
def test_guo_moments(lat, trial):
    c, _, _, _ = lat
    cf = c.astype(np.float64)
    tau = 0.6 + RNG.random()
    u = 0.05 * RNG.normal(size=3)
    F = 1e-3 * RNG.normal(size=3)
    S = oracle.guo(tau, u, F)
    pref = 1.0 - 1.0 / (2.0 * tau)
    assert abs(S.sum()) < 1e-17
    np.testing.assert_allclose(S @ cf, pref * F, atol=1e-17)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", S, cf, cf),
                               pref * (np.outer(u, F) + np.outer(F, u)), atol=1e-17)


def test_tau_bar_harmonic_mixing():
    # equal relaxation times: tau itself
    assert oracle.tau_bar(1.0, 1.0, 0.3, 0.7) == 1.0
    # pure components
    assert abs(oracle.tau_bar(0.8, 1.7, 1.0, 0.0) - 0.8) < 1e-15
    assert abs(oracle.tau_bar(0.8, 1.7, 0.0, 1.0) - 1.7) < 1e-15
    # 50/50 mix: nu_bar is the harmonic mean of the viscosities nu = (tau - 1/2)/3
    nu_a, nu_b = (0.8 - 0.5) / 3.0, (1.7 - 0.5) / 3.0
    nu_bar = 2.0 / (1.0 / nu_a + 1.0 / nu_b)
    assert abs(oracle.tau_bar(0.8, 1.7, 0.5, 0.5) - (3.0 * nu_bar + 0.5)) < 1e-15


@pytest.mark.parametrize("beta", [0.0, 0.7, 1.0])
def test_recolour_properties(lat, beta):
    c, w, _, _ = lat
    cf = c.astype(np.float64)
    rhoA, rhoB = 0.3, 0.75
    fstar = oracle.feq(rhoA + rhoB, [0.01, -0.02, 0.005]) + 1e-3 * RNG.normal(size=27)
    fstar -= w * (fstar.sum() - (rhoA + rhoB))  # make sum f* = rho exactly
    grad = np.array([0.1, -0.3, 0.2])
    fa, fb = oracle.recolour(beta, rhoA, rhoB, fstar, grad)
    np.testing.assert_allclose(fa + fb, fstar, atol=1e-16)
    assert abs(fa.sum() - rhoA) < 1e-15
    assert abs(fb.sum() - rhoB) < 1e-15
    rho = rhoA + rhoB
    if beta == 0.0:
        np.testing.assert_allclose(fa, rhoA / rho * fstar, atol=1e-17)
    else:
        # the segregation flux of A points along +grad phi (into the A phase)
        flux = (fa - rhoA / rho * fstar) @ cf
        assert np.dot(flux, grad) > 0
        cross = np.cross(flux, grad)
        assert np.linalg.norm(cross) < 1e-14


@pytest.mark.parametrize("trial", range(4))
def test_node_collide_conserves(lat, trial):
    """Per-component mass (Eqs. consconstr, ome3_1/2) and momentum j + F
    (BGK conserves momentum, the half-force shift plus Guo's source add F)."""
    c, _, _, _ = lat
    cf = c.astype(np.float64)
    p = oracle.make_params(8, 8, 8, tau_a=0.7 + RNG.random(), tau_b=0.7 + RNG.random(),
                           A_a=0.01, A_b=0.02, beta=0.7)
    fA = oracle.feq(0.4, [0.01, 0.0, -0.01]) * (1 + 0.05 * RNG.random(27))
    fB = oracle.feq(0.6, [0.01, 0.0, -0.01]) * (1 + 0.05 * RNG.random(27))
    grad = RNG.normal(size=3) * 0.3
    F = 1e-4 * RNG.normal(size=3)
    oa, ob, u = oracle.node_collide(p, fA, fB, grad, F)
    assert abs(oa.sum() - fA.sum()) < 1e-15
    assert abs(ob.sum() - fB.sum()) < 1e-15
    j = (fA + fB) @ cf
    np.testing.assert_allclose((oa + ob) @ cf, j + F, atol=1e-16)
    np.testing.assert_allclose(u, (j + F / 2) / (fA.sum() + fB.sum()), atol=1e-16)


def test_node_collide_single_fluid_is_bgk(lat):
    """With one component absent the scheme reduces to plain forced BGK:
    no perturbation or recolouring survive in the total."""
    p = oracle.make_params(8, 8, 8, tau_a=0.9, tau_b=0.9, A_a=0.01, A_b=0.01, beta=0.7)
    fB = oracle.feq(1.0, [0.02, 0.0, 0.0]) + 1e-3 * RNG.normal(size=27)
    fA = np.zeros(27)
    oa, ob, u = oracle.node_collide(p, fA, fB, np.zeros(3), np.zeros(3))
    np.testing.assert_array_equal(oa, 0.0)
    rho = fB.sum()
    expect = fB + (oracle.feq(rho, u) - fB) / 0.9
    np.testing.assert_allclose(ob, expect, atol=1e-16)
