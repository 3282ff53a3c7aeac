"""Pins of the oracle's advective numerical flux (Roe with entropy fix)."""
import numpy as np
import pytest

import oracle as O

GAMMA = 1.4


def cons(rho, u, v, w, p):
    return np.array([rho, rho * u, rho * v, rho * w, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)])


P = O.Params(n=1, N=1)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_consistency(d):
    q = cons(1.1, 0.3, -0.2, 0.4, 50.0)
    for s in (-1, 1):
        fh = O.num_flux(P, q, q, d, s)
        fa, _ = O.phys_flux(P, q, np.zeros(15), d)
        np.testing.assert_allclose(fh, s * fa, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_supersonic_upwinding(d):
    # Both states supersonic along +n: every wave speed exceeds the entropy-fix width,
    # so |A_roe| = A_roe and the Roe property A_roe (qR - qL) = F(qR) - F(qL) makes the
    # flux exactly F(qL).n.  A dropped term or a wrong eigenvector breaks this.
    vel = [0.0, 0.0, 0.0]
    vel[d] = 3.0
    qL = cons(1.0, *vel, 1.0 / GAMMA)
    vel2 = list(vel); vel2[d] = 2.6; vel2[(d + 1) % 3] = 0.3
    qR = cons(1.3, *vel2, 1.2 / GAMMA)
    fL, _ = O.phys_flux(P, qL, np.zeros(15), d)
    fR, _ = O.phys_flux(P, qR, np.zeros(15), d)
    np.testing.assert_allclose(O.num_flux(P, qL, qR, d, +1), fL, rtol=1e-13, atol=1e-13)
    # and against -n the downwind state qL sits outside, so the flux is -F(qL) . e_d
    # evaluated from the right state's side: fhat(qR, qL, -e_d) = -F(qL).
    np.testing.assert_allclose(O.num_flux(P, qR, qL, d, -1), -fL, rtol=1e-13, atol=1e-13)
    assert np.max(np.abs(fL - fR)) > 1e-2


def test_roe_antisymmetry_and_rotation():
    rng = np.random.default_rng(3)
    for _ in range(20):
        qL = cons(1 + 0.2 * rng.random(), *(0.5 * rng.standard_normal(3)), 60 + rng.random())
        qR = cons(1 + 0.2 * rng.random(), *(0.5 * rng.standard_normal(3)), 60 + rng.random())
        for d in range(3):
            f1 = O.num_flux(P, qL, qR, d, +1)
            f2 = O.num_flux(P, qR, qL, d, -1)
            np.testing.assert_allclose(f1, -f2, rtol=1e-13, atol=1e-11)
        # rotating the velocity components maps the x flux onto the y flux
        perm = [0, 2, 3, 1, 4]  # (rho, v, w, u, E): y becomes the first direction
        fx = O.num_flux(P, qL[perm], qR[perm], 0, +1)
        fy = O.num_flux(P, qL, qR, 1, +1)
        np.testing.assert_allclose(fx, fy[perm], rtol=1e-13, atol=1e-11)


def test_roe_dissipation_sign():
    # The dissipation of the upwind flux is non-negative: for a pure density jump at
    # rest the mass flux moves mass from the denser to the lighter side.
    qL = cons(1.2, 0, 0, 0, 70.0)
    qR = cons(1.0, 0, 0, 0, 70.0)
    f = O.num_flux(P, qL, qR, 0, +1)
    assert f[0] > 0


PLF = O.Params(n=1, N=1, adv_flux=1)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_lax_friedrichs_consistency_and_conservation(d):
    # equal states give the physical flux; swapping the sides and the normal negates the flux
    q = cons(1.1, 0.3, -0.2, 0.4, 50.0)
    for s in (-1, 1):
        fa, _ = O.phys_flux(PLF, q, np.zeros(15), d)
        np.testing.assert_allclose(O.num_flux(PLF, q, q, d, s), s * fa, rtol=1e-14, atol=1e-12)
    qL, qR = cons(1.0, 0.2, 0.1, -0.3, 40.0), cons(1.2, -0.1, 0.4, 0.2, 45.0)
    for s in (-1, 1):
        np.testing.assert_allclose(O.num_flux(PLF, qL, qR, d, s), -O.num_flux(PLF, qR, qL, d, -s),
                                   rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_lax_friedrichs_contact_at_rest(d):
    # fluid at rest, equal pressure, a density jump: the central part carries only the
    # pressure, and the dissipation is the fastest sound speed sqrt(gamma p / rho_min) times
    # half the jump of the conserved state (energy unchanged: same pressure, no motion)
    p, rL, rR = 30.0, 1.0, 2.0
    qL, qR = cons(rL, 0, 0, 0, p), cons(rR, 0, 0, 0, p)
    lam = np.sqrt(GAMMA * p / rL)
    fh = O.num_flux(PLF, qL, qR, d, +1)
    expect = np.zeros(5)
    expect[1 + d] = p
    expect[0] = -0.5 * lam * (rR - rL)
    np.testing.assert_allclose(fh, expect, rtol=1e-13, atol=1e-12)


def test_lax_friedrichs_dissipates_more_than_roe_across_a_shear_layer():
    # a pure shear jump (same rho, p, normal velocity): Roe damps it with |u.n| only, LF with
    # |u.n| + c, so the LF flux differs from the central flux by more
    qL, qR = cons(1.0, 0.1, 0.5, 0.0, 40.0), cons(1.0, 0.1, -0.5, 0.0, 40.0)
    fL, _ = O.phys_flux(P, qL, np.zeros(15), 0)
    fR, _ = O.phys_flux(P, qR, np.zeros(15), 0)
    central = 0.5 * (fL + fR)
    d_roe = np.linalg.norm(O.num_flux(P, qL, qR, 0, 1) - central)
    d_lf = np.linalg.norm(O.num_flux(PLF, qL, qR, 0, 1) - central)
    assert d_lf > 5 * d_roe > 0
