"""Pins of the time-marching oracle (oracle/march.py): the explicit RK3 scheme and the
linearised BDF1 steps of Sec. 4's steady-state experiment."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import oracle.march as MA
import sc_inputs as I


@pytest.mark.parametrize("z", [-0.3, -1.7, 0.5 + 1.2j, -2.4 + 0.7j])
def test_rk3_step_amplification_is_the_cubic_taylor_polynomial(z):
    """A three-stage third-order scheme advances y' = lambda y by exactly
    1 + z + z^2/2 + z^3/6, z = lambda dt."""
    lam, dt = z / 0.25, 0.25
    y1 = MA.rk3_step(lambda y: lam * y, np.array([1.0 + 0j]), dt)[0]
    assert abs(y1 - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-14


def test_rk3_global_error_is_third_order():
    """y' = -y^2, y(0) = 1 (exact 1/(1+t)) to t = 1: halving dt cuts the error 8x."""
    errs = []
    for nst in (20, 40, 80):
        y, dt = np.array([1.0]), 1.0 / nst
        for _ in range(nst):
            y = MA.rk3_step(lambda x: -x * x, y, dt)
        errs.append(abs(y[0] - 0.5))
    assert 7.0 < errs[0] / errs[1] < 9.0 and 7.0 < errs[1] / errs[2] < 9.0


def test_time_step_closed_form_at_rest():
    """Uniform state at rest, rho = 1, p = 1/(gamma Ma^2): c = 1/Ma, T = 1, mu = 1, so
    dt = cfl (h/N) Ma, and the diffusive limit dfl (h/N)^2 Re / max(4/3, gamma/Pr)."""
    p = O.Params(n=2, N=3)
    Q = np.zeros((p.K, p.nn, 5))
    Q[..., 0] = 1.0
    Q[..., 4] = 1.0 / (p.gamma * p.Ma ** 2) / (p.gamma - 1.0)
    dx = p.L / p.n / p.N
    assert abs(MA.time_step(p, Q, 0.7) - 0.7 * dx * p.Ma) < 1e-15
    lim = 0.01 * dx * dx * p.Re / max(4 / 3, p.gamma / p.Pr)
    assert abs(MA.time_step(p, Q, 1e6, dfl=0.01) - lim) < 1e-12 * lim


def test_free_stream_is_a_steady_state_of_both_marches():
    p = O.Params(n=2, N=2)
    Q = np.zeros((p.K, p.nn, 5))
    Q[..., 0], Q[..., 1], Q[..., 2] = 1.0, 0.8, -0.3
    Q[..., 4] = 1.0 / (p.gamma * p.Ma ** 2) / (p.gamma - 1.0) + 0.5 * (0.64 + 0.09)
    assert MA.steady_residual(p, Q) < 1e-9
    q1, res, _ = MA.rk3_march(p, Q, 0.5, 2)
    assert np.max(np.abs(q1 - Q)) < 1e-12
    q2, res2 = MA.implicit_march(p, Q, 0.1, 2)
    assert np.max(np.abs(q2 - Q)) < 1e-12


def _tgv(n=2, N=3, Re=30.0):
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=0)
    return O.Params(n=n, N=N, dt=dt, Re=Re), Q, dt


def test_both_marches_conserve_the_mass_weighted_totals():
    """Periodic mesh: sum_j M_jj f_j = -sum_j H_j = 0 per variable, so RK3 keeps sum M q;
    each linearised BDF1 step solves (M/dt + dH/dQ) dQ = -H(Q), whose weighted column sums
    of dH/dQ vanish, so it keeps sum M q as well."""
    p, Q, dt = _tgv()
    M = MA.mass_diagonal(p)[None, :, None]
    tot0 = np.sum(M * Q, axis=(0, 1))
    q1, _, _ = MA.rk3_march(p, Q, 0.15, 3)
    q2, _ = MA.implicit_march(p, Q, dt, 2)
    for q in (q1, q2):
        assert np.max(np.abs(np.sum(M * q, axis=(0, 1)) - tot0)) < 1e-11 * np.max(np.abs(tot0))


def test_linearised_bdf1_step_solves_the_bdf1_equation_up_to_second_order():
    """One step from Q0 with the Jacobian of Q0 is one Newton step on
    R(Q) = M (Q - Q0)/dt + H(Q) = 0 from Q0: R(Q1) is second order in the update, so it is
    far below R(Q0) = H(Q0); for a linear spatial operator (the advection-diffusion model)
    R(Q1) vanishes."""
    p, Q, dt = _tgv()
    q1, _ = MA.implicit_march(p, Q, dt, 1)
    pt = dataclasses.replace(p, dt=dt, bdf=1, with_time=True)
    r0 = np.linalg.norm(O.residual(pt, Q, Qs=Q))
    r1 = np.linalg.norm(O.residual(pt, q1, Qs=Q))
    assert r1 < 1e-3 * r0
    pl = O.Params(n=2, N=3, dt=dt, model=1, nu=0.05, adv=(1.0, 0.5, 0.2))
    q1, _ = MA.implicit_march(pl, Q, dt, 1)
    ptl = dataclasses.replace(pl, with_time=True)
    assert np.linalg.norm(O.residual(ptl, q1, Qs=Q)) < 1e-11 * np.linalg.norm(O.residual(ptl, Q, Qs=Q))
