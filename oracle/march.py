"""Time marching of the GL-DGSEM towards a steady state (test infrastructure only).

Sec. 4 (numerical example) drives the discretisation to a steady state, measured by
||M^-1 H(Q)||_inf, three ways: Williamson's low-storage third-order Runge-Kutta scheme with
a CFL-adapted step, and BDF1 steps with a fixed step whose Newton-linearised systems reuse
one Jacobian (solved globally or by static condensation).  Here:

* M: the diagonal Gauss-Lobatto mass matrix, M_jj = J w_a w_b w_c, J = (h/2)^3;
* H(Q): the oracle's residual with the time term dropped (``with_time = False``);
* RK3 (Williamson 1980, the 2N-storage form): for stages k = 1, 2, 3,
  dq <- A_k dq + dt f(q), q <- q + B_k dq, with f = -M^-1 H, A = (0, -5/9, -153/128),
  B = (1/3, 15/16, 8/15);
* time step: dt = min(cfl (h/N) / max(|v| + c), dfl (h/N)^2 / max(max(4/3, gamma/Pr) mu/(rho Re)))
  over all nodes, re-evaluated at the start of every step (dfl <= 0: no diffusive limit);
* linearised BDF1 with a frozen Jacobian: A0 = M/dt + dH/dQ at the initial state, then
  every step solves A0 dQ = -H(Q) (the Newton system of eq. NeqtonEq at the step's start,
  where Q equals the history) by sparse LU and sets Q <- Q + dQ.
"""
from __future__ import annotations

import dataclasses

import numpy as np

RK3_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK3_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)


def mass_diagonal(p) -> np.ndarray:
    """M_jj = J w_a w_b w_c per node, shape [nn] (the same for every element)."""
    from . import gl
    _, w, _ = gl(p.N)
    J = (p.L / p.n / 2.0) ** 3
    return J * np.einsum("i,j,k->kji", w, w, w).reshape(-1)


def spatial_operator(p, Q: np.ndarray) -> np.ndarray:
    """H(Q) [K, nn, 5]: the residual of eq. NeqtonEq without the time term."""
    from . import residual
    ps = dataclasses.replace(p, with_time=False)
    return residual(ps, Q)


def rhs(p, Q: np.ndarray) -> np.ndarray:
    """f(Q) = -M^-1 H(Q)."""
    return -spatial_operator(p, Q) / mass_diagonal(p)[None, :, None]


def steady_residual(p, Q: np.ndarray) -> float:
    """||M^-1 H(Q)||_inf."""
    return float(np.max(np.abs(rhs(p, Q))))


def time_step(p, Q: np.ndarray, cfl: float, dfl: float = 0.0) -> float:
    """The CFL-adapted explicit step of the state Q (formula in the module docstring)."""
    q = Q.reshape(-1, 5)
    rho = q[:, 0]
    v = q[:, 1:4] / rho[:, None]
    vv = np.sum(v * v, axis=1)
    pr = (p.gamma - 1.0) * (q[:, 4] - 0.5 * rho * vv)
    s = np.sqrt(vv) + np.sqrt(p.gamma * pr / rho)
    dx = p.L / p.n / p.N
    dt = cfl * dx / np.max(s)
    if dfl > 0.0:
        mu = np.ones_like(rho)
        if p.sutherland:
            T = p.gamma * p.Ma ** 2 * pr / rho
            mu = (1.0 + p.Ts) * T ** 1.5 / (T + p.Ts)
        nu = max(4.0 / 3.0, p.gamma / p.Pr) * mu / (rho * p.Re)
        dt = min(dt, dfl * dx * dx / np.max(nu))
    return float(dt)


def rk3_step(f, q, dt: float):
    """One step of the 2N-storage scheme for q' = f(q): the register dq starts at zero and
    the first stage's A = 0 discards it."""
    dq = np.zeros_like(q)
    for a, b in zip(RK3_A, RK3_B):
        dq = a * dq + dt * f(q)
        q = q + b * dq
    return q


def rk3_march(p, Q: np.ndarray, cfl: float, nsteps: int, dfl: float = 0.0):
    """nsteps RK3 steps; returns (Q, residual history [nsteps + 1], dt history [nsteps])."""
    q = np.array(Q, dtype=np.float64, copy=True)
    res, dts = [steady_residual(p, q)], []
    for _ in range(nsteps):
        dt = time_step(p, q, cfl, dfl)
        q = rk3_step(lambda x: rhs(p, x), q, dt)
        dts.append(dt)
        res.append(steady_residual(p, q))
    return q, np.array(res), np.array(dts)


def implicit_march(p, Q: np.ndarray, dt: float, nsteps: int):
    """nsteps linearised BDF1 steps with the Jacobian of the initial state; returns
    (Q, residual history [nsteps + 1])."""
    import scipy.sparse.linalg as spla
    from . import jacobian
    q = np.array(Q, dtype=np.float64, copy=True)
    pt = dataclasses.replace(p, dt=dt, bdf=1, with_time=True)
    lu = spla.splu(jacobian(pt, q).tocsc())
    res = [steady_residual(p, q)]
    for _ in range(nsteps):
        q = q + lu.solve(-spatial_operator(p, q).reshape(-1)).reshape(q.shape)
        res.append(steady_residual(p, q))
    return q, np.array(res)
