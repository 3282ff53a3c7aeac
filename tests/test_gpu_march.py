"""Time marching towards a steady state (Sec. 4): the GPU's explicit RK3 and frozen-Jacobian
linearised BDF1 marches through the C ABI against the oracle's (oracle/march.py)."""
import numpy as np
import pytest

import oracle as O
import oracle.march as MA
import sc_inputs as I
from gpu_common import TWO_PI, gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(n, N, Re=30.0, **cfg):
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=0)
    ctx = gpu_context(Re=Re, **cfg)
    ctx.sc_set_mesh(n, TWO_PI, N)
    ctx.sc_set_timestep(dt, 1)
    ctx.sc_set_state(Q, Q)
    return Q, dt, O.Params(n=n, N=N, dt=dt, Re=Re), ctx


def test_steady_residual_matches_oracle():
    Q, dt, p, ctx = _setup(2, 3)
    got = ctx.sc_steady_residual()
    ref = MA.steady_residual(p, Q)
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("n,N,dfl", [(2, 3, 0.0), (3, 2, 0.05)])
def test_explicit_rk3_march_matches_oracle(n, N, dfl):
    Q, dt, p, ctx = _setup(n, N)
    res, dts, ms = ctx.sc_explicit_march(0.15, 6, dfl=dfl)
    q = np.zeros(Q.size)
    ctx.sc_get_state(q)
    qo, reso, dtso = MA.rk3_march(p, Q, 0.15, 6, dfl=dfl)
    assert np.max(np.abs(dts - dtso)) <= 1e-13 * np.max(dtso)
    assert np.max(np.abs(q - qo.reshape(-1))) <= 1e-12 * np.max(np.abs(qo))
    assert np.max(np.abs(res - reso) / reso) <= 1e-9
    assert ms > 0.0


@pytest.mark.parametrize("arm", ["fp64", "mixed"])
def test_frozen_jacobian_implicit_march_matches_oracle(arm):
    from paper_1911_02366_gb300 import sc
    cfg = dict(rel_tol=1e-12, gmres_restart=60, gmres_max_iters=4000)
    if arm == "mixed":
        cfg.update(precision=sc.SC_PREC_MIXED, inner_tol=1e-4, max_refine=30)
    Q, dt, p, ctx = _setup(2, 3, **cfg)
    res, ms, its = ctx.sc_implicit_march(dt, 3, jacobian_every=0)
    q = np.zeros(Q.size)
    ctx.sc_get_state(q)
    qo, reso = MA.implicit_march(p, Q, dt, 3)
    dq = qo.reshape(-1) - Q.reshape(-1)
    assert np.linalg.norm(q - qo.reshape(-1)) <= 1e-9 * np.linalg.norm(dq)
    assert np.max(np.abs(res - reso) / reso) <= 1e-7
    assert np.all(np.diff(ms) > 0) and np.all(its > 0)
    # the residual falls: the steady state of the decaying flow is approached
    assert res[-1] < res[0]


def test_implicit_march_refreshing_the_jacobian_every_step_is_newton_per_step():
    """jacobian_every = 1 re-assembles at every step: the first step equals the frozen
    march's, later steps differ (the Jacobian follows the state)."""
    Q, dt, p, ctx = _setup(2, 2, rel_tol=1e-12, gmres_restart=60)
    r1, _, _ = ctx.sc_implicit_march(dt, 2, jacobian_every=1)
    q1 = np.zeros(Q.size)
    ctx.sc_get_state(q1)
    Q2, dt2, p2, ctx2 = _setup(2, 2, rel_tol=1e-12, gmres_restart=60)
    r2, _, _ = ctx2.sc_implicit_march(dt, 2, jacobian_every=0)
    q2 = np.zeros(Q.size)
    ctx2.sc_get_state(q2)
    assert abs(r1[1] - r2[1]) <= 1e-9 * r2[1]
    assert np.max(np.abs(q1 - q2)) > 1e-10 * np.max(np.abs(q2))
