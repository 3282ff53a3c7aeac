"""The paper's flux pair (Sec. 4): the Lax-Friedrichs advective flux and the symmetric
interior-penalty viscous flux, through the C ABI: residual, Jacobian blocks and condensed
solves against the oracle with the same fluxes."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I
from gpu_common import TWO_PI, gpu_context, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lf_case(n, N, cfl=10.0, visc_flux=0, ip_penalty=1.0, Re=1600.0, **cfg):
    from paper_1911_02366_gb300 import sc
    Q, dt = I.tgv_state(n, N, cfl=cfl, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt, adv_flux=1, visc_flux=visc_flux, ip_penalty=ip_penalty, Re=Re)
    ctx = gpu_context(adv_flux=sc.SC_FLUX_LF, visc_flux=visc_flux, ip_penalty=ip_penalty, Re=Re, **cfg)
    ctx.sc_set_mesh(n, TWO_PI, N)
    ctx.sc_set_timestep(dt, 1)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    return Q, p, ctx


@pytest.mark.parametrize("n,N", [(2, 2), (3, 2), (2, 3)])
def test_lax_friedrichs_residual_and_jacobian_match_oracle(n, N):
    Q, p, ctx = _lf_case(n, N)
    B = ctx.sc_get_rhs(np.zeros(Q.size)).reshape(Q.shape)
    R = O.residual(p, Q)
    assert rel(B, -R) < 1e-12
    R_roe = O.residual(O.Params(n=n, N=N, dt=p.dt), Q)
    assert rel(B, -R_roe) > 1e-8  # the flux option is in effect
    A = O.jacobian(p, Q).tocsr()
    ne = p.nn * 5
    scale = abs(A).max()
    for e in range(p.K):
        rows = A[e * ne:(e + 1) * ne]
        for c in sorted(set(np.unique(rows.indices // ne).tolist())):
            err = np.abs(ctx.sc_get_jacobian_block(e, c) - rows[:, c * ne:(c + 1) * ne].toarray()).max() / scale
            assert err < 1e-11, (e, c, err)


@pytest.mark.parametrize("arm", ["fp64", "mixed"])
def test_lax_friedrichs_solve_matches_oracle_global_solve(arm):
    from paper_1911_02366_gb300 import sc
    cfg = dict(rel_tol=1e-12, gmres_restart=60, gmres_max_iters=4000)
    if arm == "mixed":
        cfg.update(precision=sc.SC_PREC_MIXED, precond=sc.SC_PC_RB_SCHUR, inner_tol=1e-4, max_refine=30)
    Q, p, ctx = _lf_case(2, 3, **cfg)
    ctx.sc_condense()
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ, raise_on_not_converged=False)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11, st
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st


def _blocks_match(ctx, p, Q, tol=1e-11):
    A = O.jacobian(p, Q).tocsr()
    ne = p.nn * 5
    scale = abs(A).max()
    n = p.n
    for e in range(p.K):
        rows = A[e * ne:(e + 1) * ne]
        cols = set(np.unique(rows.indices // ne).tolist())
        for c in sorted(cols):
            err = np.abs(ctx.sc_get_jacobian_block(e, c) - rows[:, c * ne:(c + 1) * ne].toarray()).max() / scale
            assert err < tol, (e, c, err)
        # every face or edge neighbour that the oracle leaves out is zero on the GPU too (the
        # library's stencil holds both; corner neighbours are outside it)
        ex, ey, ez = e % n, (e // n) % n, e // (n * n)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    c = (ex + dx) % n + n * (((ey + dy) % n) + n * ((ez + dz) % n))
                    if abs(dx) + abs(dy) + abs(dz) <= 2 and c not in cols:
                        assert np.abs(ctx.sc_get_jacobian_block(e, c)).max() == 0.0, (e, c)


@pytest.mark.parametrize("n,N,adv", [(2, 2, 1), (3, 2, 1), (2, 3, 1), (3, 3, 0), (2, 4, 1)])
def test_interior_penalty_residual_and_jacobian_match_oracle(n, N, adv):
    from paper_1911_02366_gb300 import sc
    Q, dt = I.tgv_state(n, N, cfl=10.0, eps=1e-2)
    kw = dict(visc_flux=1, ip_penalty=1.5, Re=100.0)
    p = O.Params(n=n, N=N, dt=dt, adv_flux=adv, **kw)
    ctx = gpu_context(adv_flux=adv, **kw)
    ctx.sc_set_mesh(n, TWO_PI, N)
    ctx.sc_set_timestep(dt, 1)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    B = ctx.sc_get_rhs(np.zeros(Q.size)).reshape(Q.shape)
    R = O.residual(p, Q)
    assert rel(B, -R) < 1e-12
    R_br1 = O.residual(O.Params(**{**p.__dict__, "visc_flux": 0}), Q)
    assert rel(B, -R_br1) > 1e-8  # the flux option is in effect
    _blocks_match(ctx, p, Q)
    # compact: no element couples to an edge neighbour (n = 3 keeps them distinct)
    if n == 3:
        e = 13
        for c in (e + 1 + 3, e - 1 - 9, e + 3 + 9):
            assert np.abs(ctx.sc_get_jacobian_block(e, c)).max() == 0.0


@pytest.mark.parametrize("arm", ["fp64", "mixed"])
def test_paper_flux_pair_solve_matches_oracle_global_solve(arm):
    from paper_1911_02366_gb300 import sc
    cfg = dict(rel_tol=1e-12, gmres_restart=60, gmres_max_iters=4000)
    if arm == "mixed":
        cfg.update(precision=sc.SC_PREC_MIXED, precond=sc.SC_PC_RB_SCHUR, inner_tol=1e-4, max_refine=30)
    Q, p, ctx = _lf_case(2, 3, visc_flux=1, **cfg)
    ctx.sc_condense()
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ, raise_on_not_converged=False)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11, st
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st
