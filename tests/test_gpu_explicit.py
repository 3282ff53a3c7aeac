"""Explicit Schur blocks W_e over the extended boundary sets: the explicit condensed
operator against the oracle's dense S and the implicit operator, and a solve with it."""
import numpy as np
import pytest

import oracle as O
from gpu_common import case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(n, N, tc, explicit, cfl=10.0, **kw):
    from paper_1911_02366_gb300 import sc
    Q, dt, p, ctx = case(n, N, cfl=cfl, precision=sc.SC_PREC_MIXED, tensor_cores=tc, explicit_schur=explicit, **kw)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    return Q, dt, p, ctx


@pytest.mark.parametrize("N,tc,tol", [(2, 0, 1e-4), (3, 0, 1e-4), (4, 0, 1e-4), (3, 1, 5e-3)])
def test_explicit_operator_matches_dense_S_and_implicit_operator(N, tc, tol):
    n = 3
    Q, dt, p, ctx = _ctx(n, N, tc, 1)
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    xb = np.random.default_rng(5).standard_normal(S.shape[0])
    x = torch.tensor(xb, device="cuda")
    ye = torch.zeros_like(x)
    ctx.sc_condensed_matvec(x, ye)
    _, _, _, ci = _ctx(n, N, tc, 0)
    yi = torch.zeros_like(x)
    ci.sc_condensed_matvec(x, yi)
    torch.cuda.synchronize()
    ref = S @ xb
    assert rel(ye.cpu().numpy(), ref) < tol
    assert rel(ye.cpu().numpy(), yi.cpu().numpy()) < tol


@pytest.mark.parametrize("tc", [0, 1])
def test_explicit_solve_matches_oracle_global_solve(tc):
    n, N = 3, 2
    Q, dt, p, ctx = _ctx(n, N, tc, 1, rel_tol=1e-12, inner_tol=1e-4, gmres_restart=60, max_refine=30)
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st


def test_explicit_needs_distinct_neighbours():
    from paper_1911_02366_gb300 import sc
    from gpu_common import gpu_context
    ctx = gpu_context(precision=sc.SC_PREC_MIXED, explicit_schur=1)
    with pytest.raises(sc.SCError):
        ctx.sc_set_mesh(2, 2 * np.pi, 3)
