"""Parity of the CUDA path with the FP64 oracle at N = 5 and N = 6 (n_i = 320 and 625:
the interior inverses take the blocked Gauss-Jordan path, the S_ee blocks 760 and 1090
rows the shared-memory panel LU)."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I
from gpu_common import case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HIGH = [(1, 5), (2, 5), (1, 6)]


@pytest.mark.parametrize("n,N", HIGH)
def test_residual_and_jacobian_blocks_match_oracle(n, N):
    # the assembly is FP64 on both arms; N = 6 exists on the mixed arm only
    from paper_1911_02366_gb300 import sc
    prec = sc.SC_PREC_MIXED if N == 6 else sc.SC_PREC_FP64
    Q, dt, p, ctx = case(n, N, eps=1e-2, precision=prec)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    B = ctx.sc_get_rhs(np.zeros(Q.size)).reshape(Q.shape)
    assert rel(B, -O.residual(p, Q)) < 1e-12
    A = O.jacobian(p, Q).tocsr()
    ne = p.nn * 5
    scale = abs(A).max()
    for e in sorted({0, p.K - 1}):
        rows = A[e * ne:(e + 1) * ne]
        for c in sorted(set(np.unique(rows.indices // ne).tolist())):
            ref = rows[:, c * ne:(c + 1) * ne].toarray()
            err = np.abs(ctx.sc_get_jacobian_block(e, c) - ref).max() / scale
            assert err < 1e-11, (e, c, err)


@pytest.mark.parametrize("n,N", [(1, 5), (2, 5)])
def test_fp64_condensed_operator_matches_oracle(n, N):
    Q, dt, p, ctx = case(n, N)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    xb = np.random.default_rng(7).standard_normal(S.shape[0])
    yb = torch.zeros(S.shape[0], dtype=torch.float64, device="cuda")
    ctx.sc_condensed_matvec(torch.tensor(xb, device="cuda"), yb)
    torch.cuda.synchronize()
    assert rel(yb.cpu().numpy(), S @ xb) < 1e-11


@pytest.mark.parametrize("N", [5, 6])
def test_mixed_condensed_operator_is_fp32_close(N):
    from paper_1911_02366_gb300 import sc
    n = 1
    Q, dt, p, ctx = case(n, N, precision=sc.SC_PREC_MIXED)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    xb = np.random.default_rng(8).standard_normal(S.shape[0])
    yb = torch.zeros(S.shape[0], dtype=torch.float64, device="cuda")
    ctx.sc_condensed_matvec(torch.tensor(xb, device="cuda"), yb)
    torch.cuda.synchronize()
    assert rel(yb.cpu().numpy(), S @ xb) < 1e-4


def test_fp64_solve_matches_oracle_global_solve_n5():
    n, N = 2, 5
    Q, dt, p, ctx = case(n, N, cfl=10.0, rel_tol=1e-13, gmres_restart=60, gmres_max_iters=3000)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-12
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-10, st


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("n,N", [(2, 5), (1, 6)])
def test_mixed_solve_matches_oracle_global_solve(n, N, tc):
    from paper_1911_02366_gb300 import sc
    Q, dt, p, ctx = case(n, N, cfl=10.0, precision=sc.SC_PREC_MIXED, rel_tol=1e-12, inner_tol=1e-4,
                         gmres_restart=60, gmres_max_iters=4000, max_refine=20, tensor_cores=tc)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st


def test_mixed_solve_n6_on_2x2x2_reaches_1e8_against_oracle_residual():
    # 13,720 unknowns: the oracle's Jacobian-vector product checks the global residual
    from paper_1911_02366_gb300 import sc
    n, N = 2, 6
    Q, dt, p, ctx = case(n, N, cfl=10.0, precision=sc.SC_PREC_MIXED, gmres_restart=60, gmres_max_iters=4000,
                         max_refine=20)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    B = -O.residual(p, Q).reshape(-1)
    r = B - O.jvp(p, Q, dQ.reshape(Q.shape)).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(B) < 1e-8 * 1.01, st


def test_fp64_arm_rejects_order_6_and_explicit_rejects_order_5():
    from paper_1911_02366_gb300 import sc
    from gpu_common import gpu_context
    ctx = gpu_context()
    with pytest.raises(sc.SCError):
        ctx.sc_set_mesh(1, 2 * np.pi, 6)
    ctx = gpu_context(precision=sc.SC_PREC_MIXED, explicit_schur=1)
    with pytest.raises(sc.SCError):
        ctx.sc_set_mesh(3, 2 * np.pi, 5)
