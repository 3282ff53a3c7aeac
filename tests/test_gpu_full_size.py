"""Parity at the full sizes of the workloads, in the bench's launch configuration, on
outputs the oracle computes directly: the whole residual vector, the Jacobian rows of
sampled elements, and the FP64 global residual ||B - A dQ|| / ||B|| of the GPU solution
evaluated with the oracle's own Jacobian-vector product."""
import math

import numpy as np
import pytest

import oracle as O
import sc_inputs as I
from gpu_common import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _full_case(n, N, precision, cfl=50.0, **cfg):
    from paper_1911_02366_gb300 import sc
    Q, dt = I.tgv_state(n, N, Ma=0.1, seed=0, cfl=cfl)
    p = O.Params(n=n, N=N, dt=dt, bdf=1)
    stream = torch.cuda.current_stream()
    ctx = sc.Context(stream=stream.cuda_stream, precision=precision, Re=1600.0, Ma=0.1, gmres_restart=30,
                     gmres_max_iters=4000, rel_tol=1e-8, inner_tol=1e-4, max_refine=20, **cfg)
    ctx.sc_set_mesh(n, 2 * math.pi, N)
    ctx.sc_set_timestep(dt, 1)
    Qd = torch.tensor(Q.reshape(-1), device="cuda")
    ctx.sc_set_state(Qd, Qd)
    return Q, p, ctx, Qd


def test_bench_workload_16x16x16_N4_residual_jacobian_and_solve():
    from paper_1911_02366_gb300 import sc
    n, N = 16, 4
    Q, p, ctx, Qd = _full_case(n, N, sc.SC_PREC_MIXED, tensor_cores=1)
    ctx.sc_assemble()
    B = ctx.sc_get_rhs(np.zeros(Q.size))
    Bref = -O.residual(p, Q).reshape(-1)
    assert rel(B, Bref) < 1e-12
    # Jacobian rows of sampled elements: a corner, an interior and the last element
    ne = p.nn * 5
    for e in (0, 1365, p.K - 1):
        rows = O.jacobian_element_rows(p, Q, e)
        scale = max(np.abs(b).max() for b in rows.values())
        # nonzero: the element, its 6 face and 12 edge neighbours (BR1); the corner
        # neighbours do not couple, and the GPU stencil leaves them out
        nonzero = {c: b for c, b in rows.items() if np.any(b)}
        assert len(nonzero) == 19
        for c, ref in nonzero.items():
            err = np.abs(ctx.sc_get_jacobian_block(e, c) - ref).max() / scale
            assert err < 1e-11, (e, c, err)
    ctx.sc_condense()
    dQ = torch.zeros_like(Qd)
    st = ctx.sc_solve(dQ)
    x = dQ.cpu().numpy()
    r = Bref - O.jvp(p, Q, x.reshape(Q.shape)).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(Bref) < 1e-8 * 1.01, st
    assert st["rel_residual"] < 1e-8
    ctx.close()


def test_fp64_arm_16x16x16_N4_solve():
    from paper_1911_02366_gb300 import sc
    n, N = 16, 4
    Q, p, ctx, Qd = _full_case(n, N, sc.SC_PREC_FP64)
    ctx.sc_assemble()
    ctx.sc_condense()
    dQ = torch.zeros_like(Qd)
    st = ctx.sc_solve(dQ)
    Bref = -O.residual(p, Q).reshape(-1)
    r = Bref - O.jvp(p, Q, dQ.cpu().numpy().reshape(Q.shape)).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(Bref) < 1e-8 * 1.01, st
    ctx.close()


def test_order5_16x16x16_mixed_solve():
    # the mesh of the learned-preconditioner workload (4,423,680 DOF), block Jacobi
    from paper_1911_02366_gb300 import sc
    n, N = 16, 5
    Q, p, ctx, Qd = _full_case(n, N, sc.SC_PREC_MIXED, tensor_cores=1)
    ctx.sc_assemble()
    Bref = -O.residual(p, Q).reshape(-1)
    rows = {c: b for c, b in O.jacobian_element_rows(p, Q, 2047).items() if np.any(b)}
    scale = max(np.abs(b).max() for b in rows.values())
    for c, ref in rows.items():
        assert np.abs(ctx.sc_get_jacobian_block(2047, c) - ref).max() / scale < 1e-11, c
    ctx.sc_condense()
    dQ = torch.zeros_like(Qd)
    st = ctx.sc_solve(dQ)
    r = Bref - O.jvp(p, Q, dQ.cpu().numpy().reshape(Q.shape)).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(Bref) < 1e-8 * 1.01, st
    ctx.close()
