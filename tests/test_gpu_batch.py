"""Batched condensation of systems of uneven order (N = 2 .. 6) in grouped launches,
captured in a CUDA graph with autotuned tile widths: every system must come out exactly as
its own sc_condense makes it, and solve to the same answer."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I
from gpu_common import TWO_PI, gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDERS = [(3, 2), (3, 3), (2, 4), (1, 5), (1, 6)]  # (elements per direction, N)


def _context(n, N, rel_tol=1e-8):
    from paper_1911_02366_gb300 import sc
    ctx = gpu_context(precision=sc.SC_PREC_MIXED, rel_tol=rel_tol, gmres_restart=60, gmres_max_iters=4000,
                      max_refine=20)
    ctx.sc_set_mesh(n, TWO_PI, N)
    return ctx


def _load(ctx, n, N, seed):
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=seed)
    ctx.sc_set_timestep(dt, 1)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    return Q


def _solve(ctx, Q):
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    return dQ, st


@pytest.mark.parametrize("graph", [True, False])
def test_batched_condensation_equals_each_systems_own(graph):
    from paper_1911_02366_gb300 import sc
    ctxs = [_context(n, N) for n, N in ORDERS]
    batch = sc.Batch(ctxs)
    for seed in (0, 4):  # the second round replays the graph on new systems
        Qs = [_load(c, n, N, seed) for c, (n, N) in zip(ctxs, ORDERS)]
        batch.condense(graph=graph, autotune=True)
        for c, Q, (n, N) in zip(ctxs, Qs, ORDERS):
            dQ_b, st_b = _solve(c, Q)
            cr = _context(n, N)
            Qr = _load(cr, n, N, seed)
            cr.sc_condense()
            dQ_r, st_r = _solve(cr, Qr)
            assert st_b["gmres_iters"] == st_r["gmres_iters"], (N, seed, st_b, st_r)
            assert np.max(np.abs(dQ_b - dQ_r)) <= 1e-13 * np.max(np.abs(dQ_r)), (N, seed)
            assert st_b["rel_residual"] < 1e-8
    for cidx in range(len(ORDERS)):
        ni, by, bs, bt = batch.tiles(cidx)
        assert ni in (5, 40, 135, 320, 625) and {by, bs, bt} <= {64, 144, 256}
    batch.close()


def test_batched_condensation_solves_match_oracle_global_solves():
    """Every system of one graph-captured, autotuned batch over the orders N = 2..6 solves
    to the oracle's global sparse-LU solution x = A^-1 B (Sec. 2.1, eq. NewtonLinSys1) within
    the mixed arm's bound after FP64 refinement."""
    from paper_1911_02366_gb300 import sc
    ctxs = [_context(n, N, rel_tol=1e-12) for n, N in ORDERS]
    batch = sc.Batch(ctxs)
    Qs = [_load(c, n, N, 2) for c, (n, N) in zip(ctxs, ORDERS)]
    batch.condense(graph=True, autotune=True)
    for c, Q, (n, N) in zip(ctxs, Qs, ORDERS):
        dQ, st = _solve(c, Q)
        _, dt = I.tgv_state(n, N, cfl=10.0, seed=2)
        p = O.Params(n=n, N=N, dt=dt)
        A = O.jacobian(p, Q)
        B = -O.residual(p, Q).reshape(-1)
        x = O.global_solve(A, B)
        assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11, (N, st)
        assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, (N, st)
    batch.close()


def test_batch_rejects_unsupported_systems():
    from paper_1911_02366_gb300 import sc
    ctx = gpu_context(precision=sc.SC_PREC_FP64)
    ctx.sc_set_mesh(2, TWO_PI, 2)
    with pytest.raises(sc.SCError):
        sc.Batch([ctx])
