"""One periodic mesh of mixed polynomial order on the GPU (mortar faces between orders)
through the C ABI, against the oracle's mixed-order discretisation: residual,
Jacobian-vector products, element blocks, and the condensed solve against the oracle's
global solve."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I
from gpu_common import TWO_PI, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(n, orders, force_mortar=False, cfl=10.0, seed=0, **cfg):
    from paper_1911_02366_gb300 import sc
    Q, dt = I.tgv_state_mixed(n, orders, cfl=cfl, eps=1e-2, seed=seed)
    Q = np.ascontiguousarray(Q.reshape(-1))
    p = O.Params(n=n, N=int(max(orders)), dt=dt, adv_flux=cfg.get("adv_flux", 0))
    ctx = sc.MixedContext(n, orders, TWO_PI, force_mortar=force_mortar,
                          stream=torch.cuda.current_stream().cuda_stream, **cfg)
    ctx.set_state(Q, Q, dt=dt)
    return Q, p, ctx


CASES = [(2, "draw", False), (2, "draw", True), (3, "draw", False), (2, "equal", True)]


def _orders(n, kind):
    if kind == "equal":
        return np.full(n ** 3, 3, np.int32)
    return I.order_draw(1, n ** 3)


@pytest.mark.parametrize("n,kind,fm", CASES)
def test_mixed_residual_and_jvp_match_oracle(n, kind, fm):
    orders = _orders(n, kind)
    Q, p, ctx = _case(n, orders, fm)
    R = ctx.residual(np.zeros_like(Q))
    Ro = O.residual_mixed(p, orders, Q.reshape(-1, 5), force_mortar=fm).reshape(-1)
    assert rel(R, Ro) < 1e-12
    x = np.random.default_rng(4).standard_normal(Q.size)
    y = ctx.jvp(x, np.zeros_like(x))
    yo = O.jvp_mixed(p, orders, Q.reshape(-1, 5), x.reshape(-1, 5), force_mortar=fm).reshape(-1)
    assert rel(y, yo) < 1e-12


@pytest.mark.parametrize("n,kind,fm", CASES[:3])
def test_mixed_element_blocks_match_oracle(n, kind, fm):
    orders = _orders(n, kind)
    Q, p, ctx = _case(n, orders, fm)
    for e in sorted({0, n ** 3 // 2, n ** 3 - 1, int(np.argmax(orders)), int(np.argmin(orders))}):
        ref = O.jacobian_mixed_element_rows(p, orders, Q.reshape(-1, 5), e, force_mortar=fm)[e]
        got = ctx.own_block(e)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), e


def test_mixed_condensed_solve_reaches_the_oracle_residual():
    # 3^3 mesh of drawn orders: the residual of the solution through the oracle's own
    # Jacobian-vector product (its full Jacobian at this size is minutes of host time)
    from paper_1911_02366_gb300 import sc
    n = 3
    orders = _orders(n, "draw")
    Q, p, ctx = _case(n, orders, rel_tol=1e-11, gmres_restart=60, gmres_max_iters=6000, inner_tol=1e-4,
                      max_refine=30, precond=sc.SC_PC_BLOCK_JACOBI)
    ctx.condense()
    dQ = np.zeros_like(Q)
    st = ctx.solve(dQ)
    B = -O.residual_mixed(p, orders, Q.reshape(-1, 5)).reshape(-1)
    AdQ = O.jvp_mixed(p, orders, Q.reshape(-1, 5), dQ.reshape(-1, 5)).reshape(-1)
    assert np.linalg.norm(B - AdQ) / np.linalg.norm(B) < 1e-10, st
    assert st["refinements"] >= 1 and st["gmres_iters"] > 0


def test_mixed_condensed_solve_matches_oracle_global_solve_bdf2_on_device():
    from paper_1911_02366_gb300 import sc
    n = 2
    orders = _orders(n, "draw")
    Q, dt = I.tgv_state_mixed(n, orders, cfl=10.0, eps=1e-2, seed=5)
    Q = np.ascontiguousarray(Q.reshape(-1))
    Qs = Q * (1 + 1e-3)
    Qsm1 = Q * (1 - 1e-3)
    p = O.Params(n=n, N=int(max(orders)), dt=dt, bdf=2)
    ctx = sc.MixedContext(n, orders, TWO_PI, stream=torch.cuda.current_stream().cuda_stream, rel_tol=1e-11,
                          gmres_restart=40, max_refine=30)
    dev = lambda a: torch.tensor(a, device="cuda")
    ctx.set_state(dev(Q), dev(Qs), dev(Qsm1), dt=dt, bdf=2)
    ctx.condense()
    dQ = torch.zeros(Q.size, dtype=torch.float64, device="cuda")
    ctx.solve(dQ)
    A = O.jacobian_mixed_sparse(p, orders, Q.reshape(-1, 5))
    B = -O.residual_mixed(p, orders, Q.reshape(-1, 5), Qs.reshape(-1, 5), Qsm1.reshape(-1, 5)).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(dQ.cpu().numpy() - x) / np.linalg.norm(x) < 1e-8


def test_mixed_full_size_mesh_of_the_benchmark():
    # the 12^3 mesh of orders drawn from 2..6 (seed 1) that bench.py --arm mixedmesh times, in
    # its launch configuration: residual against the oracle's, sampled element blocks against
    # the oracle's element rows, and the solve to 1e-8 checked through the oracle's product
    from paper_1911_02366_gb300 import sc
    n = 12
    orders = I.order_draw(1, n ** 3)
    Q, p, ctx = _case(n, orders, cfl=10.0, rel_tol=1e-8, inner_tol=1e-4, max_refine=20)
    Q2 = Q.reshape(-1, 5)
    R = ctx.residual(np.zeros_like(Q))
    assert rel(R, O.residual_mixed(p, orders, Q2).reshape(-1)) < 1e-12
    for e in (int(np.argmax(orders)), int(np.argmin(orders)), 1000):
        ref = O.jacobian_mixed_element_rows(p, orders, Q2, e)[e]
        assert np.abs(ctx.own_block(e) - ref).max() <= 1e-11 * np.abs(ref).max(), e
    ctx.condense()
    dQ = np.zeros_like(Q)
    st = ctx.solve(dQ)
    B = -R
    AdQ = O.jvp_mixed(p, orders, Q2, dQ.reshape(-1, 5)).reshape(-1)
    assert np.linalg.norm(B - AdQ) / np.linalg.norm(B) < 1.01e-8, st


def test_mixed_lax_friedrichs_residual_products_and_blocks_match_oracle():
    from paper_1911_02366_gb300 import sc
    n = 2
    orders = _orders(n, "draw")
    Q, p, ctx = _case(n, orders, adv_flux=sc.SC_FLUX_LF)
    assert p.adv_flux == 1
    R = ctx.residual(np.zeros_like(Q))
    assert rel(R, O.residual_mixed(p, orders, Q.reshape(-1, 5)).reshape(-1)) < 1e-12
    assert rel(R, O.residual_mixed(O.Params(**{**p.__dict__, "adv_flux": 0}), orders, Q.reshape(-1, 5)).reshape(-1)) > 1e-8
    x = np.random.default_rng(6).standard_normal(Q.size)
    y = ctx.jvp(x, np.zeros_like(x))
    assert rel(y, O.jvp_mixed(p, orders, Q.reshape(-1, 5), x.reshape(-1, 5)).reshape(-1)) < 1e-12
    e = int(np.argmax(orders))
    ref = O.jacobian_mixed_element_rows(p, orders, Q.reshape(-1, 5), e)[e]
    assert np.abs(ctx.own_block(e) - ref).max() <= 1e-11 * np.abs(ref).max()
