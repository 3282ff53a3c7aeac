"""Red-black block Gauss-Seidel preconditioner of the condensed system through the C ABI:
one application against the oracle's sweep on its dense S, solves against the oracle's global
solve, and the iteration count against block Jacobi."""
import numpy as np
import pytest

import oracle as O
from gpu_common import case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _system(n, N, cfl=10.0, **cfg):
    Q, dt, p, ctx = case(n, N, cfl=cfl, **cfg)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    return Q, dt, p, ctx


@pytest.mark.parametrize("arm", ["fp64", "mixed"])
@pytest.mark.parametrize("n,N", [(4, 2), (2, 3)])
def test_red_black_apply_satisfies_the_sweep_equations_with_oracle_S(arm, n, N):
    """z = P v must solve the sweep's block equations with the oracle's dense S:
    S_rr z_r = v_r on red elements, S_bb z_b = v_b - sum_{red m} S_bm z_m on black ones.
    Checked as a backward error (residual of those equations against ||S|| ||z|| + ||v||),
    which does not depend on the conditioning of the element blocks; the forward difference
    to the oracle's own sweep is kappa(S_ee) times larger."""
    from paper_1911_02366_gb300 import sc
    cfg = dict(precond=sc.SC_PC_RED_BLACK)
    if arm == "mixed":
        cfg["precision"] = sc.SC_PREC_MIXED
    Q, dt, p, ctx = _system(n, N, **cfg)
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    K = n ** 3
    nb = S.shape[0] // K
    v = np.random.default_rng(3).standard_normal(S.shape[0])
    zt = torch.zeros(S.shape[0], dtype=torch.float64, device="cuda")
    ctx.sc_precond_apply(torch.tensor(v, device="cuda"), zt)
    z = zt.cpu().numpy()
    col = O.checkerboard(n)
    red = np.repeat(col == 0, nb)
    zr = np.where(red, z, 0.0)
    t = S @ zr  # black rows: sum over red m of S_bm z_m
    r = np.empty_like(v)
    for e in range(K):
        sl = slice(e * nb, (e + 1) * nb)
        r[sl] = S[sl, sl] @ z[sl] - v[sl] + (t[sl] if col[e] == 1 else 0.0)
    scale = np.max(np.sum(np.abs(S), axis=1)) * np.max(np.abs(z)) + np.max(np.abs(v))
    # the level the element factors themselves reach (S_ee is formed with the explicit interior
    # inverse): the red rows, plain block Jacobi, show it as well as the black ones
    tol = 1e-7 if arm == "fp64" else 2e-5
    re = np.abs(r).reshape(K, nb).max(axis=1) / scale
    worst = int(np.argmax(np.abs(r)))
    diag = {"red_max": float(re[col == 0].max()), "black_max": float(re[col == 1].max()),
            "worst_elem": worst // nb, "worst_row": worst % nb, "worst_colour": int(col[worst // nb]),
            "z_at_worst_elem": float(np.max(np.abs(z[(worst // nb) * nb:(worst // nb + 1) * nb])))}
    assert np.max(np.abs(r)) <= tol * scale, diag
    assert diag["black_max"] <= 10 * max(diag["red_max"], tol * 1e-3), diag  # no worse than block Jacobi rows
    # the oracle's sweep agrees to the block conditioning (FP64) and the black part is not
    # block Jacobi (the sweep reaches across the colours)
    ref = O.red_black_apply(S, n, v)
    if arm == "fp64":
        assert np.max(np.abs(z - ref)) <= 1e-5 * np.max(np.abs(ref))
    bj = np.concatenate([np.linalg.solve(S[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb], v[e * nb:(e + 1) * nb])
                         for e in range(K)])
    assert np.max(np.abs(z - bj)) > 1e-3 * np.max(np.abs(bj))


@pytest.mark.parametrize("arm", ["fp64", "mixed"])
def test_red_black_solve_matches_oracle_global_solve(arm):
    from paper_1911_02366_gb300 import sc
    n, N = 2, 3
    cfg = dict(precond=sc.SC_PC_RED_BLACK, rel_tol=1e-12, gmres_restart=60, gmres_max_iters=4000)
    if arm == "mixed":
        cfg.update(precision=sc.SC_PREC_MIXED, inner_tol=1e-4, max_refine=30)
    Q, dt, p, ctx = _system(n, N, **cfg)
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ, raise_on_not_converged=False)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st


def test_red_black_needs_fewer_gmres_iterations_than_block_jacobi():
    """4^3 elements, N = 3, dt of the CFL-13 rule (the bench's time step scale): the oracle's
    experiments give 97 iterations for block Jacobi and 50 for the red-black sweep."""
    from paper_1911_02366_gb300 import sc
    its = {}
    for name, pc in (("bj", sc.SC_PC_BLOCK_JACOBI), ("rb", sc.SC_PC_RED_BLACK)):
        Q, dt, p, ctx = _system(4, 3, cfl=13.0, precond=pc, precision=sc.SC_PREC_MIXED, rel_tol=1e-8,
                                inner_tol=1e-4, max_refine=20)
        dQ = torch.zeros(Q.size, dtype=torch.float64, device="cuda")
        st = ctx.sc_solve(dQ)
        its[name] = st["gmres_iters"]
    assert its["rb"] < 0.75 * its["bj"], its


@pytest.mark.parametrize("n,N", [(4, 2), (2, 3)])
def test_schur_corrected_apply_satisfies_the_oracle_face_schur_blocks(n, N):
    """SC_PC_RB_SCHUR: z = P v must solve the sweep's block equations with the oracle's dense S
    and the oracle's face-block Schur blocks D_b (oracle/sweep.py): S_rr z_r = v_r,
    D_b z_b = v_b - sum_{red m} S_bm z_m.  Backward error as above; D_b comes from FP32 element
    blocks, couplings and red inverses, so its entries carry kappa(S_mm) times the FP32
    rounding of the inverse."""
    import oracle.sweep as SW
    from paper_1911_02366_gb300 import sc
    Q, dt, p, ctx = _system(n, N, precond=sc.SC_PC_RB_SCHUR, precision=sc.SC_PREC_MIXED)
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    K = n ** 3
    nb = S.shape[0] // K
    D = SW.face_schur_blocks(S, n, N)
    v = np.random.default_rng(4).standard_normal(S.shape[0])
    zt = torch.zeros(S.shape[0], dtype=torch.float64, device="cuda")
    ctx.sc_precond_apply(torch.tensor(v, device="cuda"), zt)
    z = zt.cpu().numpy()
    col = O.checkerboard(n)
    t = S @ np.where(np.repeat(col == 0, nb), z, 0.0)
    r = np.empty_like(v)
    for e in range(K):
        sl = slice(e * nb, (e + 1) * nb)
        M = D[e] if col[e] == 1 else S[sl, sl]
        r[sl] = M @ z[sl] - v[sl] + (t[sl] if col[e] == 1 else 0.0)
    scale = np.max(np.sum(np.abs(S), axis=1)) * np.max(np.abs(z)) + np.max(np.abs(v))
    re = np.abs(r).reshape(K, nb).max(axis=1) / scale
    diag = {"red_max": float(re[col == 0].max()), "black_max": float(re[col == 1].max())}
    assert diag["red_max"] <= 2e-5 and diag["black_max"] <= 1e-4, diag
    # the correction is really there: against the plain sweep's black blocks the residual is large
    r0 = np.concatenate([S[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] @ z[e * nb:(e + 1) * nb] - v[e * nb:(e + 1) * nb]
                         + t[e * nb:(e + 1) * nb] for e in range(K) if col[e] == 1])
    assert np.max(np.abs(r0)) > 20 * diag["black_max"] * scale, diag
    print(f"\nSchur-corrected sweep backward error: {diag}")


def test_schur_corrected_solve_matches_oracle_global_solve():
    from paper_1911_02366_gb300 import sc
    n, N = 2, 3
    Q, dt, p, ctx = _system(n, N, precond=sc.SC_PC_RB_SCHUR, precision=sc.SC_PREC_MIXED, rel_tol=1e-12,
                            gmres_restart=60, gmres_max_iters=4000, inner_tol=1e-4, max_refine=30)
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ, raise_on_not_converged=False)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(B - A @ dQ) / np.linalg.norm(B) < 1e-11
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9, st


def test_schur_corrected_sweep_needs_fewer_iterations_than_the_plain_sweep():
    """4^3 elements, N = 3, CFL-13 time step: the oracle's experiments give 50 iterations for
    the plain sweep and 34 with the face-block Schur blocks (equal to the whole Schur block)."""
    from paper_1911_02366_gb300 import sc
    its = {}
    for name, pc in (("bj", sc.SC_PC_BLOCK_JACOBI), ("rb", sc.SC_PC_RED_BLACK), ("schur", sc.SC_PC_RB_SCHUR)):
        Q, dt, p, ctx = _system(4, 3, cfl=13.0, precond=pc, precision=sc.SC_PREC_MIXED, rel_tol=1e-8,
                                inner_tol=1e-4, max_refine=20)
        dQ = torch.zeros(Q.size, dtype=torch.float64, device="cuda")
        st = ctx.sc_solve(dQ)
        its[name] = (st["gmres_iters"], round(st["ms_gmres"], 2))
    print(f"\nGMRES iterations, ms (4^3, N = 3, CFL 13): {its}")
    assert its["schur"][0] < 0.8 * its["rb"][0] < 0.8 * its["bj"][0], its
