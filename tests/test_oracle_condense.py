"""Pins of the oracle's static condensation (Sec. 2.2, Sec. 3.2) and GMRES."""
import json
import os

import numpy as np
import pytest

import oracle as O
import sc_inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7])
def test_condensed_size_ratio_table(N):
    # Table tab:ratio / eq. ratio: counted boundary fraction of a periodic 3D mesh.
    tab = json.load(open(os.path.join(GOLD, "condensed_ratio.json")))["by_dimension"]
    In, Bn, _, _ = O.boundary_interior_split(2, N)
    counted = len(Bn) / (len(In) + len(Bn))
    assert counted == pytest.approx(eval(tab["3"], {"N": N}), rel=1e-15)
    for d in ("1", "2", "3"):
        assert O.ratio_formula(N, int(d)) == pytest.approx(eval(tab[d], {"N": N}), rel=1e-15)


@pytest.mark.parametrize("n,N", [(2, 3), (3, 2), (1, 3), (1, 5), (1, 6)])
def test_condensed_equals_global(n, N):
    # Block Gauss elimination is exact algebra (eqs. StaticCondBlock, SC_step1/2).
    Q, dt = I.tgv_state(n, N, cfl=10.0)
    p = O.Params(n=n, N=N, dt=dt)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    xg = O.global_solve(A, B)
    xc, info = O.condensed_solve(A, B, n, N, method="direct")
    assert info["aii_offblock_nnz"] == 0
    assert np.linalg.norm(xc - xg) / np.linalg.norm(xg) < 1e-9
    assert np.linalg.norm(B - A @ xc) / np.linalg.norm(B) < 1e-11


def test_condensed_gmres_matches_direct_and_is_monotone():
    n, N = 2, 3
    Q, dt = I.tgv_state(n, N, cfl=10.0)
    p = O.Params(n=n, N=N, dt=dt)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    cs = O.condensed_operator(A, n, N)
    g = cs.rhs(B)
    xd = np.linalg.solve(cs.dense_S(), g)
    xb, info = O.gmres(cs.matvec, g, precond=cs.block_jacobi(), restart=30, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(xb - xd) / np.linalg.norm(xd) < 1e-9
    h = np.array(info["history"])
    # within each restart cycle the Arnoldi residual never increases
    for c in range(0, len(h) - 1, 30):
        seg = h[c + 1:c + 31]
        assert np.all(np.diff(seg) <= 1e-12 * h[0])


def test_schur_own_block_is_the_whole_schur_on_one_element():
    # With a single periodic element every coupling is the element's own, so the
    # block-Jacobi block S_ee equals the full condensed matrix.
    n, N = 1, 3
    Q, dt = I.tgv_state(n, N)
    p = O.Params(n=n, N=N, dt=dt)
    cs = O.condensed_operator(O.jacobian(p, Q), n, N)
    S = cs.dense_S()
    np.testing.assert_allclose(cs.own_block_S(0), S, rtol=0, atol=1e-12 * np.abs(S).max())


def test_dense_global_solve_equals_sparse_global_solve():
    """The dense-LU form of x = A^-1 B agrees with the sparse-LU one (both direct)."""
    import sc_inputs as I
    n, N = 2, 2
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=0)
    p = O.Params(n=n, N=N, dt=dt)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x1, x2 = O.global_solve(A, B), O.global_solve_dense(A, B)
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
