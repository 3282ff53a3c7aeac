"""Pins of the oracle's Schur-corrected red-black sweep (oracle/sweep.py): an exact special
case where the face-block correction is the whole Schur block, the face lists against the
element geometry, and the dense definition on a Taylor-Green system."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as LN
import oracle.sweep as SW
import sc_inputs as I


def _face_coupled_pairs(N, seed=0):
    """Element-block matrix on the 2^3 checkerboard, 5 (N+1)^3 - 5 (N-1)^3 dofs per element,
    where each red element couples to one black partner only, and only through co-located
    node pairs of the partner's -x face (random 5 x 5 blocks both ways).  The red unknowns
    then eliminate pair by pair, so the black Schur complement is block diagonal and its
    blocks are exactly the face-block correction."""
    n = 2
    K = n ** 3
    nbn = (N + 1) ** 3 - (N - 1) ** 3
    nb = 5 * nbn
    rng = np.random.default_rng(seed)
    S = np.zeros((K * nb, K * nb))
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    for e in range(K):
        S[blk(e), blk(e)] = rng.standard_normal((nb, nb)) + 4 * nb ** 0.5 * np.eye(nb)
    nodes, mirror = SW.face_node_lists(N)
    for r, b in ((0, 1), (3, 2), (5, 4), (6, 7)):
        assert LN.face_neighbour(n, b, 0) == r
        for a, am in zip(nodes[0], mirror[0]):
            S[b * nb + 5 * a:b * nb + 5 * a + 5, r * nb + 5 * am:r * nb + 5 * am + 5] = rng.standard_normal((5, 5))
            S[r * nb + 5 * am:r * nb + 5 * am + 5, b * nb + 5 * a:b * nb + 5 * a + 5] = rng.standard_normal((5, 5))
    return S, n, nb


@pytest.mark.parametrize("N", [2, 3])
def test_face_lists_follow_the_element_geometry(N):
    nodes, mirror = SW.face_node_lists(N)
    bn = LN.boundary_nodes(N)
    p = N + 1
    for f in range(6):
        assert len(nodes[f]) == p * p
        d, side = f // 2, (0 if f % 2 == 0 else N)
        for a, am in zip(nodes[f], mirror[f]):
            c = [int(bn[a]) % p, (int(bn[a]) // p) % p, int(bn[a]) // (p * p)]
            cm = [int(bn[am]) % p, (int(bn[am]) // p) % p, int(bn[am]) // (p * p)]
            assert c[d] == side and cm[d] == N - side
            assert [c[i] for i in range(3) if i != d] == [cm[i] for i in range(3) if i != d]
    # every boundary node lies on one to three faces
    counts = np.zeros(len(bn), int)
    for f in range(6):
        counts[nodes[f]] += 1
    assert counts.min() == 1 and counts.max() == 3


@pytest.mark.parametrize("N", [2, 3])
def test_face_correction_is_the_exact_schur_block_when_couplings_are_co_located(N):
    S, n, nb = _face_coupled_pairs(N)
    col = O.checkerboard(n)
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    Sinv = np.linalg.inv(S)
    D = SW.face_schur_blocks(S, n, N)
    Dfull = SW.black_schur_blocks(S, n)
    for b in np.where(col == 1)[0]:
        exact = np.linalg.inv(Sinv[blk(b), blk(b)])  # independent route: block elimination
        assert np.allclose(D[int(b)], exact, rtol=0, atol=1e-9 * np.abs(exact).max())
        assert np.allclose(Dfull[int(b)], exact, rtol=0, atol=1e-9 * np.abs(exact).max())
        assert np.abs(D[int(b)] - S[blk(b), blk(b)]).max() > 1e-3  # the correction is not empty
    # so the sweep returns the exact black unknowns
    v = np.random.default_rng(3).standard_normal(S.shape[0])
    x = np.linalg.solve(S, v)
    z = O.red_black_apply(S, n, v, black_blocks=D)
    for b in np.where(col == 1)[0]:
        assert np.allclose(z[blk(b)], x[blk(b)], rtol=0, atol=1e-10 * np.abs(x).max())


@pytest.fixture(scope="module")
def tgv_4_2():
    n, N = 4, 2
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=1000)
    p = O.Params(n=n, N=N, dt=dt)
    A = O.jacobian(p, Q)
    cs = O.condensed_operator(A, n, N)
    S = cs.dense_S()
    g = cs.rhs(-O.residual(p, Q).reshape(-1))
    return S, g, n, N


def test_face_correction_matches_the_schur_block_on_a_taylor_green_system(tgv_4_2):
    """On a real system the red-black couplings also reach non-co-located nodes (through the
    elements' interiors); the face-block form leaves those out and stays within 2 %."""
    S, g, n, N = tgv_4_2
    nb = S.shape[0] // n ** 3
    D = SW.face_schur_blocks(S, n, N)
    Dfull = SW.black_schur_blocks(S, n)
    for b, Db in D.items():
        Sbb = S[b * nb:(b + 1) * nb, b * nb:(b + 1) * nb]
        corr = Dfull[b] - Sbb
        assert np.linalg.norm(corr) > 1e-3 * np.linalg.norm(Sbb)
        assert np.linalg.norm(Db - Dfull[b]) < 2e-2 * np.linalg.norm(corr)


def test_face_correction_cuts_the_sweeps_gmres_iterations(tgv_4_2):
    S, g, n, N = tgv_4_2
    its = {}
    for name, D in (("plain", None), ("face", SW.face_schur_blocks(S, n, N)), ("full", SW.black_schur_blocks(S, n))):
        x, info = O.gmres(lambda v: S @ v, g, precond=lambda v, D=D: O.red_black_apply(S, n, v, black_blocks=D),
                          restart=30, tol=1e-8, maxiter=2000)
        assert np.linalg.norm(S @ x - g) <= 1.01e-8 * np.linalg.norm(g)
        its[name] = info["iters"]
    assert its["face"] < its["plain"], its
    assert its["face"] <= its["full"] + 1, its
