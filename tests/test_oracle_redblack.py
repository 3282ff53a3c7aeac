"""Pins of the oracle's red-black block sweep and of the black-block Schur correction
(oracle/linalg.py): exact special cases of synthetic block systems."""
import numpy as np

import oracle as O


def _paired_system(n=2, nb=10, seed=0, couple=True):
    """Element-block matrix on the n^3 checkerboard where each red element couples to one
    black partner only (0-1, 3-2, 5-4, 6-7 for n = 2): the system splits into 2 x 2 element
    pairs, so the Schur complement of the red blocks is block diagonal over the blacks."""
    K = n ** 3
    rng = np.random.default_rng(seed)
    S = np.zeros((K * nb, K * nb))
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    for e in range(K):
        S[blk(e), blk(e)] = rng.standard_normal((nb, nb)) + 4 * nb ** 0.5 * np.eye(nb)
    col = O.checkerboard(n)
    assert list(col) == [0, 1, 1, 0, 1, 0, 0, 1]
    if couple:
        for r, b in ((0, 1), (3, 2), (5, 4), (6, 7)):
            S[blk(r), blk(b)] = rng.standard_normal((nb, nb))
            S[blk(b), blk(r)] = rng.standard_normal((nb, nb))
    return S, K, nb


def test_checkerboard_gives_face_neighbours_the_other_colour():
    n = 4
    col = O.checkerboard(n)
    for e in range(n ** 3):
        c = [e % n, (e // n) % n, e // (n * n)]
        for d in range(3):
            for s in (-1, 1):
                m = list(c)
                m[d] = (m[d] + s) % n
                assert col[m[0] + n * (m[1] + n * m[2])] != col[e]


def test_sweep_without_couplings_is_block_jacobi():
    S, K, nb = _paired_system(couple=False)
    v = np.random.default_rng(1).standard_normal(S.shape[0])
    z = O.red_black_apply(S, 2, v)
    assert np.allclose(z, np.linalg.solve(S, v), rtol=0, atol=1e-12)


def test_sweep_with_the_exact_schur_blocks_gives_the_exact_black_unknowns():
    """Block elimination of the red unknowns: x_B = (S_BB - S_BR S_RR^-1 S_RB)^-1
    (v_B - S_BR S_RR^-1 v_R).  With D_b the exact Schur block the sweep's black part is x_B;
    its red part is S_rr^-1 v_r (not x_r)."""
    S, K, nb = _paired_system()
    n = 2
    v = np.random.default_rng(2).standard_normal(S.shape[0])
    x = np.linalg.solve(S, v)
    col = O.checkerboard(n)
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    Sinv = np.linalg.inv(S)
    # independent route to the Schur blocks: inverse of the black-black block of S^-1
    D = {int(b): np.linalg.inv(Sinv[blk(b), blk(b)]) for b in np.where(col == 1)[0]}
    z = O.red_black_apply(S, n, v, black_blocks=D)
    for e in range(K):
        if col[e] == 1:
            assert np.allclose(z[blk(e)], x[blk(e)], rtol=0, atol=1e-10)
        else:
            assert np.allclose(z[blk(e)], np.linalg.solve(S[blk(e), blk(e)], v[blk(e)]), rtol=0, atol=1e-12)


def test_black_schur_correction_is_the_node_diagonal_of_the_schur_block():
    S, K, nb = _paired_system()
    n = 2
    col = O.checkerboard(n)
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    Sinv = np.linalg.inv(S)
    C = O.black_schur_correction(S, n)
    nbn = nb // 5
    for e in range(K):
        full = np.linalg.inv(Sinv[blk(e), blk(e)]) - S[blk(e), blk(e)] if col[e] == 1 else np.zeros((nb, nb))
        for a in range(nbn):
            assert np.allclose(C[e * nbn + a], full[5 * a:5 * a + 5, 5 * a:5 * a + 5], rtol=0, atol=1e-10)
    # and the corrected blocks put exactly those node blocks on the diagonal
    D = O.corrected_black_blocks(S, n, C)
    for b, Db in D.items():
        diff = Db - S[blk(b), blk(b)]
        for a in range(nbn):
            assert np.allclose(diff[5 * a:5 * a + 5, 5 * a:5 * a + 5], C[b * nbn + a])
        mask = np.ones((nb, nb), bool)
        for a in range(nbn):
            mask[5 * a:5 * a + 5, 5 * a:5 * a + 5] = False
        assert not np.any(diff[mask])
