"""Pins of the learned red-black correction oracle (oracle/learned.py)."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as LN
import sc_inputs as I


@pytest.mark.parametrize("N", [2, 3, 4])
def test_mirror_node_sits_at_the_same_point_in_the_neighbour(N):
    n = 3
    X = I.node_coordinates(n, N, 2 * np.pi)  # [K, nodes, 3]
    L = 2 * np.pi
    for e in (0, 13, 26):
        for m in LN.boundary_nodes(N):
            f = LN.node_face(N, int(m))
            nb = LN.face_neighbour(n, e, f)
            mm = LN.mirror_node(N, int(m), f)
            d = X[e, m] - X[nb, mm]
            d -= L * np.round(d / L)  # periodic images
            assert np.max(np.abs(d)) < 1e-12


@pytest.mark.parametrize("N", [2, 3, 4])
def test_node_face_is_the_lowest_index_face_containing_the_node(N):
    p = N + 1
    for m in LN.boundary_nodes(N):
        c = (m % p, (m // p) % p, m // (p * p))
        on = [f for f in range(6) if c[f // 2] == (0 if f % 2 == 0 else N)]
        assert on and LN.node_face(N, int(m)) == min(on)


def _fd_check(fun, P, key, idx, h=1e-6):
    Pp = {k: v.copy() for k, v in P.items()}
    Pm = {k: v.copy() for k, v in P.items()}
    Pp[key][idx] += h
    Pm[key][idx] -= h
    return (fun(Pp) - fun(Pm)) / (2 * h)


def test_mlp_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    P = LN.init_params(seed=5, scale_out=1.0)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.standard_normal(P[k].shape) * 0.1
    X = rng.standard_normal((7, LN.N_IN))
    T = rng.standard_normal((7, LN.N_OUT))

    def f(PP):
        y, _ = LN.forward(PP, X)
        return LN.loss(y, T)

    y, cache = LN.forward(P, X)
    g = LN.backward(P, cache, LN.loss_grad(y, T))
    for key in P:
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in P[key].shape)
            fd = _fd_check(f, P, key, idx)
            assert abs(fd - g[key][idx]) <= 1e-6 * max(1.0, abs(fd)), (key, idx, fd, g[key][idx])


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    y = rng.standard_normal((5, LN.N_OUT))
    T = rng.standard_normal((5, LN.N_OUT))
    g = LN.loss_grad(y, T)
    for _ in range(6):
        i, j = rng.integers(0, 5), rng.integers(0, LN.N_OUT)
        yp, ym = y.copy(), y.copy()
        yp[i, j] += 1e-6
        ym[i, j] -= 1e-6
        fd = (LN.loss(yp, T) - LN.loss(ym, T)) / 2e-6
        assert abs(fd - g[i, j]) < 1e-7


def test_first_adam_step_moves_each_parameter_by_lr_times_sign():
    """After one step the bias-corrected moments are g and g^2: the update is lr g/(|g|+eps)."""
    P = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    LN.adam_step(P, g, {}, lr=0.01)
    expect = np.array([1.0, -2.0, 3.0]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(P["w"], expect, rtol=0, atol=1e-15)


def _mesh_S(n, N, cfl=10.0):
    Q, dt = I.tgv_state(n, N, cfl=cfl)
    p = O.Params(n=n, N=N, dt=dt, bdf=1)
    cs = O.condensed_operator(O.jacobian(p, Q), n, N)
    return Q, dt, cs.dense_S()


def test_features_are_normalised_and_targets_vanish_for_node_diagonal_blocks():
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    nbn = nb // 5
    K = n ** 3
    F, T, sn = LN.features_and_targets(S, Q, n, N, 0.1, 1600.0, dt)
    for lo in (5, 30, 55, 80):
        assert np.allclose(np.linalg.norm(F[:, lo:lo + 25], axis=1), 1.0)
    assert np.allclose(F[:, 105:109], [0.1, 1.6, dt * 10.0 / (np.pi), 2.0])
    # nodes of a face, an edge, a corner: 1, 2 or 3 faces (N = 2: 6 face, 12 edge, 8 corner nodes)
    nf = np.round(F[:nbn, 109] * 3).astype(int)
    assert sorted(np.bincount(nf)[1:]) == [6, 8, 12]
    assert np.all(F[:, 110:113] > 0) and np.all(F[:, 113:] == 0)
    assert np.max(np.abs(T)) > 0
    # element blocks that are block diagonal over the nodes: the node blocks of the inverse
    # are the inverses of the node blocks, so every target vanishes
    Sd = S.copy()
    for e in range(K):
        for a in range(nbn):
            for b2 in range(nbn):
                if a != b2:
                    Sd[e * nb + 5 * a:e * nb + 5 * a + 5, e * nb + 5 * b2:e * nb + 5 * b2 + 5] = 0.0
    _, Td, _ = LN.features_and_targets(Sd, Q, n, N, 0.1, 1600.0, dt)
    assert np.max(np.abs(Td)) < 1e-12 * np.max(np.abs(T))


def test_target_is_the_node_block_of_the_inverse_and_assembly_reproduces_the_schur_correction():
    """The target's defining property, checked by a solve; with the exact targets the assembled
    correction is the co-located part of the node-diagonal Schur correction of the red
    neighbours, halved, which on these systems matches half the whole node-diagonal Schur
    correction (block elimination, oracle/linalg.py) to a few parts in a thousand."""
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    nbn = nb // 5
    F, T, sn = LN.features_and_targets(S, Q, n, N, 0.1, 1600.0, dt)
    e, a = 3, 5
    blk = slice(e * nb, (e + 1) * nb)
    Z = np.linalg.inv(S[e * nb + 5 * a:e * nb + 5 * a + 5, e * nb + 5 * a:e * nb + 5 * a + 5]) + \
        T[e * nbn + a].reshape(5, 5) / sn[e * nbn + a]
    E = np.zeros((nb, 5))
    E[5 * a:5 * a + 5] = np.eye(5)
    assert np.allclose(np.linalg.solve(S[blk, blk], E)[5 * a:5 * a + 5], Z, rtol=0, atol=1e-10 * np.max(np.abs(Z)))
    C = LN.assemble_correction(S, T, n, N)
    Cs = 0.5 * O.black_schur_correction(S, n)
    black = LN.black_mask(n, N)
    rel = np.linalg.norm((C - Cs)[black].reshape(-1, 25), axis=1) / np.linalg.norm(Cs[black].reshape(-1, 25), axis=1)
    assert np.median(rel) < 5e-3, np.median(rel)
    assert np.max(np.abs(C[~black])) == 0.0


def test_assembly_with_zero_outputs_uses_the_node_blocks_own_inverses():
    """y = 0: Z is the inverse of the neighbour's node block itself (closed form, a corner
    node with its three faces)."""
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nbn = len(LN.boundary_nodes(N))
    nb = 5 * nbn
    C = LN.assemble_correction(S, np.zeros((n ** 3 * nbn, 25)), n, N)
    Bn = LN.boundary_nodes(N)
    pos = {int(m): i for i, m in enumerate(Bn)}
    e, a = 1, 0  # element 1 is black; boundary position 0 is a corner node
    m = int(Bn[a])
    assert len(LN.node_faces(N, m)) == 3
    ref = np.zeros((5, 5))
    for f in LN.node_faces(N, m):
        ne = LN.face_neighbour(n, e, f)
        b = pos[LN.mirror_node(N, m, f)]
        r, c = e * nb + 5 * a, ne * nb + 5 * b
        ref -= 0.5 * S[r:r + 5, c:c + 5] @ np.linalg.solve(S[c:c + 5, c:c + 5], S[c:c + 5, r:r + 5])
    assert np.allclose(C[e * nbn + a], ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_corrected_apply_is_the_sweep_with_the_assembled_black_blocks():
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nbn = len(LN.boundary_nodes(N))
    v = np.random.default_rng(1).standard_normal(S.shape[0])
    Y = np.random.default_rng(2).standard_normal((n ** 3 * nbn, LN.N_OUT)) * 0.01
    z = LN.corrected_apply(S, Y, v, n, N)
    ref = O.red_black_apply(S, n, v, black_blocks=O.corrected_black_blocks(S, n, LN.assemble_correction(S, Y, n, N)))
    assert np.allclose(z, ref, rtol=0, atol=1e-12)
    z0 = LN.corrected_apply(S, 0 * Y, v, n, N)
    assert not np.allclose(z0, O.red_black_apply(S, n, v))  # the closed-form correction acts
