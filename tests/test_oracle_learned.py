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


def test_targets_vanish_without_coupling_and_features_are_normalised():
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    K = n ** 3
    Sblk = np.zeros_like(S)
    for e in range(K):
        sl = slice(e * nb, (e + 1) * nb)
        Sblk[sl, sl] = S[sl, sl]
    F, T, sn = LN.features_and_targets(Sblk, Q, n, N, 0.1, 1600.0, dt)
    assert np.max(np.abs(T)) < 1e-10 * np.max(sn)
    F, T, sn = LN.features_and_targets(S, Q, n, N, 0.1, 1600.0, dt)
    for lo in (5, 30, 55, 80):
        assert np.allclose(np.linalg.norm(F[:, lo:lo + 25], axis=1), 1.0)
    assert np.allclose(F[:, 105:109], [0.1, 1.6, dt * 10.0 / (np.pi), 2.0])
    # nodes of a face, an edge, a corner: 1, 2 or 3 faces (N = 2: 6 face, 12 edge, 8 corner nodes)
    nf = np.round(F[:len(LN.boundary_nodes(N)), 109] * 3).astype(int)
    assert sorted(np.bincount(nf)[1:]) == [6, 8, 12]
    assert np.all(F[:, 110:113] > 0) and np.all(F[:, 113:] == 0)
    # a node on one face only: the neighbour's coupling block at k' is the coupling back to k
    nbn = len(LN.boundary_nodes(N))
    nb = 5 * nbn
    for a, m in enumerate(LN.boundary_nodes(N)):
        if LN.node_face_count(N, int(m)) != 1:
            continue
        f = LN.node_face(N, int(m))
        ne = LN.face_neighbour(n, 0, f)
        b = list(LN.boundary_nodes(N)).index(LN.mirror_node(N, int(m), f))
        blk = S[ne * nb + 5 * b:ne * nb + 5 * b + 5, 5 * a:5 * a + 5]
        assert np.allclose(F[a, 55:80], (blk / np.linalg.norm(blk)).reshape(-1))
        break
    black = LN.black_mask(n, N)
    assert np.max(np.abs(T[~black])) == 0 and np.max(np.abs(T[black])) > 0


def test_targets_are_half_the_node_diagonal_schur_correction():
    """Black targets times ||[S_ee]_kk||_F: half the node blocks of -sum_red S_bm S_mm^-1 S_mb,
    here formed through the exact inverse of each two-element patch [[S_bb, S_bm], [S_mb, S_mm]]
    (block elimination: S_bb - S_bm S_mm^-1 S_mb = inverse of the patch inverse's bb block)."""
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    nbn = nb // 5
    F, T, sn = LN.features_and_targets(S, Q, n, N, 0.1, 1600.0, dt)
    col = O.checkerboard(n)
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    for b in np.where(col == 1)[0][:3]:
        corr = np.zeros((nb, nb))
        for m in np.where(col == 0)[0]:
            if not np.any(S[blk(b), blk(m)]):
                continue
            ids = np.r_[np.arange(b * nb, (b + 1) * nb), np.arange(m * nb, (m + 1) * nb)]
            Pinv = np.linalg.inv(S[np.ix_(ids, ids)])
            corr += np.linalg.inv(Pinv[:nb, :nb]) - S[blk(b), blk(b)]
        for a in range(nbn):
            s = b * nbn + a
            ref = 0.5 * corr[5 * a:5 * a + 5, 5 * a:5 * a + 5] / sn[s]
            assert np.allclose(T[s].reshape(5, 5), ref, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ref))))


def test_corrected_apply_without_correction_is_the_red_black_sweep():
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    K = n ** 3
    v = np.random.default_rng(1).standard_normal(S.shape[0])
    y = np.zeros((K * nb // 5, LN.N_OUT))
    z = LN.corrected_apply(S, y, np.ones(K * nb // 5), v, n)
    assert np.allclose(z, O.red_black_apply(S, n, v), rtol=0, atol=1e-12)
