"""Pins of the learned block-Jacobi correction oracle (oracle/learned.py)."""
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


def test_patch_inverse_block_equals_schur_complement_inverse():
    """[S_patch^-1]_ee = (S_ee - S_en S_nn^-1 S_ne)^-1 (block elimination)."""
    rng = np.random.default_rng(9)
    m = 12
    A = rng.standard_normal((2 * m, 2 * m)) + 6 * np.eye(2 * m)
    Pinv = np.linalg.inv(A)
    See, Sen, Sne, Snn = A[:m, :m], A[:m, m:], A[m:, :m], A[m:, m:]
    T = See - Sen @ np.linalg.solve(Snn, Sne)
    assert np.allclose(Pinv[:m, :m], np.linalg.inv(T), atol=1e-12)


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
    assert np.allclose(np.linalg.norm(F[:, 5:30], axis=1), 1.0)
    assert np.allclose(np.linalg.norm(F[:, 30:55], axis=1), 1.0)
    assert np.allclose(F[:, 55:59], [0.1, 1.6, dt * 10.0 / (np.pi), 2.0])
    assert np.all(F[:, 59:] == 0)
    assert np.max(np.abs(T)) > 0


def test_corrected_apply_without_correction_is_block_jacobi():
    n, N = 2, 2
    Q, dt, S = _mesh_S(n, N)
    nb = 5 * len(LN.boundary_nodes(N))
    K = n ** 3
    v = np.random.default_rng(1).standard_normal(S.shape[0])
    y = np.zeros((K * nb // 5, LN.N_OUT))
    z = LN.corrected_apply(S, y, np.ones(K * nb // 5), v, K, nb)
    for e in range(K):
        sl = slice(e * nb, (e + 1) * nb)
        assert np.allclose(S[sl, sl] @ z[sl], v[sl])
