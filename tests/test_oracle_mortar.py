"""Pins of the oracle on meshes of mixed polynomial order (mortar faces between orders).

Reading of the unstated case (the paper treats one order per mesh): at a face between
orders N_L != N_R both traces are interpolated to the Gauss-Lobatto nodes of order
max(N_L, N_R), qhat and fhat are formed there, and each side takes their L2 projection
onto its own face polynomials with a Gauss rule exact to degree 2 max(N_L, N_R)."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I

ORDERS_2x2x2 = np.array([2, 3, 3, 2, 3, 2, 2, 3])  # checkerboard: every face is a mortar


def test_equal_orders_through_the_mortar_reduce_to_the_conforming_face():
    # interpolation to the common order is the identity and the L2 projection of a
    # polynomial of the element's own degree returns it: residual and Jacobian-vector
    # product of the conforming oracle
    n, N = 2, 3
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    Qs = Q * (1 + 1e-3 * np.random.default_rng(1).standard_normal(Q.shape))
    Qsm1 = Q * (1 + 1e-3 * np.random.default_rng(2).standard_normal(Q.shape))
    orders = np.full(n ** 3, N)
    for bdf in (1, 2):
        p = O.Params(n=n, N=N, dt=dt, bdf=bdf)
        R = O.residual(p, Q, Qs, Qsm1).reshape(-1, 5)
        for force in (True, False):  # the mortar, and the mixed code's conforming faces
            Rm = O.residual_mixed(p, orders, Q.reshape(-1, 5), Qs.reshape(-1, 5), Qsm1.reshape(-1, 5),
                                  force_mortar=force)
            assert np.abs(Rm - R).max() < 1e-12 * np.abs(R).max()
    x = np.random.default_rng(3).standard_normal(Q.shape)
    y = O.jvp(p, Q, x).reshape(-1, 5)
    ym = O.jvp_mixed(p, orders, Q.reshape(-1, 5), x.reshape(-1, 5), force_mortar=True)
    assert np.abs(ym - y).max() < 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("orders", [ORDERS_2x2x2, np.array([2, 4, 5, 3, 6, 2, 4, 3])])
@pytest.mark.parametrize("viscous", [True, False])
def test_free_stream_is_preserved_across_mortars(orders, viscous):
    n = 2
    Q = I.uniform_state_mixed(n, orders)
    p = O.Params(n=n, N=int(orders.max()), viscous=viscous, with_time=False)
    R = O.residual_mixed(p, orders, Q)
    assert np.abs(R).max() < 1e-11 * np.abs(Q).max()


def test_discrete_conservation_across_mortars():
    # the projection keeps each face integral (constants lie in every face space), the
    # mortar fluxes are single valued with opposite signs on the two sides, and
    # sum_j phi_j = 1 removes the volume terms: the rows of H sum to zero per variable
    n = 3
    orders = I.order_draw(1, n ** 3)
    assert len(set(orders.tolist())) > 2
    Q, dt = I.tgv_state_mixed(n, orders, eps=1e-2)
    p = O.Params(n=n, N=int(orders.max()), dt=dt, with_time=False)
    R = O.residual_mixed(p, orders, Q)
    tot = R.sum(0)
    assert np.all(np.abs(tot) < 1e-12 * np.abs(R).max() * R.shape[0] ** 0.5)


def test_order_draw_is_uniform_on_2_to_6():
    o = I.order_draw(1, 1728)
    assert set(np.unique(o).tolist()) == {2, 3, 4, 5, 6}
    counts = np.bincount(o)[2:]
    assert counts.min() > 0.15 * 1728 and counts.max() < 0.25 * 1728


def test_mixed_jacobian_matches_central_differences_and_the_product():
    n = 2
    orders = ORDERS_2x2x2
    Q, dt = I.tgv_state_mixed(n, orders, eps=1e-2)
    p = O.Params(n=n, N=3, dt=dt)
    x = np.random.default_rng(5).standard_normal(Q.shape)
    y = O.jvp_mixed(p, orders, Q, x)
    h = 1e-5
    fd = (O.residual_mixed(p, orders, Q + h * x, Q) - O.residual_mixed(p, orders, Q - h * x, Q)) / (2 * h)
    assert np.abs(y - fd).max() / np.abs(y).max() < 1e-8
    A = O.jacobian_mixed(p, orders, Q)
    assert np.abs(A @ x.reshape(-1) - y.reshape(-1)).max() < 1e-12 * np.abs(y).max()


def _split_mixed(orders):
    """Interior / boundary dof lists of every element of a mixed-order mesh."""
    I_, B_, off = [], [], 0
    for N in orders:
        p = int(N) + 1
        c = np.array([(m % p, (m // p) % p, m // (p * p)) for m in range(p ** 3)])
        inner = np.all((c > 0) & (c < int(N)), axis=1)
        dof = lambda nodes: ((off + nodes[:, None]) * 5 + np.arange(5)).reshape(-1)
        I_.append(dof(np.nonzero(inner)[0]))
        B_.append(dof(np.nonzero(~inner)[0]))
        off += p ** 3
    return I_, B_


def test_interior_blocks_stay_element_diagonal_and_condensation_is_exact():
    # only face dofs cross a mortar, so A_ii is block diagonal and the condensed solve
    # (eqs. SC_step1/2 with element blocks of uneven sizes) equals the global one
    n = 2
    orders = np.array([2, 3, 4, 2, 3, 2, 2, 3])
    Q, dt = I.tgv_state_mixed(n, orders, cfl=10.0)
    p = O.Params(n=n, N=4, dt=dt)
    A = O.jacobian_mixed(p, orders, Q)
    B = -O.residual_mixed(p, orders, Q).reshape(-1)
    I_, B_ = _split_mixed(orders)
    If, Bf = np.concatenate(I_), np.concatenate(B_)
    Aii = A[np.ix_(If, If)]
    sizes = [len(i) for i in I_]
    mask = np.zeros_like(Aii, bool)
    o = 0
    for s in sizes:
        mask[o:o + s, o:o + s] = True
        o += s
    assert np.abs(Aii[~mask]).max() == 0.0
    # condensation element block by element block
    Aib, Abi, Abb = A[np.ix_(If, Bf)], A[np.ix_(Bf, If)], A[np.ix_(Bf, Bf)]
    Y = np.zeros_like(Aib)
    g = B[Bf].copy()
    yi = np.zeros(len(If))
    o = 0
    for s in sizes:
        blk = Aii[o:o + s, o:o + s]
        Y[o:o + s] = np.linalg.solve(blk, Aib[o:o + s])
        yi[o:o + s] = np.linalg.solve(blk, B[If][o:o + s])
        o += s
    S = Abb - Abi @ Y
    xb = np.linalg.solve(S, g - Abi @ yi)
    xi = yi - Y @ xb
    x = np.zeros(len(B))
    x[If], x[Bf] = xi, xb
    xg = np.linalg.solve(A, B)
    assert np.linalg.norm(x - xg) / np.linalg.norm(xg) < 1e-10
    assert np.linalg.norm(B - A @ x) / np.linalg.norm(B) < 1e-11


def _advection_l2_error(n, orders):
    """Mass-weighted L2 error of the linear-advection operator (model 1) of a smooth
    periodic field against its exact divergence."""
    a = (1.0, 0.5, -0.25)
    xyz = I.node_coordinates_mixed(n, orders)
    X, Y, Z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    Q = np.repeat((np.sin(X) + np.cos(Y) * np.sin(Z))[:, None], 5, -1)
    p = O.Params(n=n, N=int(max(orders)), model=1, adv=a, viscous=False, with_time=False)
    R = O.residual_mixed(p, orders, Q)
    h = 2 * np.pi / n
    mass = []
    for N_e in orders:
        _, w, _ = O.gl(int(N_e))
        mass.append((h / 2) ** 3 * np.einsum("i,j,k->kji", w, w, w).reshape(-1))
    m = np.concatenate(mass)
    div = a[0] * np.cos(X) - a[1] * np.sin(Y) * np.sin(Z) + a[2] * np.cos(Y) * np.cos(Z)
    err = R[:, 0] / m - div
    return np.sqrt((m * err * err).sum() / (m * div * div).sum())


def test_mixed_orders_are_as_accurate_as_the_lower_order_and_converge_spectrally():
    # checkerboards of orders N / N + 1: every face is a mortar; the operator's L2 error
    # is no larger than that of the conforming mesh of order N and falls spectrally
    n = 2
    mixed, uniform = {}, {}
    for N in (3, 4, 5, 6):
        mixed[N] = _advection_l2_error(n, np.array([N, N + 1, N + 1, N, N + 1, N, N, N + 1]))
        uniform[N] = _advection_l2_error(n, np.full(8, N))
        assert mixed[N] <= 1.05 * uniform[N], (N, mixed[N], uniform[N])
    assert mixed[5] < 0.1 * mixed[3] and mixed[6] < 0.1 * mixed[4], mixed


def test_mortar_faces_take_the_own_block_out_of_the_gl_index_pattern():
    # through interpolation and projection a face node's fluxes depend on every node of its
    # face, and through the lifted gradients on the lines through them: the own block of an
    # element with mortar faces leaves the conforming pattern (node pairs sharing a GL
    # index), which a conforming mesh of the same order keeps
    n = 2
    Q, dt = I.tgv_state_mixed(n, ORDERS_2x2x2, eps=1e-2)
    p = O.Params(n=n, N=3, dt=dt)
    A = O.jacobian_mixed(p, ORDERS_2x2x2, Q)
    N = int(ORDERS_2x2x2[0])
    q = N + 1
    c = np.array([(m % q, (m // q) % q, m // (q * q)) for m in range(q ** 3)])
    share = (c[:, None, :] == c[None, :, :]).any(axis=2)
    blk = A[:5 * q ** 3, :5 * q ** 3].reshape(q ** 3, 5, q ** 3, 5)
    assert ((blk != 0).any(axis=(1, 3)) & ~share).any()
    Qc, dtc = I.tgv_state(n, N, eps=1e-2)
    Ac = O.jacobian_mixed(O.Params(n=n, N=N, dt=dtc), np.full(8, N), Qc.reshape(-1, 5))
    bc = Ac[:5 * q ** 3, :5 * q ** 3].reshape(q ** 3, 5, q ** 3, 5)
    assert not ((bc != 0).any(axis=(1, 3)) & ~share).any()


def test_the_uneven_order_workload_mesh_preserves_free_stream_and_conserves():
    # the 12^3 mesh with orders drawn from 2..6 (seed 1) at full size
    n = 12
    orders = I.order_draw(1, n ** 3)
    Q = I.uniform_state_mixed(n, orders)
    p = O.Params(n=n, N=6, with_time=False)
    R = O.residual_mixed(p, orders, Q)
    assert np.abs(R).max() < 1e-11 * np.abs(Q).max()
    Q, dt = I.tgv_state_mixed(n, orders, eps=1e-2)
    R = O.residual_mixed(p, orders, Q)
    assert np.all(np.abs(R.sum(0)) < 1e-12 * np.abs(R).max() * R.shape[0] ** 0.5)


def test_sparse_mixed_jacobian_equals_the_dense_one_and_the_product():
    n = 2
    Q, dt = I.tgv_state_mixed(n, ORDERS_2x2x2, eps=1e-2)
    p = O.Params(n=n, N=3, dt=dt)
    assert np.abs(O.jacobian_mixed_sparse(p, ORDERS_2x2x2, Q).toarray()
                  - O.jacobian_mixed(p, ORDERS_2x2x2, Q)).max() == 0.0
    n = 3
    orders = np.array([2, 3, 4, 3, 2, 4, 2, 3, 4] * 3)
    Q, dt = I.tgv_state_mixed(n, orders, eps=1e-2)
    p = O.Params(n=n, N=4, dt=dt)
    A = O.jacobian_mixed_sparse(p, orders, Q)
    x = np.random.default_rng(9).standard_normal(Q.shape)
    y = O.jvp_mixed(p, orders, Q, x).reshape(-1)
    assert np.abs(A @ x.reshape(-1) - y).max() < 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("method", ["direct", "gmres"])
def test_mixed_condensed_solve_equals_the_global_solve(method):
    # condensation with element blocks of uneven sizes on a 3^3 mesh of orders 2..4
    n = 3
    orders = np.array([2, 3, 4, 3, 2, 4, 2, 3, 4] * 3)
    Q, dt = I.tgv_state_mixed(n, orders, cfl=10.0)
    p = O.Params(n=n, N=4, dt=dt)
    A = O.jacobian_mixed_sparse(p, orders, Q)
    B = -O.residual_mixed(p, orders, Q).reshape(-1)
    xg = np.linalg.solve(A.toarray(), B)  # dense: sparse LU fills in heavily here
    xc, info = O.condensed_solve_mixed(A, B, orders, method=method, tol=1e-12, restart=60, maxiter=3000)
    assert info["aii_offblock_nnz"] == 0
    assert np.linalg.norm(xc - xg) / np.linalg.norm(xg) < 1e-9
    assert np.linalg.norm(B - A @ xc) / np.linalg.norm(B) < 1e-11


def test_mixed_element_rows_equal_the_sparse_jacobian():
    n = 3
    orders = np.array([2, 3, 4, 3, 2, 4, 2, 3, 4] * 3)
    Q, dt = I.tgv_state_mixed(n, orders, eps=1e-2)
    p = O.Params(n=n, N=4, dt=dt)
    A = O.jacobian_mixed_sparse(p, orders, Q).tocsr()
    off = np.concatenate([[0], np.cumsum([5 * (int(N) + 1) ** 3 for N in orders])])
    for e in (0, 13, 26):
        rows = O.jacobian_mixed_element_rows(p, orders, Q, e)
        assert len(rows) == 27
        for c, blk in rows.items():
            ref = A[off[e]:off[e + 1], off[c]:off[c + 1]].toarray()
            assert np.abs(blk - ref).max() <= 1e-14 * np.abs(A.data).max(), (e, c)


def test_lax_friedrichs_across_mortars_keeps_free_stream_and_conservation():
    # the paper's advective flux on mixed-order meshes: the same two invariants as Roe's
    n = 3
    orders = I.order_draw(1, n ** 3)
    U = I.uniform_state_mixed(n, orders)
    p = O.Params(n=n, N=int(orders.max()), with_time=False, adv_flux=1)
    assert np.abs(O.residual_mixed(p, orders, U)).max() < 1e-11 * np.abs(U).max()
    Q, _ = I.tgv_state_mixed(n, orders, eps=1e-2)
    R = O.residual_mixed(p, orders, Q)
    assert np.abs(R.sum(axis=0)).max() < 1e-10 * np.abs(R).max()
    roe = O.residual_mixed(O.Params(**{**p.__dict__, "adv_flux": 0}), orders, Q)
    assert np.abs(R - roe).max() > 1e-8 * np.abs(R).max()
