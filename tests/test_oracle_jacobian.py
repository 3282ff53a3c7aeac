"""Pins of the oracle Jacobian A = dR/dQ (eq. NewtonLinSys1) and its structure (Sec. 3.1)."""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I


@pytest.fixture(scope="module")
def tgv_small():
    n, N = 3, 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt)
    return p, Q, O.jacobian(p, Q)


def test_jacobian_matches_central_differences(tgv_small):
    p, Q, A = tgv_small
    rng = np.random.default_rng(1)
    for _ in range(2):
        x = rng.standard_normal(Q.shape)
        y = (A @ x.reshape(-1)).reshape(Q.shape)
        h = 1e-5
        fd = (O.residual(p, Q + h * x, Q) - O.residual(p, Q - h * x, Q)) / (2 * h)
        assert np.abs(y - fd).max() / np.abs(y).max() < 1e-8


@pytest.mark.parametrize("N", [5, 6])
def test_high_order_jacobian_matches_central_differences(N):
    # the orders of the two largest workloads: the 1-direction dual product against
    # central differences of the residual, and one element's rows of the 5-direction
    # build against that product
    n = 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt)
    x = np.random.default_rng(7).standard_normal(Q.shape)
    y = O.jvp(p, Q, x)
    h = 1e-5
    fd = (O.residual(p, Q + h * x, Q) - O.residual(p, Q - h * x, Q)) / (2 * h)
    assert np.abs(y - fd).max() / np.abs(y).max() < 1e-8
    e = 3
    ye = sum(blk @ x[c].reshape(-1) for c, blk in O.jacobian_element_rows(p, Q, e).items())
    assert np.abs(ye - y[e].reshape(-1)).max() < 1e-12 * np.abs(y).max()


def test_jvp_equals_matrix(tgv_small):
    p, Q, A = tgv_small
    x = np.random.default_rng(2).standard_normal(Q.shape)
    y = (A @ x.reshape(-1)).reshape(Q.shape)
    np.testing.assert_allclose(O.jvp(p, Q, x), y, rtol=0, atol=1e-12 * np.abs(y).max())


def test_time_term_is_the_mass_matrix(tgv_small):
    p, Q, A = tgv_small
    ps = O.Params(**{**p.__dict__, "with_time": False})
    As = O.jacobian(ps, Q)
    _, w, _ = O.gl(p.N)
    h = p.L / p.n
    W = np.einsum("i,j,k->kji", w, w, w).reshape(-1)
    Mdiag = np.repeat(np.tile((h / 2) ** 3 * W, p.K), 5) / p.dt
    D = (A - As).toarray()
    np.testing.assert_allclose(np.diag(D), Mdiag, rtol=1e-12)
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12 * Mdiag.max()
    p2 = O.Params(**{**p.__dict__, "bdf": 2})
    A2 = O.jacobian(p2, Q)
    np.testing.assert_allclose(np.diag((A2 - As).toarray()), 1.5 * Mdiag, rtol=1e-12)


def test_conservation_of_column_sums(tgv_small):
    # sum over all rows of one variable of dH/dq_r vanishes (H's rows sum to zero for
    # every state on a periodic mesh, so do their derivatives).
    p, Q, _ = tgv_small
    ps = O.Params(**{**p.__dict__, "with_time": False})
    H = O.jacobian(ps, Q)
    cs = np.zeros((5, H.shape[1]))
    Hc = H.tocoo()
    np.add.at(cs, (Hc.row % 5, Hc.col), Hc.data)
    assert np.abs(cs).max() < 1e-11 * np.abs(H.data).max()


def _classify(n, N):
    In, Bn, I_, B_ = O.boundary_interior_split(n, N)
    K = n ** 3
    nn = (N + 1) ** 3
    is_b = np.zeros(K * nn * 5, bool)
    is_b[B_.reshape(-1)] = True
    elem = np.arange(K * nn * 5) // (nn * 5)
    return is_b, elem


@pytest.mark.parametrize("viscous", [True, False])
def test_sparsity_structure(viscous):
    # Sec. 3.1 summary: off-diagonal (element-to-element) entries need j AND r on the
    # boundary (advective case) or j OR r on the boundary (diffusive case), so A_ii is
    # block diagonal.  The corner neighbours never couple (stencil of Roe + BR1).
    n, N = 3, 3
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt, viscous=viscous)
    A = O.jacobian(p, Q).tocoo()
    is_b, elem = _classify(n, N)
    off = elem[A.row] != elem[A.col]
    rb, cb = is_b[A.row[off]], is_b[A.col[off]]
    assert off.sum() > 0
    assert np.all(rb | cb)                      # never interior-interior across elements
    if not viscous:
        assert np.all(rb & cb)                  # advective: boundary-boundary only
    else:
        assert np.any(rb & ~cb) and np.any(~rb & cb)
    # element-level stencil: face and edge neighbours only
    def ec(e):
        return np.stack([e % n, (e // n) % n, e // (n * n)], -1)
    d = np.abs(ec(elem[A.row[off]]) - ec(elem[A.col[off]]))
    d = np.minimum(d, n - d)
    hops = d.sum(-1)
    assert hops.max() == (2 if viscous else 1)


def test_linear_model_jacobian_is_state_independent():
    n, N = 2, 2
    p = O.Params(n=n, N=N, model=1, adv=(0.7, -0.3, 0.2), nu=0.05, dt=0.3)
    rng = np.random.default_rng(4)
    A1 = O.jacobian(p, rng.standard_normal((n ** 3, (N + 1) ** 3, 5)))
    A2 = O.jacobian(p, rng.standard_normal((n ** 3, (N + 1) ** 3, 5)))
    assert abs(A1 - A2).max() < 1e-13 * abs(A1).max()


@pytest.mark.parametrize("n,N", [(3, 2), (3, 3), (3, 4), (2, 5), (2, 6)])
def test_own_block_couples_only_nodes_sharing_a_gl_index(n, N):
    """Own element block of the Jacobian: node a couples to node b only if they share at
    least one of the three GL indices (volume terms act along grid lines, the BR1 viscous
    terms along lines of lines).  The condensed operator stores only these node blocks,
    so every other block must be exactly zero; the pattern is also tight (each kept
    node pair carries a nonzero entry somewhere on the mesh).  On the 2^3 meshes (N = 5,
    6) an element's neighbours across opposite faces coincide but are never the element."""
    Q, dt = I.tgv_state(n, N, cfl=50.0)
    p = O.Params(n=n, N=N, dt=dt, bdf=1)
    A = O.jacobian(p, Q).tocsr()
    nn = (N + 1) ** 3
    ne = 5 * nn
    idx = np.array([(m % (N + 1), (m // (N + 1)) % (N + 1), m // (N + 1) ** 2) for m in range(nn)])
    share = (idx[:, None, :] == idx[None, :, :]).any(axis=2)
    seen = np.zeros((nn, nn), bool)
    for e in range(n ** 3):
        blk = A[e * ne:(e + 1) * ne, e * ne:(e + 1) * ne].toarray().reshape(nn, 5, nn, 5)
        nz = (blk != 0).any(axis=(1, 3))
        assert not (nz & ~share).any()
        seen |= nz
    assert (seen == share).all()


def test_lax_friedrichs_jacobian_matches_central_differences():
    # |u . n| and the larger of the two wave speeds are not differentiable where u . n = 0
    # or where the two sides tie: the Taylor-Green velocity vanishes on whole grid planes, so
    # a mean flow is added (same pressure) to keep the faces away from those kinks
    n, N = 3, 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    Q = Q.copy()
    rho = Q[..., 0]
    v = Q[..., 1:4] / rho[..., None]
    U = np.array([0.6, 0.45, 0.35])
    Q[..., 4] += 0.5 * rho * (np.sum((v + U) ** 2, axis=-1) - np.sum(v ** 2, axis=-1))
    Q[..., 1:4] += rho[..., None] * U
    p = O.Params(n=n, N=N, dt=dt, adv_flux=1)
    A = O.jacobian(p, Q)
    x = np.random.default_rng(3).standard_normal(Q.shape)
    y = (A @ x.reshape(-1)).reshape(Q.shape)
    h = 1e-5
    fd = (O.residual(p, Q + h * x, Q) - O.residual(p, Q - h * x, Q)) / (2 * h)
    assert np.abs(y - fd).max() / np.abs(y).max() < 1e-8


def test_lax_friedrichs_keeps_the_jacobian_pattern_and_the_exact_condensation():
    # the flux pair only changes values: the same face-node couplings, so the same pattern,
    # and the condensed solve still equals the global one
    n, N = 2, 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    A_roe = O.jacobian(O.Params(n=n, N=N, dt=dt), Q).tocsr()
    p = O.Params(n=n, N=N, dt=dt, adv_flux=1)
    A_lf = O.jacobian(p, Q).tocsr()
    # node-pair (5 x 5 block) pattern: the scalar lambda of Lax-Friedrichs fills entries inside
    # blocks where Roe's dissipation has zeros, but couples no new pair of nodes
    pat = lambda A: set(zip(*(i // 5 for i in A.nonzero())))
    assert pat(A_lf) == pat(A_roe)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A_lf, B)
    xc, _ = O.condensed_solve(A_lf, B, n, N, method="direct")
    assert np.linalg.norm(xc - x) <= 1e-10 * np.linalg.norm(x)
