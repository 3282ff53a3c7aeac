"""Pins of the oracle's symmetric interior-penalty viscous flux (the paper's experiment,
Sec. 4; compact fluxes, Sec. 2.1).

The flux is read inside the paper's mixed form: the volume term keeps the lifted gradient
with qhat = {{q}}, and the face flux takes the elements' own gradients and the penalty
sigma [[q]], sigma = C_IP (N+1)^2 nu_ref / h.  For linear diffusion the residual is then
the SIPG bilinear form a(q, phi_j) under Gauss-Lobatto quadrature; the pins below check it
through facts that hold for that form and not for BR1 (or for a slip in either).
"""
import numpy as np
import pytest

import oracle as O
import sc_inputs as I

NU = 0.3


def _diffusion(n, N, **kw):
    return O.Params(n=n, N=N, model=1, adv=(0.0, 0.0, 0.0), nu=NU, with_time=False, visc_flux=1, **kw)


def _continuous_state(n, N):
    """A smooth periodic field sampled at the nodes: co-located face nodes of neighbours
    carry the same value, so every jump [[q]] vanishes."""
    xyz = I.node_coordinates(n, N)
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    u = 0.2 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -0.2 * np.cos(x) * np.sin(y) * np.cos(z)
    w = 0.05 * np.sin(z + 0.3)
    rho = 1.0 + 0.1 * np.cos(x + 2 * y)
    p = (1.0 + 0.2 * np.sin(y) * np.sin(z)) / (1.4 * 0.1 ** 2)
    return np.ascontiguousarray(I.conserved_from_primitive(rho, u, v, w, p))


@pytest.mark.parametrize("n,N", [(2, 2), (3, 3), (2, 4)])
def test_continuous_states_give_the_br1_residual(n, N):
    # with [[q]] = 0 the penalty and the lifting corrections vanish, so the local and the
    # lifted face gradients coincide: the residuals agree to rounding (Navier-Stokes,
    # Sutherland, time term) while a perturbed state separates them
    Q = _continuous_state(n, N)
    Qs = Q * 0.999
    br1 = O.Params(n=n, N=N, dt=0.1, Re=50.0)
    ip = O.Params(**{**br1.__dict__, "visc_flux": 1})
    R1, R2 = O.residual(br1, Q, Qs), O.residual(ip, Q, Qs)
    assert np.abs(R1 - R2).max() <= 1e-12 * np.abs(R1).max()
    Qp, _ = I.tgv_state(n, N, eps=1e-2)
    assert np.abs(O.residual(br1, Qp) - O.residual(ip, Qp)).max() > 1e-6 * np.abs(O.residual(br1, Qp)).max()


@pytest.mark.parametrize("n,N,C", [(2, 2, 1.0), (3, 3, 2.5)])
def test_penalty_energy_of_a_piecewise_constant_state(n, N, C):
    # q constant in each element: grad q = 0 inside, so q^T R = sum over faces of
    # sigma [[q]]^2 integrated over the face, = 4 sigma (h/2)^2 sum_F sum_k (q+ - q-)^2
    # (the face weights sum to 4).  BR1 gives the lifted-gradient energy instead.
    p = _diffusion(n, N, ip_penalty=C)
    K, nn = n ** 3, (N + 1) ** 3
    c = np.random.default_rng(5).standard_normal((K, 5))
    Q = np.ascontiguousarray(np.repeat(c[:, None, :], nn, axis=1))
    R = O.residual(p, Q)
    h = p.L / n
    sigma = C * (N + 1) ** 2 * NU / h
    jumps = 0.0
    for e in range(K):
        ex, ey, ez = e % n, (e // n) % n, e // (n * n)
        for nb in (((ex + 1) % n) + n * (ey + n * ez), ex + n * (((ey + 1) % n) + n * ez),
                   ex + n * (ey + n * ((ez + 1) % n))):
            jumps += np.sum((c[e] - c[nb]) ** 2)
    expected = 4.0 * sigma * (h / 2) ** 2 * jumps
    assert abs(np.sum(Q * R) - expected) <= 1e-11 * expected
    br1 = O.Params(**{**p.__dict__, "visc_flux": 0})
    assert abs(np.sum(Q * O.residual(br1, Q)) - expected) > 1e-3 * expected


@pytest.mark.parametrize("n,N", [(2, 2), (2, 3), (3, 2)])
def test_linear_diffusion_operator_is_symmetric_positive_semidefinite(n, N):
    # a(q, v) of SIPG is symmetric; with C_IP = 1 it is also coercive on this mesh: the
    # only null vectors are the five constants.  A dropped half in the face average, a
    # one-sided local gradient or a wrong penalty sign breaks one of the two.
    A = O.jacobian(_diffusion(n, N), np.zeros((n ** 3, (N + 1) ** 3, 5))).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    # the five variables decouple: one scalar operator
    As = A[0::5, 0::5]
    ev = np.linalg.eigvalsh(0.5 * (As + As.T))
    scale = ev.max()
    assert abs(ev[0]) <= 1e-11 * scale and ev[1] > 1e-6 * scale
    flipped = O.jacobian(_diffusion(n, N, ip_penalty=-1.0), np.zeros((n ** 3, (N + 1) ** 3, 5))).toarray()
    assert np.linalg.eigvalsh(0.5 * (flipped + flipped.T)[0::5, 0::5])[0] < -1e-6 * scale


def test_sipg_converges_like_the_diffusion_operator():
    # H / (J w) of a smooth field tends to -nu lap f = 2 nu f, spectrally in the order
    def st(x):
        return np.repeat((np.sin(x[..., 0]) * np.cos(x[..., 1]))[..., None], 5, -1)

    errs = []
    n = 2
    for N in (3, 5, 7, 9):
        _, w, _ = O.gl(N)
        W = np.einsum("i,j,k->kji", w, w, w).reshape(-1)
        p = _diffusion(n, N)
        Q = np.ascontiguousarray(st(I.node_coordinates(n, N)))
        H = O.residual(p, Q) / (((p.L / n) / 2) ** 3 * W)[None, :, None]
        errs.append(np.abs(H - 2 * NU * Q).max() / np.abs(2 * NU * Q).max())
    assert errs[-1] < 1e-4 and all(errs[i + 1] < 0.25 * errs[i] for i in range(3)), errs


@pytest.mark.parametrize("adv_flux", [0, 1])
def test_free_stream_and_conservation(adv_flux):
    n, N = 2, 3
    p = O.Params(n=n, N=N, with_time=False, visc_flux=1, adv_flux=adv_flux)
    U = I.uniform_state(n, N)
    R = O.residual(p, U)
    assert np.abs(R).max() < 1e-10 * np.abs(U).max()
    Q, _ = I.tgv_state(n, N, eps=1e-2)
    R = O.residual(p, Q)
    assert np.abs(R.sum(axis=(0, 1))).max() < 1e-10 * np.abs(R).max()


def test_jacobian_matches_central_differences():
    # the paper's flux pair; a mean flow (same pressure) keeps every face away from the
    # kinks of the Lax-Friedrichs speed (u . n = 0, or the two sides tying)
    n, N = 3, 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt, Re=50.0, visc_flux=1, adv_flux=1)
    Q = Q.copy()
    rho = Q[..., 0]
    v = Q[..., 1:4] / rho[..., None]
    U = np.array([0.6, 0.45, 0.35])
    Q[..., 4] += 0.5 * rho * (np.sum((v + U) ** 2, axis=-1) - np.sum(v ** 2, axis=-1))
    Q[..., 1:4] += rho[..., None] * U
    A = O.jacobian(p, Q)
    x = np.random.default_rng(9).standard_normal(Q.shape)
    y = (A @ x.reshape(-1)).reshape(Q.shape)
    h = 1e-5
    fd = (O.residual(p, Q + h * x, Q) - O.residual(p, Q - h * x, Q)) / (2 * h)
    assert np.abs(y - fd).max() / np.abs(y).max() < 1e-8
    np.testing.assert_allclose(O.jvp(p, Q, x), y, rtol=0, atol=1e-12 * np.abs(y).max())


def test_compact_stencil_and_exact_condensation():
    # the compact flux couples an element to its six face neighbours only (BR1 adds the
    # edge neighbours); A_ii stays block diagonal, so the condensed solve is exact
    n, N = 3, 2
    Q, dt = I.tgv_state(n, N, eps=1e-2)
    p = O.Params(n=n, N=N, dt=dt, Re=50.0, visc_flux=1)
    A = O.jacobian(p, Q).tocoo()
    elem = np.arange(p.ndof) // (p.nn * 5)

    def hops(A):
        off = elem[A.row] != elem[A.col]
        ec = lambda e: np.stack([e % n, (e // n) % n, e // (n * n)], -1)
        d = np.abs(ec(elem[A.row[off]]) - ec(elem[A.col[off]]))
        return np.minimum(d, n - d).sum(-1)

    assert hops(A).max() == 1
    assert hops(O.jacobian(O.Params(n=n, N=N, dt=dt, Re=50.0), Q).tocoo()).max() == 2
    A = A.tocsr()
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    xc, _ = O.condensed_solve(A, B, n, N, method="direct")
    assert np.linalg.norm(xc - x) <= 1e-10 * np.linalg.norm(x)


def test_mixed_order_meshes_reject_the_interior_penalty():
    p = O.Params(n=2, N=2, visc_flux=1)
    orders = np.full(8, 2, np.int32)
    Q, _ = I.tgv_state_mixed(2, orders)
    with pytest.raises(ValueError):
        O.residual_mixed(p, orders, Q)
