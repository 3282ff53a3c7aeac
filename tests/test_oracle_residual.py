"""Pins of the oracle's weak-form residual (eq. DGSEMsystem) against exact results.

Manufactured fields on the periodic box: the discrete operator H divided by the
diagonal mass J_j w_j must converge spectrally to the divergence of the exact flux,
computed here from closed forms (or sympy derivatives of the App. B flux definitions).
"""
import numpy as np
import pytest
import sympy

import oracle as O
import sc_inputs as I

GAMMA, PR, MA, RE = 1.4, 0.72, 0.1, 1600.0
TS = 110.4 / 288.15


def mass(n, N):
    _, w, _ = O.gl(N)
    h = 2 * np.pi / n
    W = np.einsum("i,j,k->kji", w, w, w).reshape(-1)
    return (h / 2) ** 3 * np.tile(W, (n ** 3, 1))[..., None]


def spatial(p, Q):
    ps = O.Params(**{**p.__dict__, "with_time": False})
    return O.residual(ps, Q) / mass(p.n, p.N)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("vel", [(1.0, 0.3, -0.2), (0.0, 0.0, 0.0)])
def test_free_stream_preservation(N, vel):
    n = 3
    Q = I.uniform_state(n, N, vel=vel)
    for visc in (True, False):
        p = O.Params(n=n, N=N, viscous=visc, with_time=False)
        R = O.residual(p, Q)
        assert np.abs(R).max() < 1e-11 * np.abs(Q).max()


@pytest.mark.parametrize("N", [3, 5, 6])
def test_discrete_conservation(N):
    # On a periodic mesh the face fluxes cancel pairwise and sum_j phi_j = 1 kills the
    # volume term, so the rows of H sum to zero for every conserved variable.
    Q, dt = I.tgv_state(3, N, eps=1e-2)
    p = O.Params(n=3, N=N, dt=dt, with_time=False)
    R = O.residual(p, Q)
    tot = R.reshape(-1, 5).sum(0)
    scale = np.abs(R).max()
    assert np.all(np.abs(tot) < 1e-12 * scale * R.shape[0] ** 0.5)


def _errors(make_state, exact_div, Ns, n=2, **kw):
    errs = []
    for N in Ns:
        xyz = I.node_coordinates(n, N)
        Q = make_state(xyz)
        p = O.Params(n=n, N=N, **kw)
        H = spatial(p, Q)
        ref = exact_div(xyz)
        errs.append(np.abs(H - ref).max() / max(np.abs(ref).max(), 1e-300))
    return errs


def test_linear_advection_spectral_convergence():
    a = (1.0, 0.5, -0.25)

    def st(x):
        f = np.sin(x[..., 0]) + np.cos(2 * x[..., 1]) * np.sin(x[..., 2])
        return np.repeat(f[..., None], 5, -1)

    def div(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        f = a[0] * np.cos(X) - 2 * a[1] * np.sin(2 * Y) * np.sin(Z) + a[2] * np.cos(2 * Y) * np.cos(Z)
        return np.repeat(f[..., None], 5, -1)

    errs = _errors(st, div, [3, 5, 7, 9], model=1, adv=a, viscous=False)
    assert errs[-1] < 1e-3 and all(errs[i + 1] < 0.2 * errs[i] for i in range(3)), errs


def test_diffusion_spectral_convergence():
    nu = 0.3

    def st(x):
        f = np.sin(x[..., 0]) * np.cos(x[..., 1])
        return np.repeat(f[..., None], 5, -1)

    def div(x):  # div(-nu grad f) = -nu lap f = 2 nu f
        return 2 * nu * st(x)

    errs = _errors(st, div, [3, 5, 7, 9], model=1, adv=(0.0, 0.0, 0.0), nu=nu)
    assert errs[-1] < 1e-4 and all(errs[i + 1] < 0.25 * errs[i] for i in range(3)), errs


def test_ns_viscous_shear_layer():
    # rho = 1, T = 1 (p = p0), u = eps sin y: the inviscid flux is divergence free and
    # div(f^nu) has (x-momentum, energy) components (-eps sin y, eps^2 cos 2y)/Re.
    eps = 0.5
    p0 = 1 / (GAMMA * MA ** 2)

    def st(x):
        u = eps * np.sin(x[..., 1]); z = np.zeros_like(u)
        return I.conserved_from_primitive(np.ones_like(u), u, z, z, np.full_like(u, p0))

    def div(x):
        y = x[..., 1]
        out = np.zeros(x.shape[:-1] + (5,))
        out[..., 1] = eps * np.sin(y) / RE
        out[..., 4] = -eps ** 2 * np.cos(2 * y) / RE
        return out

    errs = _errors(st, div, [3, 5, 7, 9])
    assert errs[-1] < 2e-4 and all(errs[i + 1] < 0.2 * errs[i] for i in range(3)), errs


def test_ns_heat_conduction_with_sutherland():
    # u = 0, p = p0, rho = 1 + eps sin x  =>  T = 1/rho varies; only the heat flux
    # survives: div(f) = -(1/Re) d/dx (kappa(T) dT/dx) in the energy equation,
    # kappa = mu(T)/((gamma-1) Pr Ma^2), mu from Sutherland's law (App. B).
    eps = 0.2
    p0 = 1 / (GAMMA * MA ** 2)
    xs = sympy.symbols("x")
    rho = 1 + eps * sympy.sin(xs)
    T = GAMMA * MA ** 2 * p0 / rho
    mu = (1 + TS) / (T + TS) * T ** sympy.Rational(3, 2)
    kappa = mu / ((GAMMA - 1) * PR * MA ** 2)
    q = -sympy.diff(kappa * sympy.diff(T, xs), xs) / RE
    qf = sympy.lambdify(xs, q, "numpy")

    def st(x):
        r = 1 + eps * np.sin(x[..., 0]); z = np.zeros_like(r)
        return I.conserved_from_primitive(r, z, z, z, np.full_like(r, p0))

    def div(x):
        out = np.zeros(x.shape[:-1] + (5,))
        out[..., 4] = qf(x[..., 0])
        return out

    errs = _errors(st, div, [3, 5, 7, 9], n=4)
    assert errs[-1] < 1e-4 and all(errs[i + 1] < 0.1 * errs[i] for i in range(3)), errs


def test_euler_smooth_state():
    # Smooth 2D state, inviscid: H/(J w) -> div f^a(q(x)) with f^a from App. B,
    # differentiated symbolically.
    X, Y = sympy.symbols("x y")
    rho = 1 + 0.1 * sympy.sin(X) * sympy.cos(Y)
    u = 0.5 + 0.2 * sympy.cos(X)
    v = 0.3 * sympy.sin(Y)
    p = 1 / (GAMMA * MA ** 2) * (1 + 0.05 * sympy.sin(X + Y))
    E = p / (GAMMA - 1) + rho * (u ** 2 + v ** 2) / 2
    fx = [rho * u, rho * u ** 2 + p, rho * u * v, 0, u * (E + p)]
    fy = [rho * v, rho * u * v, rho * v ** 2 + p, 0, v * (E + p)]
    divs = [sympy.lambdify((X, Y), sympy.diff(fx[k], X) + sympy.diff(fy[k], Y), "numpy") for k in range(5)]
    prims = [sympy.lambdify((X, Y), e, "numpy") for e in (rho, u, v, p)]

    def st(x):
        a, b = x[..., 0], x[..., 1]
        r, uu, vv, pp = (f(a, b) * np.ones_like(a) for f in prims)
        return I.conserved_from_primitive(r, uu, vv, np.zeros_like(a), pp)

    def div(x):
        a, b = x[..., 0], x[..., 1]
        return np.stack([np.asarray(f(a, b)) * np.ones_like(a) for f in divs], -1)

    errs = _errors(st, div, [3, 5, 7, 9], viscous=False)
    assert errs[-1] < 1e-4 and all(errs[i + 1] < 0.1 * errs[i] for i in range(3)), errs


@pytest.mark.parametrize("N", [2, 4])
def test_lax_friedrichs_free_stream_and_conservation(N):
    Q = I.uniform_state(3, N, vel=(1.0, 0.3, -0.2))
    R = O.residual(O.Params(n=3, N=N, with_time=False, adv_flux=1), Q)
    assert np.abs(R).max() < 1e-11 * np.abs(Q).max()
    Q, dt = I.tgv_state(3, N, eps=1e-2)
    R = O.residual(O.Params(n=3, N=N, dt=dt, with_time=False, adv_flux=1), Q)
    tot = R.reshape(-1, 5).sum(0)
    assert np.all(np.abs(tot) < 1e-12 * np.abs(R).max() * R.shape[0] ** 0.5)
    # and the residual is not Roe's
    R_roe = O.residual(O.Params(n=3, N=N, dt=dt, with_time=False), Q)
    assert np.abs(R - R_roe).max() > 1e-6 * np.abs(R).max()
