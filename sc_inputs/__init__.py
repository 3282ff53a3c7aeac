"""Seeded synthetic inputs for the condensed GL-DGSEM Newton solve.

This module is shared by both sides of every parity check (the CPU oracle and the
CUDA library) and by the benchmark.  It holds no discretisation arithmetic: it only
places sample points, evaluates a Taylor-Green-shaped primitive state at them, applies
a counter-based multiplicative perturbation and picks the time step from a CFL rule.

Workload recipe (the paper's cylinder mesh is not available, so periodic synthetic
states stand in for it):
  * domain [0, 2*pi]^3, periodic, n^3 Cartesian hexahedra of side h = 2*pi/n;
  * nodes: tensor-product Gauss-Lobatto points of order N in each element;
  * state: Taylor-Green vortex at Mach Ma (V0 = rho0 = T0 = 1);
  * perturbation: q <- q * (1 + eps * U), U in [-1, 1) from splitmix64(seed, dof index);
  * time step: dt = CFL * (h / N) / max(|v| + c) over the unperturbed nodes.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """Counter-based splitmix64 (Steele, Lea & Flood, OOPSLA 2014).

    The generator state for draw ``counter`` is ``(seed << 40) ^ counter``; one
    splitmix64 step (add the golden gamma, then the two xor-shift-multiply rounds)
    turns it into the 64-bit output.  Deterministic and order-free, so any subset of
    draws can be regenerated independently.
    """
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) << np.uint64(40)) ^ c
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, counter: np.ndarray) -> np.ndarray:
    """Doubles in [-1, 1) from the top 53 bits of splitmix64(seed, counter)."""
    z = splitmix64(seed, counter)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def lobatto_points(N: int) -> np.ndarray:
    """The N+1 Legendre-Gauss-Lobatto points on [-1, 1] (ascending).

    Interior points are the roots of P_N' (numpy's Legendre class), the ends are +-1.
    Used only to place sample points of the synthetic state.
    """
    if N < 1:
        raise ValueError("N >= 1 required")
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots() if N > 1 else np.array([])
    pts = np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])
    return 0.5 * (pts - pts[::-1])  # exact antisymmetry


def node_coordinates(n: int, N: int, L: float = 2.0 * np.pi) -> np.ndarray:
    """Physical coordinates [K, (N+1)^3, 3] of every node.

    Element e = ex + n*(ey + n*ez); node = i + (N+1)*(j + (N+1)*k) (i fastest).
    """
    xi = lobatto_points(N)
    h = L / n
    p = N + 1
    ex, ey, ez = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ex, ey, ez = (a.transpose(2, 1, 0).reshape(-1) for a in (ex, ey, ez))
    i, j, k = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    i, j, k = (a.transpose(2, 1, 0).reshape(-1) for a in (i, j, k))
    x = h * ex[:, None] + 0.5 * h * (1.0 + xi[i][None, :])
    y = h * ey[:, None] + 0.5 * h * (1.0 + xi[j][None, :])
    z = h * ez[:, None] + 0.5 * h * (1.0 + xi[k][None, :])
    return np.stack([x, y, z], axis=-1)


def taylor_green_primitive(xyz: np.ndarray, Ma: float, gamma: float = 1.4):
    """Taylor-Green-shaped primitive fields (rho, u, v, w, p) at points xyz[..., 3].

    Velocity: u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 (divergence free).
    Pressure: p = p0 + (1/16)(cos 2x + cos 2y)(cos 2z + 2), p0 = 1/(gamma Ma^2).
    The fluctuating part solves the incompressible pressure Poisson equation
    lap p = -rho0 (d_i u_j)(d_j u_i) for this velocity.  With w = 0,
    (d_i u_j)(d_j u_i) = u_x^2 + v_y^2 + 2 u_y v_x
                       = 2 cos^2 z (cos^2 x cos^2 y - sin^2 x sin^2 y)
                       = (1/2)(1 + cos 2z)(cos 2x + cos 2y).
    Writing p' = A (cos 2x + cos 2y) + B cos 2z (cos 2x + cos 2y), the Laplacian
    multiplies the two parts by -4 and -8, so A = 1/8 and B = 1/16, i.e.
    p' = (1/16)(cos 2x + cos 2y)(cos 2z + 2).
    Temperature is uniform, T = 1, so rho = gamma Ma^2 p.
    """
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p0 = 1.0 / (gamma * Ma * Ma)
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    rho = gamma * Ma * Ma * p
    return rho, u, v, w, p


def conserved_from_primitive(rho, u, v, w, p, gamma: float = 1.4) -> np.ndarray:
    """Stack [rho, rho u, rho v, rho w, rho E] with rho E = p/(gamma-1) + rho|v|^2/2."""
    rhoE = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, rhoE], axis=-1)


def perturb(q: np.ndarray, seed: int, eps: float) -> np.ndarray:
    """q <- q * (1 + eps*U) with U = uniform_pm1(seed, flat dof index)."""
    flat = q.reshape(-1)
    U = uniform_pm1(seed, np.arange(flat.size, dtype=np.uint64))
    return (flat * (1.0 + eps * U)).reshape(q.shape)


def cfl_timestep(n: int, N: int, prim, cfl: float, gamma: float = 1.4, L: float = 2.0 * np.pi) -> float:
    """dt = CFL * (h/N) / max(|v| + c), c = sqrt(gamma p / rho), on the primitive fields."""
    rho, u, v, w, p = prim
    smax = float(np.max(np.sqrt(u * u + v * v + w * w) + np.sqrt(gamma * p / rho)))
    return cfl * (L / n / N) / smax


def tgv_state(n: int, N: int, Ma: float = 0.1, seed: int = 0, eps: float = 1e-3,
              cfl: float = 50.0, gamma: float = 1.4):
    """Perturbed Taylor-Green state Q [K, (N+1)^3, 5] (float64) and its CFL time step."""
    xyz = node_coordinates(n, N)
    prim = taylor_green_primitive(xyz, Ma, gamma)
    q = conserved_from_primitive(*prim, gamma=gamma)
    dt = cfl_timestep(n, N, prim, cfl, gamma)
    return np.ascontiguousarray(perturb(q, seed, eps)), dt


def uniform_state(n: int, N: int, Ma: float = 0.1, vel=(1.0, 0.3, -0.2), gamma: float = 1.4):
    """Uniform free-stream state (rho = 1, T = 1) used by free-stream tests."""
    K, nn = n ** 3, (N + 1) ** 3
    rho = np.ones((K, nn))
    p = np.full((K, nn), 1.0 / (gamma * Ma * Ma))
    u, v, w = (np.full((K, nn), c) for c in vel)
    return np.ascontiguousarray(conserved_from_primitive(rho, u, v, w, p, gamma))


def order_draw(seed: int, K: int) -> np.ndarray:
    """Per-element polynomial orders N_e = 2 + (splitmix64(seed, e) mod 5), e = 0..K-1."""
    return (2 + (splitmix64(seed, np.arange(K, dtype=np.uint64)) % np.uint64(5))).astype(np.int32)


def node_coordinates_mixed(n: int, orders, L: float = 2.0 * np.pi) -> np.ndarray:
    """Coordinates [sum_e (N_e+1)^3, 3] of every node of a mesh whose element e has order
    orders[e], element by element (each block as node_coordinates gives it for its order)."""
    orders = np.asarray(orders)
    by_order = {int(N): node_coordinates(n, int(N), L) for N in np.unique(orders)}
    return np.concatenate([by_order[int(N)][e] for e, N in enumerate(orders)])


def tgv_state_mixed(n: int, orders, Ma: float = 0.1, seed: int = 0, eps: float = 1e-3,
                    cfl: float = 50.0, gamma: float = 1.4):
    """Perturbed Taylor-Green state on a mixed-order mesh, flat [sum_e (N_e+1)^3, 5], and
    the CFL time step taken with the largest order (the finest node spacing)."""
    xyz = node_coordinates_mixed(n, orders)
    prim = taylor_green_primitive(xyz, Ma, gamma)
    q = conserved_from_primitive(*prim, gamma=gamma)
    dt = cfl_timestep(n, int(np.max(orders)), prim, cfl, gamma)
    return np.ascontiguousarray(perturb(q, seed, eps)), dt


def uniform_state_mixed(n: int, orders, Ma: float = 0.1, vel=(1.0, 0.3, -0.2), gamma: float = 1.4):
    """Uniform free-stream state on a mixed-order mesh, flat [sum_e (N_e+1)^3, 5]."""
    tot = int(sum((int(N) + 1) ** 3 for N in orders))
    rho = np.ones(tot)
    p = np.full(tot, 1.0 / (gamma * Ma * Ma))
    u, v, w = (np.full(tot, c) for c in vel)
    return np.ascontiguousarray(conserved_from_primitive(rho, u, v, w, p, gamma))


# The five workloads, named by what they are.
WORKLOADS = {
    "tgv_4x4x4_N3_cfl50": dict(n=4, N=3, Ma=0.1, Re=1600.0, cfl=50.0, seed=0),
    "tgv_16x16x16_N4_cfl50": dict(n=16, N=4, Ma=0.1, Re=1600.0, cfl=50.0, seed=0),
    "tgv_16x16x16_N5_cfl50": dict(n=16, N=5, Ma=0.1, Re=1600.0, cfl=50.0, seed=0),
    "tgv_16x16x16_N6_cfl100": dict(n=16, N=6, Ma=0.1, Re=1600.0, cfl=100.0, seed=0),
    # orders N_e = 2 + (splitmix64(1, e) mod 5): order_draw(order_seed, n^3), tgv_state_mixed
    "tgv_12x12x12_N2to6_cfl50": dict(n=12, N=None, order_seed=1, Ma=0.1, Re=1600.0, cfl=50.0, seed=0),
}
