"""FP64 CPU oracle for the statically condensed GL-DGSEM Newton solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The product
library never links, imports or calls it, and it imports nothing from the product
package: the only module both sides share is ``sc_inputs`` (seeded inputs).

Layers:
  * ``oracle/sc_oracle.cpp`` (compiled to ``oracle/_build/liboracle.so``): Gauss-Lobatto
    basis, weak-form residual (Sec. 2.1, eq. DGSEMsystem), dual-number Jacobian
    (eq. NewtonLinSys1) and Jacobian-vector products.
  * ``oracle/linalg.py``: the static condensation of Sec. 2.2 / 3.2 (eqs. StaticCondBlock,
    SC_step1, SC_step2) and a right-preconditioned restarted GMRES, on numpy/scipy.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed forms,
invariants and brute-force solves.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/sc_oracle.cpp with g++ (-O3 -fopenmp) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    src = os.path.join(_HERE, "sc_oracle.cpp")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("N", ctypes.c_int), ("L", ctypes.c_double), ("dt", ctypes.c_double),
        ("bdf", ctypes.c_int), ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Re", ctypes.c_double), ("Ma", ctypes.c_double), ("Ts", ctypes.c_double),
        ("sutherland", ctypes.c_int), ("model", ctypes.c_int), ("viscous", ctypes.c_int),
        ("adv", ctypes.c_double * 3), ("nu", ctypes.c_double), ("roe_delta", ctypes.c_double),
        ("with_time", ctypes.c_int), ("adv_flux", ctypes.c_int),
        ("visc_flux", ctypes.c_int), ("ip_penalty", ctypes.c_double),
    ]


@dataclass
class Params:
    """Problem definition: mesh, order, physics and time step."""
    n: int
    N: int
    dt: float = 1.0
    L: float = 2.0 * np.pi
    bdf: int = 1
    gamma: float = 1.4
    Pr: float = 0.72
    Re: float = 1600.0
    Ma: float = 0.1
    Ts: float = 110.4 / 288.15
    sutherland: bool = True
    model: int = 0          # 0 Navier-Stokes, 1 linear advection-diffusion (5 copies)
    viscous: bool = True
    adv: tuple = (1.0, 0.0, 0.0)
    nu: float = 0.0
    roe_delta: float = 0.05
    with_time: bool = True
    adv_flux: int = 0       # 0 Roe (entropy fix), 1 local Lax-Friedrichs
    visc_flux: int = 0      # 0 BR1, 1 symmetric interior penalty (compact)
    ip_penalty: float = 1.0  # C_IP in sigma = C_IP (N+1)^2 nu_ref / h

    @property
    def K(self) -> int:
        return self.n ** 3

    @property
    def nn(self) -> int:
        return (self.N + 1) ** 3

    @property
    def ndof(self) -> int:
        return self.K * self.nn * 5

    def c(self) -> _Params:
        p = _Params()
        p.n, p.N, p.L, p.dt, p.bdf = self.n, self.N, self.L, self.dt, self.bdf
        p.gamma, p.Pr, p.Re, p.Ma, p.Ts = self.gamma, self.Pr, self.Re, self.Ma, self.Ts
        p.sutherland, p.model, p.viscous = int(self.sutherland), self.model, int(self.viscous)
        p.adv = (ctypes.c_double * 3)(*self.adv)
        p.nu, p.roe_delta, p.with_time = self.nu, self.roe_delta, int(self.with_time)
        p.adv_flux = int(self.adv_flux)
        p.visc_flux, p.ip_penalty = int(self.visc_flux), float(self.ip_penalty)
        return p


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_gl.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_lagrange.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.or_lifting.argtypes = [P, dp, dp]
        L.or_residual.argtypes = [P, dp, dp, dp, dp]
        L.or_jvp.argtypes = [P, dp, dp, dp]
        L.or_jacobian_coo.argtypes = [P, dp, ctypes.c_long, ip, ip, dp]
        L.or_jacobian_coo.restype = ctypes.c_long
        L.or_jacobian_elem_rows.argtypes = [P, dp, ctypes.c_int, ip, dp]
        L.or_num_flux.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.or_phys_flux.argtypes = [P, dp, dp, ctypes.c_int, dp, dp]
        L.or_residual_mixed.argtypes = [P, ip, ctypes.c_int, dp, dp, dp, dp]
        L.or_jvp_mixed.argtypes = [P, ip, ctypes.c_int, dp, dp, dp]
        L.or_jacobian_mixed.argtypes = [P, ip, ctypes.c_int, dp, dp]
        L.or_jacobian_mixed_coo.argtypes = [P, ip, ctypes.c_int, dp, ctypes.c_long, ip, ip, dp]
        L.or_jacobian_mixed_coo.restype = ctypes.c_long
        L.or_jacobian_mixed_elem_rows.argtypes = [P, ip, ctypes.c_int, dp, ctypes.c_int, ip, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().or_num_threads())


def gl(N: int):
    """Gauss-Lobatto nodes, weights and derivative matrix D[a, i] = l_i'(xi_a)."""
    xi = np.zeros(N + 1); w = np.zeros(N + 1); D = np.zeros((N + 1, N + 1))
    if lib().or_gl(N, _dp(xi), _dp(w), _dp(D)) != 0:
        raise ValueError("bad N")
    return xi, w, D


def lagrange(N: int, i: int, x: float):
    v = ctypes.c_double(); d = ctypes.c_double()
    lib().or_lagrange(N, i, x, ctypes.byref(v), ctypes.byref(d))
    return v.value, d.value


def lifting(p: Params, Q: np.ndarray) -> np.ndarray:
    Q = _f64(Q)
    g = np.zeros((p.K, p.nn, 3, 5))
    lib().or_lifting(ctypes.byref(p.c()), _dp(Q), _dp(g))
    return g


def residual(p: Params, Q: np.ndarray, Qs: np.ndarray | None = None, Qsm1: np.ndarray | None = None) -> np.ndarray:
    """R(Q) of eq. NeqtonEq, shape [K, nn, 5]."""
    Q = _f64(Q)
    Qs = Q if Qs is None else _f64(Qs)
    Qsm1 = Qs if Qsm1 is None else _f64(Qsm1)
    R = np.zeros((p.K, p.nn, 5))
    lib().or_residual(ctypes.byref(p.c()), _dp(Q), _dp(Qs), _dp(Qsm1), _dp(R))
    return R


def jvp(p: Params, Q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """(dR/dQ)(Q) x, shape [K, nn, 5]."""
    Q = _f64(Q); x = _f64(x)
    y = np.zeros((p.K, p.nn, 5))
    lib().or_jvp(ctypes.byref(p.c()), _dp(Q), _dp(x), _dp(y))
    return y


def jacobian(p: Params, Q: np.ndarray):
    """Global Jacobian A = dR/dQ as a scipy CSR matrix (global dof order)."""
    import scipy.sparse as sp
    Q = _f64(Q)
    ne = p.nn * 5
    cap = int(p.K * 27 * ne * ne * 0.6) + 1024
    while True:
        rows = np.zeros(cap, np.int32); cols = np.zeros(cap, np.int32); vals = np.zeros(cap)
        nnz = lib().or_jacobian_coo(ctypes.byref(p.c()), _dp(Q), cap, _ip(rows), _ip(cols), _dp(vals))
        if nnz <= cap:
            break
        cap = int(nnz)
    A = sp.csr_matrix((vals[:nnz], (rows[:nnz], cols[:nnz])), shape=(p.ndof, p.ndof))
    A.sum_duplicates()
    return A


def jacobian_element_rows(p: Params, Q: np.ndarray, e: int):
    """Rows of element e: dict {column element c: dense block [nn*5, nn*5]} (natural order)."""
    Q = _f64(Q)
    ne = p.nn * 5
    elems = np.zeros(27, np.int32)
    blocks = np.zeros((27, ne, ne))
    cnt = lib().or_jacobian_elem_rows(ctypes.byref(p.c()), _dp(Q), e, _ip(elems), _dp(blocks))
    return {int(elems[i]): blocks[i].copy() for i in range(cnt)}


def num_flux(p: Params, qL, qR, d: int, s: int) -> np.ndarray:
    f = np.zeros(5)
    lib().or_num_flux(ctypes.byref(p.c()), _dp(_f64(qL)), _dp(_f64(qR)), d, s, _dp(f))
    return f


def phys_flux(p: Params, q, g, d: int):
    fa = np.zeros(5); fv = np.zeros(5)
    lib().or_phys_flux(ctypes.byref(p.c()), _dp(_f64(q)), _dp(_f64(g)), d, _dp(fa), _dp(fv))
    return fa, fv


from .linalg import (  # noqa: E402
    MixedCondensedSystem, black_schur_correction, boundary_interior_split, boundary_interior_split_mixed,
    checkerboard, condensed_operator, condensed_solve, condensed_solve_mixed, corrected_black_blocks, global_solve,
    global_solve_dense, gmres, ratio_formula, red_black_apply,
)


# ---- meshes of mixed order (element e of order orders[e]; mortar faces between orders)
# States are flat [sum_e (N_e+1)^3, 5], element by element.  `force_mortar` routes the
# faces between equal orders through the mortar too (it must then reduce to the
# conforming face).

def _orders(p: Params, orders) -> np.ndarray:
    o = np.ascontiguousarray(orders, dtype=np.int32)
    if o.shape != (p.K,):
        raise ValueError("one order per element")
    return o


def mixed_nodes(orders) -> int:
    return int(sum((int(N) + 1) ** 3 for N in orders))


def residual_mixed(p: Params, orders, Q, Qs=None, Qsm1=None, force_mortar: bool = False) -> np.ndarray:
    """R(Q) of eq. NeqtonEq on a mixed-order mesh, flat [nodes, 5]."""
    o = _orders(p, orders)
    Q = _f64(Q)
    Qs = Q if Qs is None else _f64(Qs)
    Qsm1 = Qs if Qsm1 is None else _f64(Qsm1)
    R = np.zeros((mixed_nodes(o), 5))
    if lib().or_residual_mixed(ctypes.byref(p.c()), _ip(o), int(force_mortar), _dp(Q), _dp(Qs), _dp(Qsm1),
                               _dp(R)) != 0:
        raise ValueError("orders must lie in 1..7, with the BR1 viscous flux")
    return R


def jvp_mixed(p: Params, orders, Q, x, force_mortar: bool = False) -> np.ndarray:
    """(dR/dQ)(Q) x on a mixed-order mesh, flat [nodes, 5]."""
    o = _orders(p, orders)
    Q = _f64(Q); x = _f64(x)
    y = np.zeros((mixed_nodes(o), 5))
    if lib().or_jvp_mixed(ctypes.byref(p.c()), _ip(o), int(force_mortar), _dp(Q), _dp(x), _dp(y)) != 0:
        raise ValueError("orders must lie in 1..7, with the BR1 viscous flux")
    return y


def jacobian_mixed(p: Params, orders, Q, force_mortar: bool = False) -> np.ndarray:
    """Dense dR/dQ on a (small) mixed-order mesh, [dofs, dofs]."""
    o = _orders(p, orders)
    Q = _f64(Q)
    dofs = mixed_nodes(o) * 5
    A = np.zeros((dofs, dofs))
    if lib().or_jacobian_mixed(ctypes.byref(p.c()), _ip(o), int(force_mortar), _dp(Q), _dp(A)) != 0:
        raise ValueError("orders must lie in 1..7, with the BR1 viscous flux")
    return A


def jacobian_mixed_sparse(p: Params, orders, Q, force_mortar: bool = False):
    """dR/dQ on a mixed-order mesh as a scipy CSR matrix (flat ragged dof order)."""
    import scipy.sparse as sp
    o = _orders(p, orders)
    Q = _f64(Q)
    dofs = mixed_nodes(o) * 5
    ne_max = 5 * (int(o.max()) + 1) ** 3
    cap = int(dofs * min(27 * ne_max, dofs) * 0.3) + 1024
    while True:
        rows = np.zeros(cap, np.int32); cols = np.zeros(cap, np.int32); vals = np.zeros(cap)
        nnz = lib().or_jacobian_mixed_coo(ctypes.byref(p.c()), _ip(o), int(force_mortar), _dp(Q), cap,
                                          _ip(rows), _ip(cols), _dp(vals))
        if nnz < 0:
            raise ValueError("orders must lie in 1..7, with the BR1 viscous flux")
        if nnz <= cap:
            break
        cap = int(nnz)
    A = sp.csr_matrix((vals[:nnz], (rows[:nnz], cols[:nnz])), shape=(dofs, dofs))
    A.sum_duplicates()
    return A


def jacobian_mixed_element_rows(p: Params, orders, Q, e: int, force_mortar: bool = False):
    """Rows of element e on a mixed-order mesh: {column element c: dense block
    [(N_e+1)^3 5, (N_c+1)^3 5]} over the 3x3x3 block of elements around e."""
    o = _orders(p, orders)
    Q = _f64(Q)
    ne = lambda x: 5 * (int(o[x]) + 1) ** 3
    elems = np.zeros(27, np.int32)
    total = ne(e) * 27 * 5 * (int(o.max()) + 1) ** 3
    blocks = np.zeros(total)
    cnt = lib().or_jacobian_mixed_elem_rows(ctypes.byref(p.c()), _ip(o), int(force_mortar), _dp(Q), int(e),
                                            _ip(elems), _dp(blocks))
    if cnt < 0:
        raise ValueError("orders must lie in 1..7, with the BR1 viscous flux")
    out, off = {}, 0
    for i in range(cnt):
        c = int(elems[i])
        size = ne(e) * ne(c)
        out[c] = blocks[off:off + size].reshape(ne(e), ne(c)).copy()
        off += size
    return out

