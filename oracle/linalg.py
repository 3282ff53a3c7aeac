"""Static condensation and Krylov solves of the oracle (test infrastructure only).

Follows Sec. 2.2 (eqs. BlockSystem, StaticCondBlock, SC_step1, SC_step2) and Sec. 3
(eq. StaticDGSEM_QbQiSystem) of the paper, written in the row-column convention:
``A_bi`` holds rows on element boundaries and columns in element interiors, ``A_ib``
the reverse.  With that convention the condensed system reads

    S x_b = g,   S = A_bb - A_bi A_ii^{-1} A_ib,   g = B_b - A_bi A_ii^{-1} B_i,
    x_i = A_ii^{-1} (B_i - A_ib x_b).

Library primitives used as single steps: scipy's dense LU (lu_factor / lu_solve) for
each element block and for the small dense condensed matrix, and scipy's sparse LU
for the global reference solve x = A^{-1} B.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def ratio_formula(N: int, d: int = 3) -> float:
    """n1/(n1+n2) = ((N+1)^d - (N-1)^d)/(N+1)^d (eq. ratio, Table tab:ratio)."""
    return ((N + 1) ** d - (N - 1) ** d) / (N + 1) ** d


def boundary_interior_split(n: int, N: int):
    """Local interior / boundary node lists and the global dof indices of each set.

    A node (i, j, k) is interior when 0 < i, j, k < N.  Returns
    (interior_nodes, boundary_nodes, I[K, 5*ni_nodes], B[K, 5*nb_nodes]).
    """
    p = N + 1
    nn = p ** 3
    idx = np.arange(nn)
    i, j, k = idx % p, (idx // p) % p, idx // (p * p)
    inner = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    In = idx[inner]
    Bn = idx[~inner]
    K = n ** 3
    e = np.arange(K)[:, None, None]
    I = ((e * nn + In[None, :, None]) * 5 + np.arange(5)[None, None, :]).reshape(K, -1)
    B = ((e * nn + Bn[None, :, None]) * 5 + np.arange(5)[None, None, :]).reshape(K, -1)
    return In, Bn, I, B


class CondensedSystem:
    """The pieces of the condensed system built from a global CSR Jacobian."""

    def __init__(self, A: sp.csr_matrix, n: int, N: int):
        self.n, self.N = n, N
        self.In, self.Bn, self.I, self.B = boundary_interior_split(n, N)
        K = n ** 3
        If = self.I.reshape(-1)
        Bf = self.B.reshape(-1)
        A = A.tocsr()
        self.A_ii = A[If][:, If].tocsr()
        self.A_ib = A[If][:, Bf].tocsr()   # rows interior, columns boundary
        self.A_bi = A[Bf][:, If].tocsr()   # rows boundary, columns interior
        self.A_bb = A[Bf][:, Bf].tocsr()
        ni = self.I.shape[1]
        # A_ii must be block diagonal: one dense block per element (Sec. 3.1).
        coo = self.A_ii.tocoo()
        self.aii_offblock_nnz = int(np.count_nonzero((coo.row // ni) != (coo.col // ni)))
        self.blocks = []
        for e in range(K):
            blk = self.A_ii[e * ni:(e + 1) * ni, e * ni:(e + 1) * ni].toarray()
            self.blocks.append(sla.lu_factor(blk))
        self.ni = ni
        self.nb = self.B.shape[1]
        self.K = K

    def aii_solve(self, v: np.ndarray) -> np.ndarray:
        """A_ii^{-1} v, element by element with the LU factors."""
        v = v.reshape(self.K, self.ni)
        out = np.empty_like(v)
        for e in range(self.K):
            out[e] = sla.lu_solve(self.blocks[e], v[e])
        return out.reshape(-1)

    def aii_solve_mat(self, M: np.ndarray) -> np.ndarray:
        M = M.reshape(self.K, self.ni, -1)
        out = np.empty_like(M)
        for e in range(self.K):
            out[e] = sla.lu_solve(self.blocks[e], M[e])
        return out.reshape(self.K * self.ni, -1)

    def matvec(self, xb: np.ndarray) -> np.ndarray:
        """S x_b = A_bb x_b - A_bi A_ii^{-1} A_ib x_b (eq. SC_step1, left-hand side)."""
        return self.A_bb @ xb - self.A_bi @ self.aii_solve(self.A_ib @ xb)

    def rhs(self, Bvec: np.ndarray) -> np.ndarray:
        """g = B_b - A_bi A_ii^{-1} B_i (eq. SC_step1, right-hand side)."""
        Bb = Bvec[self.B.reshape(-1)]
        Bi = Bvec[self.I.reshape(-1)]
        return Bb - self.A_bi @ self.aii_solve(Bi)

    def back_substitute(self, Bvec: np.ndarray, xb: np.ndarray) -> np.ndarray:
        """x_i = A_ii^{-1} (B_i - A_ib x_b) (eq. SC_step2); returns the full x."""
        Bi = Bvec[self.I.reshape(-1)]
        xi = self.aii_solve(Bi - self.A_ib @ xb)
        x = np.zeros(self.K * (self.ni + self.nb))
        x[self.I.reshape(-1)] = xi
        x[self.B.reshape(-1)] = xb
        return x

    def dense_S(self) -> np.ndarray:
        Y = self.aii_solve_mat(self.A_ib.toarray())
        return self.A_bb.toarray() - self.A_bi @ Y

    def own_block_S(self, e: int) -> np.ndarray:
        """S_ee = A_bb[e,e] - A_bi[e,e] A_ii[e]^{-1} A_ib[e,e]: element e's own block."""
        ni, nb = self.ni, self.nb
        rb = slice(e * nb, (e + 1) * nb)
        ri = slice(e * ni, (e + 1) * ni)
        Abb = self.A_bb[rb, rb].toarray()
        Abi = self.A_bi[rb, ri].toarray()
        Aib = self.A_ib[ri, rb].toarray()
        return Abb - Abi @ sla.lu_solve(self.blocks[e], Aib)

    def block_jacobi(self):
        """Factors of every S_ee; returns the preconditioner z = blockdiag(S_ee)^{-1} v."""
        facs = [sla.lu_factor(self.own_block_S(e)) for e in range(self.K)]
        nb = self.nb

        def apply(v):
            v = v.reshape(self.K, nb)
            out = np.empty_like(v)
            for e in range(self.K):
                out[e] = sla.lu_solve(facs[e], v[e])
            return out.reshape(-1)
        return apply


def condensed_operator(A, n: int, N: int) -> CondensedSystem:
    return CondensedSystem(A, n, N)


def global_solve(A: sp.csr_matrix, Bvec: np.ndarray) -> np.ndarray:
    """x = A^{-1} B by sparse LU (the plain definition of the Newton update)."""
    return spla.splu(A.tocsc()).solve(Bvec)


def global_solve_dense(A, Bvec: np.ndarray) -> np.ndarray:
    """x = A^{-1} B by dense LU with partial pivoting (LAPACK getrf/getrs through scipy);
    faster than the sparse LU once the element couplings fill the factors (20,480 dofs)."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.array(A, dtype=np.float64)
    return sla.lu_solve(sla.lu_factor(Ad, overwrite_a=True, check_finite=False), Bvec, check_finite=False)


def gmres(matvec, b: np.ndarray, precond=None, restart: int = 30, tol: float = 1e-8,
          maxiter: int = 2000, atol: float | None = None):
    """Right-preconditioned restarted GMRES(m) with classical Gram-Schmidt applied
    twice and Givens rotations; x0 = 0.  Stops when ||b - A x|| <= max(tol*||b||, atol).

    Returns (x, info) with info = {'iters', 'history', 'converged'}; history holds the
    Arnoldi residual estimate after every iteration.
    """
    M = precond if precond is not None else (lambda v: v)
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    target = max(tol * bnorm, atol or 0.0)
    r = b.copy()
    beta = np.linalg.norm(r)
    hist = [beta]
    total = 0
    if beta <= target:
        return x, {"iters": 0, "history": hist, "converged": True}
    while total < maxiter:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart); sn = np.zeros(restart)
        gvec = np.zeros(restart + 1); gvec[0] = beta
        V[0] = r / beta
        jlast = 0
        for j in range(restart):
            w = matvec(M(V[j]))
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den; sn[j] = H[j + 1, j] / den
            H[j, j] = den; H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            jlast = j
            hist.append(abs(gvec[j + 1]))
            if abs(gvec[j + 1]) <= target or total >= maxiter:
                break
        k = jlast + 1
        y = sla.solve_triangular(H[:k, :k], gvec[:k])
        x = x + M(V[:k].T @ y)
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= target:
            return x, {"iters": total, "history": hist, "converged": True}
    return x, {"iters": total, "history": hist, "converged": False}


def condensed_solve(A, Bvec: np.ndarray, n: int, N: int, method: str = "direct",
                    tol: float = 1e-10, restart: int = 30, maxiter: int = 2000):
    """Solve A x = B by static condensation: condense (eq. SC_step1), solve for the
    boundary unknowns (dense LU or block-Jacobi GMRES), back-substitute (eq. SC_step2).
    Returns (x, info)."""
    cs = CondensedSystem(A, n, N)
    g = cs.rhs(Bvec)
    info = {"aii_offblock_nnz": cs.aii_offblock_nnz}
    if method == "direct":
        xb = np.linalg.solve(cs.dense_S(), g)
    else:
        bnorm = np.linalg.norm(Bvec)
        xb, ginfo = gmres(cs.matvec, g, precond=cs.block_jacobi(), restart=restart,
                          tol=0.0, atol=tol * bnorm, maxiter=maxiter)
        info.update(ginfo)
    return cs.back_substitute(Bvec, xb), info


# ---- meshes of mixed order: element blocks of uneven sizes --------------------------

def boundary_interior_split_mixed(orders):
    """Per element, the global dof indices of its interior and boundary nodes (flat
    ragged order, element by element; a node (i, j, k) of an order-N element is interior
    when 0 < i, j, k < N).  Returns (I_list, B_list)."""
    I_list, B_list, off = [], [], 0
    for N in orders:
        N = int(N)
        p = N + 1
        idx = np.arange(p ** 3)
        i, j, k = idx % p, (idx // p) % p, idx // (p * p)
        inner = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
        dof = lambda nodes: ((off + nodes[:, None]) * 5 + np.arange(5)[None, :]).reshape(-1)
        I_list.append(dof(idx[inner]))
        B_list.append(dof(idx[~inner]))
        off += p ** 3
    return I_list, B_list


class MixedCondensedSystem:
    """The condensed system of a mixed-order mesh (same algebra as CondensedSystem, with
    element blocks of uneven sizes): S = A_bb - A_bi A_ii^{-1} A_ib, one dense LU per A_ii."""

    def __init__(self, A, orders):
        self.I_list, self.B_list = boundary_interior_split_mixed(orders)
        If, Bf = np.concatenate(self.I_list), np.concatenate(self.B_list)
        self.If, self.Bf = If, Bf
        A = sp.csr_matrix(A)
        self.A_ii = A[If][:, If].tocsr()
        self.A_ib = A[If][:, Bf].tocsr()
        self.A_bi = A[Bf][:, If].tocsr()
        self.A_bb = A[Bf][:, Bf].tocsr()
        self.isz = [len(x) for x in self.I_list]
        self.bsz = [len(x) for x in self.B_list]
        self.ioff = np.concatenate([[0], np.cumsum(self.isz)])
        self.boff = np.concatenate([[0], np.cumsum(self.bsz)])
        coo = self.A_ii.tocoo()
        blk = np.searchsorted(self.ioff, np.arange(len(If)), side="right") - 1
        self.aii_offblock_nnz = int(np.count_nonzero(blk[coo.row] != blk[coo.col]))
        self.blocks = [sla.lu_factor(self.A_ii[a:b, a:b].toarray()) if b > a else None
                       for a, b in zip(self.ioff[:-1], self.ioff[1:])]

    def aii_solve(self, v):
        out = np.empty_like(v)
        for e, (a, b) in enumerate(zip(self.ioff[:-1], self.ioff[1:])):
            if b > a:
                out[a:b] = sla.lu_solve(self.blocks[e], v[a:b])
        return out

    def matvec(self, xb):
        return self.A_bb @ xb - self.A_bi @ self.aii_solve(self.A_ib @ xb)

    def rhs(self, Bvec):
        return Bvec[self.Bf] - self.A_bi @ self.aii_solve(Bvec[self.If])

    def back_substitute(self, Bvec, xb):
        x = np.zeros(Bvec.size)
        x[self.If] = self.aii_solve(Bvec[self.If] - self.A_ib @ xb)
        x[self.Bf] = xb
        return x

    def dense_S(self):
        Y = np.zeros((len(self.If), len(self.Bf)))
        Aib = self.A_ib.toarray()
        for e, (a, b) in enumerate(zip(self.ioff[:-1], self.ioff[1:])):
            if b > a:
                Y[a:b] = sla.lu_solve(self.blocks[e], Aib[a:b])
        return self.A_bb.toarray() - self.A_bi @ Y

    def block_jacobi(self):
        """z = blockdiag(S_ee)^{-1} v with every element's own Schur block."""
        facs = []
        for e in range(len(self.bsz)):
            rb = slice(self.boff[e], self.boff[e + 1])
            ri = slice(self.ioff[e], self.ioff[e + 1])
            Abb = self.A_bb[rb, rb].toarray()
            if self.isz[e]:
                Y = sla.lu_solve(self.blocks[e], self.A_ib[ri, rb].toarray())
                Abb = Abb - self.A_bi[rb, ri].toarray() @ Y
            facs.append(sla.lu_factor(Abb))

        def apply(v):
            out = np.empty_like(v)
            for e in range(len(self.bsz)):
                rb = slice(self.boff[e], self.boff[e + 1])
                out[rb] = sla.lu_solve(facs[e], v[rb])
            return out
        return apply


def condensed_solve_mixed(A, Bvec: np.ndarray, orders, method: str = "direct", tol: float = 1e-10,
                          restart: int = 30, maxiter: int = 2000):
    """condensed_solve on a mixed-order mesh."""
    cs = MixedCondensedSystem(A, orders)
    g = cs.rhs(Bvec)
    info = {"aii_offblock_nnz": cs.aii_offblock_nnz}
    if method == "direct":
        xb = np.linalg.solve(cs.dense_S(), g)
    else:
        bnorm = np.linalg.norm(Bvec)
        xb, ginfo = gmres(cs.matvec, g, precond=cs.block_jacobi(), restart=restart,
                          tol=0.0, atol=tol * bnorm, maxiter=maxiter)
        info.update(ginfo)
    return cs.back_substitute(Bvec, xb), info


# ---- red-black block Gauss-Seidel preconditioner of the condensed system -------------
# Not in the paper (its GMRES uses point Jacobi, Sec. 4).  Elements coloured like a
# checkerboard, colour(e) = (ex + ey + ez) mod 2 (0 = red); one application is one forward
# block sweep over the element blocks of S: red blocks first, then every black block
# against what the red elements already hold.

def checkerboard(n: int) -> np.ndarray:
    """colour[e] for e = ex + n (ey + n ez)."""
    e = np.arange(n ** 3)
    return ((e % n) + (e // n) % n + e // (n * n)) % 2


def red_black_apply(S: np.ndarray, n: int, v: np.ndarray, black_blocks=None) -> np.ndarray:
    """z = P v for the dense condensed matrix S (element-major, nb dofs per element):
    z_r = S_rr^-1 v_r on red elements, then z_b = D_b^-1 (v_b - sum_n S_bn z_n) on black ones,
    D_b = S_bb or black_blocks[b] (a dict of replacement blocks)."""
    K = n ** 3
    nb = S.shape[0] // K
    col = checkerboard(n)
    z = np.zeros_like(v)
    for e in np.where(col == 0)[0]:
        sl = slice(e * nb, (e + 1) * nb)
        z[sl] = np.linalg.solve(S[sl, sl], v[sl])
    t = S @ z  # black rows: sum over red n of S_bn z_n (z is zero on the black elements)
    for e in np.where(col == 1)[0]:
        sl = slice(e * nb, (e + 1) * nb)
        D = S[sl, sl] if black_blocks is None else black_blocks[e]
        z[sl] = np.linalg.solve(D, v[sl] - t[sl])
    return z


def black_schur_correction(S: np.ndarray, n: int) -> np.ndarray:
    """The node-diagonal 5 x 5 blocks of -sum_{red n} S_bn S_nn^-1 S_nb for every black
    element b (zero for red elements): what eliminating the red neighbours adds to the
    diagonal of the black block.  Returns [K * nbn, 5, 5] in the condensed order."""
    K = n ** 3
    nb = S.shape[0] // K
    nbn = nb // 5
    col = checkerboard(n)
    C = np.zeros((K * nbn, 5, 5))
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    for b in np.where(col == 1)[0]:
        acc = np.zeros((nb, nb))
        for m in np.where(col == 0)[0]:
            Sbm, Smb = S[blk(b), blk(m)], S[blk(m), blk(b)]
            if not (np.any(Sbm) and np.any(Smb)):
                continue
            acc -= Sbm @ np.linalg.solve(S[blk(m), blk(m)], Smb)
        for a in range(nbn):
            C[b * nbn + a] = acc[5 * a:5 * a + 5, 5 * a:5 * a + 5]
    return C


def corrected_black_blocks(S: np.ndarray, n: int, C: np.ndarray) -> dict:
    """D_b = S_bb plus the per-node blocks C on its diagonal node blocks, black elements."""
    K = n ** 3
    nb = S.shape[0] // K
    nbn = nb // 5
    out = {}
    for b in np.where(checkerboard(n) == 1)[0]:
        D = S[b * nb:(b + 1) * nb, b * nb:(b + 1) * nb].copy()
        for a in range(nbn):
            D[5 * a:5 * a + 5, 5 * a:5 * a + 5] += C[b * nbn + a]
        out[int(b)] = D
    return out
