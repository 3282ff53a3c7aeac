"""Schur-corrected red-black block sweep of the condensed system (test infrastructure only).

Not in the paper: its GMRES on S x_b = g (Sec. 2.2, eq. SC_step1) is preconditioned by point
Jacobi (Sec. 4).  The preconditioner here is one forward block Gauss-Seidel sweep over the
checkerboard colouring (red: ex + ey + ez even), z_r = S_rr^{-1} v_r, then
z_b = D_b^{-1} (v_b - sum_m S_bm z_m) on the black elements (``linalg.red_black_apply``).

Eliminating the red unknowns from S leaves the black Schur complement
Sigma = S_bb - S_br S_rr^{-1} S_rb, and the sweep's preconditioned operator has the spectrum
of D^{-1} Sigma (plus ones), so the best block-diagonal D is the block diagonal of Sigma,
S_bb - sum_m S_bm S_mm^{-1} S_mb over the red face neighbours m of b.  Its dominant part
comes through the co-located node pairs of each shared face: for a face f of b with red
neighbour m, node k of b on f and k' the node of m at the same point,

    C_b[k, l] -= S_(k,k') [S_mm^{-1}]_(k',l') S_(l',l)      for every k, l on f,

with the whole face block of the neighbour's inverse [S_mm^{-1}]_(f',f') (the diagonal node
blocks alone, or the first-order off-diagonal terms, lose most of the gain).  D_b = S_bb + C_b.
Everything here is a plain FP64 restatement on the oracle's dense S (element-major, boundary
nodes in the natural order of ``learned.boundary_nodes``, 5 variables per node).
"""
from __future__ import annotations

import numpy as np

from . import learned as LN
from .linalg import checkerboard


def face_node_lists(N: int):
    """For each face f (0..5 = -x, +x, -y, +y, -z, +z): the condensed indices of the
    element's boundary nodes on f (ascending) and of the neighbour's nodes at the same
    points (the neighbour sees them on the opposite face)."""
    bn = LN.boundary_nodes(N)
    pos = {int(m): i for i, m in enumerate(bn)}
    nodes, mirror = [], []
    for f in range(6):
        on = [a for a, m in enumerate(bn) if f in LN.node_faces(N, int(m))]
        nodes.append(on)
        mirror.append([pos[LN.mirror_node(N, int(bn[a]), f)] for a in on])
    return nodes, mirror


def _dofs(nodes) -> np.ndarray:
    return np.concatenate([np.arange(5 * a, 5 * a + 5) for a in nodes])


def face_schur_correction(S: np.ndarray, n: int, N: int) -> dict:
    """C_b (nb x nb) for every black element b: the co-located face-block Schur correction
    of the red face neighbours defined in the module docstring."""
    K = n ** 3
    nb = S.shape[0] // K
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    nodes, mirror = face_node_lists(N)
    col = checkerboard(n)
    inv = {}
    out = {}
    for b in np.where(col == 1)[0]:
        C = np.zeros((nb, nb))
        for f in range(6):
            m = LN.face_neighbour(n, int(b), f)
            if col[m] == 1:  # odd n: the periodic wrap joins two black elements; no red to eliminate
                continue
            if m not in inv:
                inv[m] = np.linalg.inv(S[blk(m), blk(m)])
            Sbm, Smb = S[blk(b), blk(m)], S[blk(m), blk(b)]
            fb, fm = _dofs(nodes[f]), _dofs(mirror[f])
            Z = inv[m][np.ix_(fm, fm)]
            # co-located couplings: 5 x 5 blocks on the node-pair diagonal
            Skc = np.zeros((len(fb), len(fm)))
            Sck = np.zeros((len(fm), len(fb)))
            for i in range(len(nodes[f])):
                r, c = fb[5 * i:5 * i + 5], fm[5 * i:5 * i + 5]
                Skc[5 * i:5 * i + 5, 5 * i:5 * i + 5] = Sbm[np.ix_(r, c)]
                Sck[5 * i:5 * i + 5, 5 * i:5 * i + 5] = Smb[np.ix_(c, r)]
            C[np.ix_(fb, fb)] -= Skc @ Z @ Sck
        out[int(b)] = C
    return out


def face_schur_blocks(S: np.ndarray, n: int, N: int) -> dict:
    """D_b = S_bb + C_b for every black element (the ``black_blocks`` of red_black_apply)."""
    K = n ** 3
    nb = S.shape[0] // K
    return {b: S[b * nb:(b + 1) * nb, b * nb:(b + 1) * nb] + C
            for b, C in face_schur_correction(S, n, N).items()}


def black_schur_blocks(S: np.ndarray, n: int) -> dict:
    """The block diagonal of the black Schur complement with the red blocks taken one by
    one, S_bb - sum_m S_bm S_mm^{-1} S_mb (every red element m coupled to b): the quantity
    the face-block correction approximates, written out for its pins."""
    K = n ** 3
    nb = S.shape[0] // K
    blk = lambda e: slice(e * nb, (e + 1) * nb)
    col = checkerboard(n)
    out = {}
    for b in np.where(col == 1)[0]:
        D = S[blk(b), blk(b)].copy()
        for m in np.where(col == 0)[0]:
            Sbm, Smb = S[blk(b), blk(m)], S[blk(m), blk(b)]
            if np.any(Sbm) and np.any(Smb):
                D -= Sbm @ np.linalg.solve(S[blk(m), blk(m)], Smb)
        out[int(b)] = D
    return out
