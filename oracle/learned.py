"""Learned correction of the red-black block sweep (test infrastructure only).

Not in the paper: the condensed system S x_b = g of Sec. 2.2 (eq. SC_step1) is solved by
GMRES preconditioned with one forward block sweep over the checkerboard colouring of the
elements (red: ex + ey + ez even): z_r = S_rr^{-1} v_r, then z_b = D_b^{-1} (v_b - sum S_bm z_m).
The black blocks are corrected, D_b = S_bb + C_b, C_b block-diagonal over the 5 x 5 node
blocks, from a network's prediction of the node blocks of the face-block inverses.
Everything here is a plain FP64 restatement, written against the dense condensed matrix S of
the oracle.

Definitions (one sample per element e and boundary node k of e; boundary nodes in the
natural order of the oracle's condensed system, 5 variables per node):

* for each face f of e containing k: n_f = the face neighbour across it, k'_f = the node of
  n_f at the same point (k with its index normal to f mirrored, 0 <-> N); the lowest of these
  faces (order -x, +x, -y, +y, -z, +z) is f, with n and k';
* Z_k = [S_ee^{-1}]_kk, the diagonal node block of the inverse of the element's face block;
* target = (Z_k - [S_ee]_kk^{-1}) ||[S_ee]_kk||_F for every sample;
* correction of a black element b: C_k = -(1/2) sum_f S_(k,k'_f) Z_(k'_f) S_(k'_f,k), with
  Z_(k') = [S_nn]_(k'k')^{-1} + y_(k') / ||[S_nn]_(k'k')||_F from the network's output y (the
  exact Z for y = target): the co-located part of the Schur correction of the red
  neighbours, halved;
* features (128): q_k over free-stream scales (5); [S_ee]_kk, [S]_(k,k'), [S]_(k',k) and
  [S_nn]_(k',k'), each over its Frobenius norm (4 x 25); (Ma, Re / 1000, dt c_inf / h, N) (4);
  the number of faces of e containing k over 3 (1); the Frobenius norms of [S]_(k,k'),
  [S]_(k',k) and [S_nn]_(k',k') over that of [S_ee]_kk (3); 15 zeros;
* network: 128 -> 256 -> 256 -> 25, ReLU after the two hidden layers;
* loss: mean over samples of ||y - t||^2 / (||t||^2 + eps) (squared relative Frobenius
  error of the scaled correction).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 128, 256, 25
LOSS_EPS = 1e-12


def boundary_nodes(N: int) -> np.ndarray:
    """Natural indices of the boundary nodes of one element, in the condensed order."""
    p = N + 1
    idx = np.arange(p ** 3)
    i, j, k = idx % p, (idx // p) % p, idx // (p * p)
    inner = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    return idx[~inner]


def node_face(N: int, m: int) -> int:
    """Lowest-index face (0..5 = -x, +x, -y, +y, -z, +z) containing boundary node m."""
    p = N + 1
    c = (m % p, (m // p) % p, m // (p * p))
    for d in range(3):
        if c[d] == 0:
            return 2 * d
        if c[d] == N:
            return 2 * d + 1
    raise ValueError("interior node")


def mirror_node(N: int, m: int, face: int) -> int:
    """The node of the neighbour across `face` that sits at the same point as m."""
    p = N + 1
    c = [m % p, (m // p) % p, m // (p * p)]
    d = face // 2
    c[d] = N - c[d]
    return c[0] + p * (c[1] + p * c[2])


def face_neighbour(n: int, e: int, face: int) -> int:
    """Periodic face neighbour of element e = ex + n (ey + n ez)."""
    c = [e % n, (e // n) % n, e // (n * n)]
    d, s = face // 2, (1 if face % 2 else -1)
    c[d] = (c[d] + s) % n
    return c[0] + n * (c[1] + n * c[2])


def free_stream_scales(gamma: float, Ma: float) -> np.ndarray:
    """rho_inf = 1, |v_inf| = 1 and rho E_inf = p_inf / (gamma - 1) + 1/2."""
    p_inf = 1.0 / (gamma * Ma * Ma)
    return np.array([1.0, 1.0, 1.0, 1.0, p_inf / (gamma - 1.0) + 0.5])


def _unit(b: np.ndarray) -> np.ndarray:
    nrm = np.linalg.norm(b)
    return b / nrm if nrm > 0 else np.zeros_like(b)


def node_face_count(N: int, m: int) -> int:
    """Number of element faces containing boundary node m (1 on a face, 2 on an edge, 3 at a corner)."""
    p = N + 1
    c = (m % p, (m // p) % p, m // (p * p))
    return sum(1 for d in range(3) if c[d] in (0, N))


LEARNED_DAMPING = 0.5


def node_faces(N: int, m: int) -> list:
    """The faces (0..5 = -x, +x, -y, +y, -z, +z) containing boundary node m, ascending."""
    p = N + 1
    c = (m % p, (m // p) % p, m // (p * p))
    out = []
    for d in range(3):
        if c[d] == 0:
            out.append(2 * d)
        elif c[d] == N:
            out.append(2 * d + 1)
    return out


def features_and_targets(S: np.ndarray, Q: np.ndarray, n: int, N: int, Ma: float, Re: float, dt: float,
                         L: float = 2.0 * np.pi, gamma: float = 1.4):
    """Features [K*nbn, 128], scaled targets [K*nbn, 25] and the block norms ||[S_ee]_kk||_F.

    S: dense condensed matrix (K*nb x K*nb) in the element-major condensed order.
    Q: state [K, (N+1)^3, 5].
    """
    Bn = boundary_nodes(N)
    nbn = len(Bn)
    nb = 5 * nbn
    K = n ** 3
    pos = {int(m): i for i, m in enumerate(Bn)}
    scale = free_stream_scales(gamma, Ma)
    h = L / n
    scal = np.array([Ma, Re / 1000.0, dt * (1.0 / Ma) / h, float(N)])
    F = np.zeros((K * nbn, N_IN))
    T = np.zeros((K * nbn, N_OUT))
    snorm = np.zeros(K * nbn)
    for e in range(K):
        blk = slice(e * nb, (e + 1) * nb)
        Sinv = np.linalg.inv(S[blk, blk])
        for a, m in enumerate(Bn):
            f = node_face(N, int(m))
            nbe = face_neighbour(n, e, f)
            b = pos[mirror_node(N, int(m), f)]
            r, c = e * nb + 5 * a, nbe * nb + 5 * b
            Skk, Skc, Sck, Scc = S[r:r + 5, r:r + 5], S[r:r + 5, c:c + 5], S[c:c + 5, r:r + 5], S[c:c + 5, c:c + 5]
            s = e * nbn + a
            nk = np.linalg.norm(Skk)
            F[s, 0:5] = Q[e, m] / scale
            F[s, 5:30] = _unit(Skk).reshape(-1)
            F[s, 30:55] = _unit(Skc).reshape(-1)
            F[s, 55:80] = _unit(Sck).reshape(-1)
            F[s, 80:105] = _unit(Scc).reshape(-1)
            F[s, 105:109] = scal
            F[s, 109] = len(node_faces(N, int(m))) / 3.0
            F[s, 110:113] = [np.linalg.norm(Skc) / nk, np.linalg.norm(Sck) / nk, np.linalg.norm(Scc) / nk]
            snorm[s] = nk
            T[s] = ((Sinv[5 * a:5 * a + 5, 5 * a:5 * a + 5] - np.linalg.inv(Skk)) * nk).reshape(-1)
    return F, T, snorm


def assemble_correction(S: np.ndarray, Y: np.ndarray, n: int, N: int) -> np.ndarray:
    """C [K*nbn, 5, 5]: for black elements C_k = -(1/2) sum_f S_(k,k'_f) Z_(k'_f) S_(k'_f,k) with
    Z_(k') = [S_nn]_(k'k')^{-1} + y_(k') / ||[S_nn]_(k'k')||_F; zero for red elements."""
    from .linalg import checkerboard
    Bn = boundary_nodes(N)
    nbn = len(Bn)
    nb = 5 * nbn
    K = n ** 3
    pos = {int(m): i for i, m in enumerate(Bn)}
    C = np.zeros((K * nbn, 5, 5))
    for e in np.where(checkerboard(n) == 1)[0]:
        for a, m in enumerate(Bn):
            r = e * nb + 5 * a
            for f in node_faces(N, int(m)):
                nbe = face_neighbour(n, e, f)
                b = pos[mirror_node(N, int(m), f)]
                c = nbe * nb + 5 * b
                Scc = S[c:c + 5, c:c + 5]
                Z = np.linalg.inv(Scc) + Y[nbe * nbn + b].reshape(5, 5) / np.linalg.norm(Scc)
                C[e * nbn + a] -= LEARNED_DAMPING * S[r:r + 5, c:c + 5] @ Z @ S[c:c + 5, r:r + 5]
    return C


def black_mask(n: int, N: int) -> np.ndarray:
    """True for the samples of black elements (the ones the correction applies to)."""
    from .linalg import checkerboard
    return np.repeat(checkerboard(n) == 1, len(boundary_nodes(N)))


# ---- the network -------------------------------------------------------------------

def init_params(seed: int = 0, scale_out: float = 0.1):
    """He-style initial weights (counter-free numpy generator; the GPU side receives the
    same arrays)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((N_H, N_IN)) * np.sqrt(2.0 / N_IN)
    W2 = rng.standard_normal((N_H, N_H)) * np.sqrt(2.0 / N_H)
    W3 = rng.standard_normal((N_OUT, N_H)) * np.sqrt(1.0 / N_H) * scale_out
    return {"W1": W1, "b1": np.zeros(N_H), "W2": W2, "b2": np.zeros(N_H), "W3": W3, "b3": np.zeros(N_OUT)}


def forward(P, X):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X; returns (y, cache)."""
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"].T + P["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(y, T):
    """Mean squared relative Frobenius error."""
    num = np.sum((y - T) ** 2, axis=1)
    den = np.sum(T ** 2, axis=1) + LOSS_EPS
    return float(np.mean(num / den))


def loss_grad(y, T):
    """d loss / d y."""
    den = np.sum(T ** 2, axis=1, keepdims=True) + LOSS_EPS
    return 2.0 * (y - T) / den / y.shape[0]


def backward(P, cache, dy):
    """Gradients of sum(dy * y) with respect to every parameter (chain rule, layer by layer)."""
    X, z1, h1, z2, h2 = cache
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(P, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, bias-corrected moments) in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)


def corrected_apply(S: np.ndarray, Y: np.ndarray, v: np.ndarray, n: int, N: int):
    """The learned sweep: red-black with D_b = S_bb + C, C assembled from the network outputs Y."""
    from .linalg import corrected_black_blocks, red_black_apply
    C = assemble_correction(S, Y, n, N)
    return red_black_apply(S, n, v, black_blocks=corrected_black_blocks(S, n, C))
