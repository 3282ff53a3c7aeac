"""Learned correction of the block-Jacobi preconditioner (test infrastructure only).

Not in the paper: the condensed system S x_b = g of Sec. 2.2 (eq. SC_step1) is solved by
GMRES preconditioned with the inverses of the element blocks S_ee; a small network adds
a 5 x 5 correction to the diagonal node blocks of each S_ee^{-1}.  Everything here is a
plain FP64 restatement, written against the dense condensed matrix S of the oracle.

Definitions (one sample per element e and boundary node k of e; boundary nodes in the
natural order of the oracle's condensed system, 5 variables per node):

* face of k: the lowest-index face containing k in the order -x, +x, -y, +y, -z, +z;
  n = the face neighbour of e across it; k' = the node of n at the same point (k with
  its index normal to the face mirrored, 0 <-> N);
* S_patch = S restricted to the boundary dofs of e and n;
* target  C*_k = [S_patch^{-1}]_kk - [S_ee^{-1}]_kk;
* features (64): q_k over free-stream scales (5); [S_ee]_kk and [S]_(k, k'), each over
  its Frobenius norm (25 + 25); (Ma, Re / 1000, dt c_inf / h, N) (4); 5 zeros;
* the network predicts the target times ||[S_ee]_kk||_F (a dimensionless 5 x 5 block);
* network: 64 -> 256 -> 256 -> 25, ReLU after the two hidden layers;
* loss: mean over samples of ||y - t||^2 / (||t||^2 + eps) (squared relative Frobenius
  error of the scaled correction).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 64, 256, 25
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


def features_and_targets(S: np.ndarray, Q: np.ndarray, n: int, N: int, Ma: float, Re: float, dt: float,
                         L: float = 2.0 * np.pi, gamma: float = 1.4):
    """Features [K*nbn, 64], scaled targets [K*nbn, 25] and the block norms ||[S_ee]_kk||_F.

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
    Sinv_ee = [np.linalg.inv(S[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb]) for e in range(K)]
    patch_inv = {}
    for e in range(K):
        for a, m in enumerate(Bn):
            f = node_face(N, int(m))
            nbe = face_neighbour(n, e, f)
            b = pos[mirror_node(N, int(m), f)]
            r = e * nb + 5 * a
            c = nbe * nb + 5 * b
            Skk = S[r:r + 5, r:r + 5]
            Skc = S[r:r + 5, c:c + 5]
            s = e * nbn + a
            F[s, 0:5] = Q[e, m] / scale
            F[s, 5:30] = _unit(Skk).reshape(-1)
            F[s, 30:55] = _unit(Skc).reshape(-1)
            F[s, 55:59] = scal
            if (e, f) not in patch_inv:
                ids = np.concatenate([np.arange(e * nb, (e + 1) * nb), np.arange(nbe * nb, (nbe + 1) * nb)])
                patch_inv[(e, f)] = np.linalg.inv(S[np.ix_(ids, ids)])
            Pinv = patch_inv[(e, f)]
            Cstar = Pinv[5 * a:5 * a + 5, 5 * a:5 * a + 5] - Sinv_ee[e][5 * a:5 * a + 5, 5 * a:5 * a + 5]
            snorm[s] = np.linalg.norm(Skk)
            T[s] = (Cstar * snorm[s]).reshape(-1)
    return F, T, snorm


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


def corrected_apply(S: np.ndarray, y: np.ndarray, snorm: np.ndarray, v: np.ndarray, K: int, nb: int):
    """P v = S_ee^{-1} v_e + C_k v_k with C_k = y_k / ||[S_ee]_kk||_F, per element."""
    out = np.empty_like(v)
    nbn = nb // 5
    for e in range(K):
        sl = slice(e * nb, (e + 1) * nb)
        z = np.linalg.solve(S[sl, sl], v[sl])
        for a in range(nbn):
            s = e * nbn + a
            C = y[s].reshape(5, 5) / snorm[s]
            z[5 * a:5 * a + 5] += C @ v[e * nb + 5 * a:e * nb + 5 * a + 5]
        out[sl] = z
    return out
