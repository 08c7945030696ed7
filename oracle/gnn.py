"""FP64 oracle of the learned block preconditioner for PCG on the reduced
camera system (RCS) of a sub-block.

TEST INFRASTRUCTURE ONLY: the tests load this module to check the CUDA
network kernels; nothing in the library package imports it.

The paper solves the RCS with conjugate gradients and block-Jacobi
preconditioning (Sec. 5.5: the 6x6 camera blocks on the diagonal). This
network predicts a correction of each camera's block so that the
preconditioned system is closer to the identity. Definitions, in the order
they are applied:

Graph. One node per camera of the system (S of size 6n x 6n, block (i, j) the
6x6 block of cameras i and j). An edge joins i != j when S_ij has a non-zero
entry (the two cameras share a point).

Node features x_i (21), from the diagonal block B_i = S_ii:
  x_i[0:6]  = log B_i[k,k] - mean over the system's nodes of log B_.[k,k]
  x_i[6:21] = B_i[k,l] / sqrt(B_i[k,k] B_i[l,l]) for (k,l) = (1,0), (2,0),
              (2,1), (3,0), ... (strict lower triangle, row by row)
Edge weight e_ij = ||S_ij||_F / sqrt(||B_i||_F ||B_j||_F).

Network (hidden width 64, three message-passing layers):
  h0   = relu(W0 x + b0)
  m_t  = sum_{j ~ i} e_ij h_{t-1, j}
  h_t  = relu(A_t h_{t-1} + B_t m_t + c_t),    t = 1, 2, 3
  C    = Wo h3 + bo           (21 values: a lower-triangular 6x6, row by row)

Preconditioner block: E = 0.5 tanh(C) (lower triangular, diagonal included),
L = chol(B_i), P_i = L (I + E)(I + E)^T L^T, so P_i is SPD whenever
|E_kk| < 1, and P_i = B_i (block-Jacobi) when the output layer is zero.
P_i^-1 = G^T G with G = (I + E)^-1 L^-1.

Loss over a set of systems with probe vectors z^p (u^p = S z^p):
  loss = sum_sys sum_p sum_i ||P_i^-1 u_i^p - z_i^p||^2 / sum ||z^p||^2
(for a block-diagonal P, (P^-1 S z)_i = P_i^-1 (S z)_i).

Parameters are one flat vector in the order W0, b0, (A_t, B_t, c_t) for
t = 1..3, Wo, bo; matrices row-major (out x in).
"""

from __future__ import annotations

import numpy as np

NF = 21
HID = 64
LAYERS = 3
EPS = 0.5
TRIL = [(r, c) for r in range(6) for c in range(r + 1)]           # 21, with diagonal
STRICT = [(r, c) for r in range(6) for c in range(r)]             # 15


def param_shapes():
    sh = [("W0", (HID, NF)), ("b0", (HID,))]
    for t in range(1, LAYERS + 1):
        sh += [(f"A{t}", (HID, HID)), (f"B{t}", (HID, HID)), (f"c{t}", (HID,))]
    sh += [("Wo", (NF, HID)), ("bo", (NF,))]
    return sh


def param_count():
    return int(sum(np.prod(s) for _, s in param_shapes()))


def unpack(w):
    out, o = {}, 0
    for name, s in param_shapes():
        n = int(np.prod(s))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in param_shapes()])


def to_bf16(w):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(w, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# graph and features of one system
# ---------------------------------------------------------------------------
def _sym(S):
    """The symmetric matrix held by the lower triangle of S."""
    Lw = np.tril(S)
    return Lw + np.tril(S, -1).T


def graph(S, n):
    """Features, CSR adjacency (sorted neighbours), edge weights and the
    Cholesky factors of the diagonal blocks of one system."""
    A = _sym(np.asarray(S, dtype=np.float64)[:6 * n, :6 * n])
    B = [A[6 * i:6 * i + 6, 6 * i:6 * i + 6] for i in range(n)]
    logd = np.array([np.log(np.diag(b)) for b in B]).reshape(n, 6)
    x = np.zeros((n, NF))
    if n:
        x[:, :6] = logd - logd.mean(0)
    for i, b in enumerate(B):
        d = np.sqrt(np.diag(b))
        x[i, 6:] = [b[r, c] / (d[r] * d[c]) for r, c in STRICT]
    nb = np.array([np.linalg.norm(b) for b in B])
    ptr, adj, e = [0], [], []
    for i in range(n):
        for j in range(n):
            if j == i:
                continue
            blk = A[6 * i:6 * i + 6, 6 * j:6 * j + 6]
            if np.any(blk != 0.0):
                adj.append(j)
                e.append(np.linalg.norm(blk) / np.sqrt(nb[i] * nb[j]))
        ptr.append(len(adj))
    L = np.array([np.linalg.cholesky(b) for b in B]).reshape(n, 6, 6)
    return dict(x=x, ptr=np.array(ptr), adj=np.array(adj, dtype=np.int64), e=np.array(e), L=L, A=A)


# ---------------------------------------------------------------------------
# forward, head, loss and backward
# ---------------------------------------------------------------------------
def _aggregate(ptr, adj, e, h):
    m = np.zeros_like(h)
    for i in range(h.shape[0]):
        for a in range(ptr[i], ptr[i + 1]):
            m[i] += e[a] * h[adj[a]]
    return m


def forward(w, g):
    p = unpack(w)
    x = g["x"]
    h = [np.maximum(x @ p["W0"].T + p["b0"], 0.0)]
    m = []
    for t in range(1, LAYERS + 1):
        mt = _aggregate(g["ptr"], g["adj"], g["e"], h[-1])
        m.append(mt)
        h.append(np.maximum(h[-1] @ p[f"A{t}"].T + mt @ p[f"B{t}"].T + p[f"c{t}"], 0.0))
    C = h[-1] @ p["Wo"].T + p["bo"]
    return dict(h=h, m=m, C=C)


def lower(c):
    """21 packed values -> lower-triangular 6x6."""
    M = np.zeros((6, 6))
    for v, (r, cc) in zip(c, TRIL):
        M[r, cc] = v
    return M


def block_inverse(C_i, L_i):
    """P_i^-1 = G^T G, G = (I + E)^-1 L^-1, E = 0.5 tanh(C)."""
    M = np.eye(6) + lower(EPS * np.tanh(C_i))
    G = np.linalg.solve(M, np.linalg.inv(L_i))
    return G.T @ G


def preconditioner(w, g):
    f = forward(w, g)
    return np.array([block_inverse(f["C"][i], g["L"][i]) for i in range(g["x"].shape[0])])


def loss_and_grad(w, systems):
    """systems: list of (graph, z) with z of shape (n_probes, 6 n).
    Returns the loss and its gradient with respect to the flat parameters."""
    p = unpack(w)
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    num, den = 0.0, 0.0
    cache = []
    for g, z in systems:
        f = forward(w, g)
        n = g["x"].shape[0]
        U = z @ g["A"]                     # rows u^p = S z^p (S symmetric)
        dC = np.zeros((n, NF))
        for i in range(n):
            L = g["L"][i]
            th = np.tanh(f["C"][i])
            M = np.eye(6) + lower(EPS * th)
            Mbar = np.zeros((6, 6))
            for pz, pu in zip(z, U):
                zi, ui = pz[6 * i:6 * i + 6], pu[6 * i:6 * i + 6]
                a = np.linalg.solve(L, ui)
                y1 = np.linalg.solve(M, a)
                y2 = np.linalg.solve(M.T, y1)
                r = np.linalg.solve(L.T, y2) - zi
                num += r @ r
                # backward of r = L^-T M^-T M^-1 a - z (the 1/den scale is applied below)
                rb = 2.0 * r
                y2b = np.linalg.solve(L, rb)
                y1b = np.linalg.solve(M, y2b)
                Mbar -= np.outer(y2, y1b)
                ab = np.linalg.solve(M.T, y1b)
                Mbar -= np.outer(ab, y1)
            Ebar = np.array([Mbar[r, c] for r, c in TRIL])
            dC[i] = Ebar * EPS * (1.0 - th * th)
        den += float(np.sum(z * z))
        cache.append((g, f, dC))
    for g, f, dC in cache:
        h, m = f["h"], f["m"]
        grads["Wo"] += dC.T @ h[-1]
        grads["bo"] += dC.sum(0)
        dh = dC @ p["Wo"]
        for t in range(LAYERS, 0, -1):
            dz = dh * (h[t] > 0.0)
            grads[f"A{t}"] += dz.T @ h[t - 1]
            grads[f"B{t}"] += dz.T @ m[t - 1]
            grads[f"c{t}"] += dz.sum(0)
            dm = dz @ p[f"B{t}"]
            dh = dz @ p[f"A{t}"] + _aggregate(g["ptr"], g["adj"], g["e"], dm)  # e_ij = e_ji
        dz0 = dh * (h[0] > 0.0)
        grads["W0"] += dz0.T @ g["x"]
        grads["b0"] += dz0.sum(0)
    grad = pack(grads) / den
    return num / den, grad


def loss(w, systems):
    return loss_and_grad(w, systems)[0]
