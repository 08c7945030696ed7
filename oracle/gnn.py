"""FP64 oracle of the learned preconditioner for PCG on the reduced camera
system (RCS) of a sub-block.

TEST INFRASTRUCTURE ONLY: the tests load this module to check the CUDA
network kernels; nothing in the library package imports it.

The paper solves the RCS with conjugate gradients and block-Jacobi
preconditioning (Sec. 5.5: the inverses of the 6x6 camera blocks S_ii). This
network predicts a correction of each camera's block and a coupling gain for
every pair of cameras that share points, forming a factorised sparse
approximate inverse P^-1 = G^T G. Definitions, in the order they are applied:

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
  C_i  = Wo h3_i + bo                  (21 values: a lower-triangular 6x6, row by row)
  q_ij = ws . (h3_i + h3_j) + wp . (h3_i * h3_j) + we e_ij + bq   (every edge i > j)

Preconditioner. L_i = chol(B_i), M_i = I + 0.5 tanh(C_i) (lower triangular),
gamma_ij = tanh(q_ij), N_ij = gamma_ij L_i^-1 S_ij L_j^-T for i > j (the
normalised coupling), and
  G = M^-1 (I - N) L^-1      (block lower triangular, M, L block diagonal)
  P^-1 = G^T G.
P^-1 is SPD for every parameter value; with a zero output layer and zero
edge head it is block-Jacobi, blockdiag(B_i)^-1.

Loss (Kaporin's condition number of A = G S G^T, per unit of dimension d=6n,
less its constant log det S):
  l = log(tr(A) / d) - (1/d) log det A
    = log(tr(A) / d) + (2/d) sum_i (log det M_i + log det L_i) - (1/d) log det S
with tr(A) estimated from the probe vectors z^p (Hutchinson):
  tr(A) ~ (1/n_p) sum_p v_p^T S v_p,   v_p = G^T z_p.
The reported loss is l + (1/d) log det S averaged over the systems (the
constant dropped), so it equals log(T/d) + (2/d) sum_i log det(M_i L_i).
K >= 1 always; block-Jacobi minimises it among block-diagonal
preconditioners, so what the network gains comes from the coupling N.

Parameters are one flat vector in the order W0, b0, (A_t, B_t, c_t) for
t = 1..3, Wo, bo, ws, wp, we, bq; matrices row-major (out x in).
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
    sh += [("Wo", (NF, HID)), ("bo", (NF,)), ("ws", (HID,)), ("wp", (HID,)), ("we", (1,)), ("bq", (1,))]
    return sh


# parameters applied as matrices (BF16 in the CUDA kernels); the rest are biases
MATRICES = {"W0", "A1", "B1", "A2", "B2", "A3", "B3", "Wo"}


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
    return np.tril(S) + np.tril(S, -1).T


def graph(S, n):
    """Features, CSR adjacency (sorted neighbours), edge weights, the
    Cholesky factors of the diagonal blocks and the normalised couplings of
    one system."""
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
    L = np.array([np.linalg.cholesky(b) for b in B]).reshape(n, 6, 6)
    Li = np.array([np.linalg.inv(l) for l in L]).reshape(n, 6, 6)
    ptr, adj, e = [0], [], []
    lower = []                          # (i, j) with i > j, in CSR order of i
    Shat = []
    for i in range(n):
        for j in range(n):
            if j == i:
                continue
            blk = A[6 * i:6 * i + 6, 6 * j:6 * j + 6]
            if np.any(blk != 0.0):
                adj.append(j)
                e.append(np.linalg.norm(blk) / np.sqrt(nb[i] * nb[j]))
                if j < i:
                    lower.append((i, j, len(adj) - 1))
                    Shat.append(Li[i] @ blk @ Li[j].T)
        ptr.append(len(adj))
    return dict(x=x, ptr=np.array(ptr), adj=np.array(adj, dtype=np.int64), e=np.array(e), L=L, Li=Li, A=A,
                lower=lower, Shat=np.array(Shat).reshape(-1, 6, 6), n=n)


# ---------------------------------------------------------------------------
# forward
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
    hl = h[-1]
    q = np.array([p["ws"] @ (hl[i] + hl[j]) + p["wp"] @ (hl[i] * hl[j]) + p["we"][0] * g["e"][a] + p["bq"][0]
                  for i, j, a in g["lower"]])
    return dict(h=h, m=m, C=C, q=q)


def lower(c):
    """21 packed values -> lower-triangular 6x6."""
    M = np.zeros((6, 6))
    for v, (r, cc) in zip(c, TRIL):
        M[r, cc] = v
    return M


def factor(w, g, f=None):
    """Dense G = M^-1 (I - N) L^-1 of one system."""
    f = forward(w, g) if f is None else f
    n = g["n"]
    Mi = np.zeros((6 * n, 6 * n))
    Lb = np.zeros((6 * n, 6 * n))
    N = np.zeros((6 * n, 6 * n))
    for i in range(n):
        Mi[6 * i:6 * i + 6, 6 * i:6 * i + 6] = np.linalg.inv(np.eye(6) + lower(EPS * np.tanh(f["C"][i])))
        Lb[6 * i:6 * i + 6, 6 * i:6 * i + 6] = g["Li"][i]
    for k, (i, j, _) in enumerate(g["lower"]):
        N[6 * i:6 * i + 6, 6 * j:6 * j + 6] = np.tanh(f["q"][k]) * g["Shat"][k]
    return Mi @ (np.eye(6 * n) - N) @ Lb


def precondition(w, g, r):
    """P^-1 r = G^T G r for one system."""
    G = factor(w, g)
    return G.T @ (G @ r)


# ---------------------------------------------------------------------------
# loss and backward
# ---------------------------------------------------------------------------
def system_loss(w, g, z, f=None):
    f = forward(w, g) if f is None else f
    G = factor(w, g, f)
    d = 6 * g["n"]
    V = z @ G                                 # rows v_p^T = (G^T z_p)^T
    T = np.mean(np.einsum("pi,ij,pj->p", V, g["A"], V))
    ld = 0.0
    for i in range(g["n"]):
        M = np.eye(6) + lower(EPS * np.tanh(f["C"][i]))
        ld += np.sum(np.log(np.diag(M))) + np.sum(np.log(np.diag(g["L"][i])))
    return np.log(T / d) + 2.0 * ld / d


def loss(w, systems):
    return float(np.mean([system_loss(w, g, z) for g, z in systems]))


def loss_and_grad(w, systems):
    """systems: list of (graph, z), z of shape (n_probes, 6 n). Mean over the
    systems of the Kaporin loss, and its gradient with respect to the flat
    parameters."""
    p = unpack(w)
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    total = 0.0
    ns = len(systems)
    for g, z in systems:
        f = forward(w, g)
        n, d, npr = g["n"], 6 * g["n"], z.shape[0]
        Mb = [np.eye(6) + lower(EPS * np.tanh(f["C"][i])) for i in range(n)]
        gam = np.tanh(f["q"])
        Nk = [gam[k] * g["Shat"][k] for k in range(len(g["lower"]))]
        # forward per probe: t = M^-T z, s = (I - N)^T t, v = L^-T s, u = S v
        T = 0.0
        cache = []
        for zp in z:
            t = np.concatenate([np.linalg.solve(Mb[i].T, zp[6 * i:6 * i + 6]) for i in range(n)])
            s = t.copy()
            for k, (i, j, _) in enumerate(g["lower"]):
                s[6 * j:6 * j + 6] -= Nk[k].T @ t[6 * i:6 * i + 6]
            v = np.concatenate([np.linalg.solve(g["L"][i].T, s[6 * i:6 * i + 6]) for i in range(n)])
            u = g["A"] @ v
            T += v @ u / npr
            cache.append((t, s, v, u))
        ld = sum(np.sum(np.log(np.diag(Mb[i]))) + np.sum(np.log(np.diag(g["L"][i]))) for i in range(n))
        total += (np.log(T / d) + 2.0 * ld / d) / ns
        # backward
        Mbar = [np.zeros((6, 6)) for _ in range(n)]
        gbar = np.zeros(len(g["lower"]))
        for t, s, v, u in cache:
            vb = (2.0 / (npr * T)) * u / ns
            sb = np.concatenate([np.linalg.solve(g["L"][i], vb[6 * i:6 * i + 6]) for i in range(n)])
            tb = sb.copy()
            for k, (i, j, _) in enumerate(g["lower"]):
                tb[6 * i:6 * i + 6] -= Nk[k] @ sb[6 * j:6 * j + 6]
                gbar[k] -= t[6 * i:6 * i + 6] @ g["Shat"][k] @ sb[6 * j:6 * j + 6]
            for i in range(n):
                ti, tbi = t[6 * i:6 * i + 6], tb[6 * i:6 * i + 6]
                Mbar[i] -= np.outer(ti, np.linalg.solve(Mb[i], tbi))
        dC = np.zeros((n, NF))
        for i in range(n):
            Mbar[i] += np.diag(2.0 / (d * ns) / np.diag(Mb[i]))
            th = np.tanh(f["C"][i])
            dC[i] = np.array([Mbar[i][r, c] for r, c in TRIL]) * EPS * (1.0 - th * th)
        qb = gbar * (1.0 - gam * gam)
        # edge head
        h, m = f["h"], f["m"]
        hl = h[-1]
        dh = dC @ p["Wo"]
        grads["Wo"] += dC.T @ hl
        grads["bo"] += dC.sum(0)
        for k, (i, j, a) in enumerate(g["lower"]):
            grads["ws"] += qb[k] * (hl[i] + hl[j])
            grads["wp"] += qb[k] * hl[i] * hl[j]
            grads["we"][0] += qb[k] * g["e"][a]
            grads["bq"][0] += qb[k]
            dh[i] += qb[k] * (p["ws"] + p["wp"] * hl[j])
            dh[j] += qb[k] * (p["ws"] + p["wp"] * hl[i])
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
    return total, pack(grads)
