"""Pins of the FP64 oracle of the learned preconditioner (oracle/gnn.py) to
facts it does not compute itself: central finite differences, the
block-Jacobi special case written densely, Kaporin's number from dense trace
and determinant (>= 1 by AM-GM, = 1 for a block-diagonal system), the block
structure and definiteness of the factor, feature equivariance, and bfloat16
rounding."""

import numpy as np
import pytest

from oracle import gnn
from paper_1910_08138_gb300 import synth


def _systems(seed=1, sizes=(8, 5), n_probes=3):
    return [(gnn.graph(S, S.shape[0] // 6), z) for S, z in synth.rcs_like_systems(seed, sizes=sizes, n_probes=n_probes)]


def _weights(seed=0, scale=0.1):
    return np.random.default_rng(seed).normal(size=gnn.param_count()) * scale


def test_param_layout():
    assert gnn.param_count() == 64 * 21 + 64 + 3 * (2 * 64 * 64 + 64) + 21 * 64 + 21 + 64 + 64 + 1 + 1
    w = _weights()
    np.testing.assert_array_equal(gnn.pack(gnn.unpack(w)), w)


def test_gradient_matches_central_differences():
    gs = _systems()
    w = _weights()
    _, grad = gnn.loss_and_grad(w, gs)
    rng = np.random.default_rng(3)
    # some entries of every parameter group
    idx, o = [], 0
    for _, s in gnn.param_shapes():
        n = int(np.prod(s))
        idx += list(o + rng.choice(n, min(n, 3), replace=False))
        o += n
    checked = 0
    for i in idx:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (gnn.loss(wp, gs) - gnn.loss(wm, gs)) / (2 * h)
        if abs(fd) < 1e-9 and abs(grad[i]) < 1e-9:
            continue  # a ReLU that is off for every node
        assert abs(grad[i] - fd) <= 2e-5 * max(abs(fd), 1e-3), (i, grad[i], fd)
        checked += 1
    assert checked >= 15


def _zero_heads(w):
    p = gnn.unpack(w)
    for k in ("Wo", "bo", "ws", "wp", "we", "bq"):
        p[k][:] = 0.0
    return gnn.pack(p)


def _exact_probes(n):
    """sqrt(d) e_p for p = 1..d: the trace estimate is then exact."""
    d = 6 * n
    return np.sqrt(d) * np.eye(d)


def test_zero_heads_are_block_jacobi():
    (S, _), = synth.rcs_like_systems(4, sizes=(9,), n_probes=1)
    g = gnn.graph(S, 9)
    w = _zero_heads(_weights())
    A = np.tril(S) + np.tril(S, -1).T
    D = np.zeros_like(A)
    for i in range(9):
        D[6 * i:6 * i + 6, 6 * i:6 * i + 6] = np.linalg.inv(A[6 * i:6 * i + 6, 6 * i:6 * i + 6])
    r = np.random.default_rng(1).normal(size=54)
    np.testing.assert_allclose(gnn.precondition(w, g, r), D @ r, rtol=1e-9)
    # the loss is Kaporin's number of D^-1/2 S D^-1/2 per dimension, plus log det S / d
    z = _exact_probes(9)
    K = D @ A
    want = np.log(np.trace(K) / 54) - np.linalg.slogdet(K)[1] / 54 + np.linalg.slogdet(A)[1] / 54
    assert gnn.loss(w, [(g, z)]) == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_kaporin_number_is_at_least_one_and_exact_with_exact_probes():
    (S, _), = synth.rcs_like_systems(6, sizes=(7,), n_probes=1)
    g = gnn.graph(S, 7)
    A = np.tril(S) + np.tril(S, -1).T
    z = _exact_probes(7)
    base = np.linalg.slogdet(A)[1] / 42
    for seed in range(4):
        w = _weights(seed, 0.3)
        G = gnn.factor(w, g)
        M = G @ A @ G.T
        want = np.log(np.trace(M) / 42) - np.linalg.slogdet(M)[1] / 42
        got = gnn.loss(w, [(g, z)]) - base
        assert got == pytest.approx(want, rel=1e-9, abs=1e-12)
        assert got >= -1e-12  # AM-GM on the eigenvalues of G S G^T


def test_preconditioner_is_spd_and_block_lower_factor():
    (S, _), = synth.rcs_like_systems(7, sizes=(8,), n_probes=1)
    g = gnn.graph(S, 8)
    w = _weights(5, 0.3)
    G = gnn.factor(w, g)
    # block lower triangular, non-zero only on the diagonal and the camera graph
    for i in range(8):
        for j in range(i + 1, 8):
            assert not np.any(G[6 * i:6 * i + 6, 6 * j:6 * j + 6])
    Pinv = G.T @ G
    assert np.all(np.linalg.eigvalsh(0.5 * (Pinv + Pinv.T)) > 0)
    r = np.random.default_rng(2).normal(size=48)
    np.testing.assert_allclose(gnn.precondition(w, g, r), Pinv @ r, rtol=1e-10)


def test_feature_permutation_equivariance_and_ranges():
    (S, _), = synth.rcs_like_systems(5, sizes=(10,), n_probes=1)
    n = 10
    perm = np.random.default_rng(2).permutation(n)
    idx = np.concatenate([np.arange(6 * c, 6 * c + 6) for c in perm])
    A = np.tril(S) + np.tril(S, -1).T
    Sp = A[np.ix_(idx, idx)]
    g, gp = gnn.graph(S, n), gnn.graph(Sp, n)
    np.testing.assert_allclose(gp["x"], g["x"][perm], atol=1e-12)
    assert np.all(np.abs(g["x"][:, 6:]) <= 1.0)
    np.testing.assert_allclose(g["x"][:, :6].sum(0), 0.0, atol=1e-10)
    # the edge weights are symmetric
    e = {(i, int(g["adj"][a])): g["e"][a] for i in range(n) for a in range(g["ptr"][i], g["ptr"][i + 1])}
    for (i, j), v in e.items():
        assert e[(j, i)] == pytest.approx(v, rel=1e-14)
    # normalised couplings: L_i^-1 S_ij L_j^-T
    for k, (i, j, _) in enumerate(g["lower"]):
        blk = A[6 * i:6 * i + 6, 6 * j:6 * j + 6]
        np.testing.assert_allclose(np.linalg.cholesky(A[6 * i:6 * i + 6, 6 * i:6 * i + 6]) @ g["Shat"][k]
                                   @ np.linalg.cholesky(A[6 * j:6 * j + 6, 6 * j:6 * j + 6]).T, blk,
                                   rtol=1e-10, atol=1e-12 * np.abs(blk).max())


def test_block_diagonal_system_has_no_edges_and_unit_kaporin_number():
    rng = np.random.default_rng(11)
    n = 4
    S = np.zeros((24, 24))
    for i in range(n):
        X = rng.normal(size=(6, 6))
        S[6 * i:6 * i + 6, 6 * i:6 * i + 6] = X @ X.T + np.eye(6)
    g = gnn.graph(S, n)
    assert g["adj"].size == 0
    w = _zero_heads(_weights())
    got = gnn.loss(w, [(g, _exact_probes(n))]) - np.linalg.slogdet(S)[1] / 24
    assert got == pytest.approx(0.0, abs=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8])
    np.testing.assert_array_equal(gnn.to_bf16(v), [1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6])
