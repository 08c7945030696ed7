"""Pins of the FP64 oracle of the learned block preconditioner (oracle/gnn.py)
to facts it does not compute itself: central finite differences, the
block-Jacobi special case written densely, the SPD construction of P_i from
its definition, permutation equivariance, and bfloat16 rounding."""

import numpy as np
import pytest

from oracle import gnn
from paper_1910_08138_gb300 import synth


def _systems(seed=1, sizes=(8, 5), n_probes=3):
    return [(gnn.graph(S, S.shape[0] // 6), z) for S, z in synth.rcs_like_systems(seed, sizes=sizes, n_probes=n_probes)]


def _weights(seed=0, scale=0.1):
    return np.random.default_rng(seed).normal(size=gnn.param_count()) * scale


def test_param_layout():
    assert gnn.param_count() == 64 * 21 + 64 + 3 * (2 * 64 * 64 + 64) + 21 * 64 + 21
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
        assert abs(grad[i] - fd) <= 1e-6 * max(abs(fd), 1e-3), (i, grad[i], fd)
        checked += 1
    assert checked >= 15


def test_zero_output_layer_is_block_jacobi():
    (S, z), = synth.rcs_like_systems(4, sizes=(9,), n_probes=2)
    g = gnn.graph(S, 9)
    w = _weights()
    p = gnn.unpack(w)
    p["Wo"][:] = 0.0
    p["bo"][:] = 0.0
    w = gnn.pack(p)
    Pinv = gnn.preconditioner(w, g)
    A = np.tril(S) + np.tril(S, -1).T
    D = np.zeros_like(A)
    for i in range(9):
        blk = A[6 * i:6 * i + 6, 6 * i:6 * i + 6]
        np.testing.assert_allclose(Pinv[i], np.linalg.inv(blk), rtol=1e-9, atol=1e-12 * np.abs(np.linalg.inv(blk)).max())
        D[6 * i:6 * i + 6, 6 * i:6 * i + 6] = np.linalg.inv(blk)
    R = (D @ A - np.eye(54)) @ z.T
    assert gnn.loss(w, [(g, z)]) == pytest.approx(np.sum(R * R) / np.sum(z * z), rel=1e-10)


def test_block_inverse_is_the_inverse_of_the_spd_definition():
    rng = np.random.default_rng(7)
    for _ in range(5):
        X = rng.normal(size=(6, 6))
        B = X @ X.T + 6 * np.eye(6)
        L = np.linalg.cholesky(B)
        C = rng.normal(size=21) * 3.0
        E = np.zeros((6, 6))
        k = 0
        for r in range(6):
            for c in range(r + 1):
                E[r, c] = 0.5 * np.tanh(C[k])
                k += 1
        P = L @ (np.eye(6) + E) @ (np.eye(6) + E).T @ L.T
        assert np.all(np.linalg.eigvalsh(P) > 0)
        np.testing.assert_allclose(gnn.block_inverse(C, L) @ P, np.eye(6), atol=1e-9)


def test_permutation_equivariance_and_feature_ranges():
    (S, _), = synth.rcs_like_systems(5, sizes=(10,), n_probes=1)
    n = 10
    perm = np.random.default_rng(2).permutation(n)
    idx = np.concatenate([np.arange(6 * c, 6 * c + 6) for c in perm])
    A = np.tril(S) + np.tril(S, -1).T
    Sp = A[np.ix_(idx, idx)]
    w = _weights(9, 0.2)
    g, gp = gnn.graph(S, n), gnn.graph(Sp, n)
    np.testing.assert_allclose(gp["x"], g["x"][perm], atol=1e-12)
    np.testing.assert_allclose(gnn.preconditioner(w, gp), gnn.preconditioner(w, g)[perm], rtol=1e-9, atol=1e-15)
    assert np.all(np.abs(g["x"][:, 6:]) <= 1.0)
    np.testing.assert_allclose(g["x"][:, :6].sum(0), 0.0, atol=1e-10)
    # the edge weights are symmetric
    e = {(i, int(g["adj"][a])): g["e"][a] for i in range(n) for a in range(g["ptr"][i], g["ptr"][i + 1])}
    for (i, j), v in e.items():
        assert e[(j, i)] == pytest.approx(v, rel=1e-14)


def test_block_diagonal_system_has_no_edges_and_zero_loss_at_block_jacobi():
    rng = np.random.default_rng(11)
    n = 4
    S = np.zeros((24, 24))
    for i in range(n):
        X = rng.normal(size=(6, 6))
        S[6 * i:6 * i + 6, 6 * i:6 * i + 6] = X @ X.T + np.eye(6)
    g = gnn.graph(S, n)
    assert g["adj"].size == 0
    p = gnn.unpack(_weights())
    p["Wo"][:] = 0.0
    p["bo"][:] = 0.0
    z = rng.normal(size=(2, 24))
    assert gnn.loss(gnn.pack(p), [(g, z)]) == pytest.approx(0.0, abs=1e-20)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8])
    np.testing.assert_array_equal(gnn.to_bf16(v), [1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6])
