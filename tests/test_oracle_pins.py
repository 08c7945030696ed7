"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks one part of the oracle against geometry, a library routine,
a brute-force dense computation, an invariant or a statistical property, so
that a dropped term, a wrong sign or index or a transposed operand in the
oracle fails at least one of them. No GPU is used.
"""

import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import norm

import oracle
from paper_1910_08138_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers (numpy, independent of the oracle's arithmetic)
# --------------------------------------------------------------------------
def pose_R(pose):
    return Rotation.from_rotvec(pose[:3]).as_matrix()


def camera_centres(poses):
    R = Rotation.from_rotvec(poses[:, :3]).as_matrix()
    return -np.einsum("mba,mb->ma", R, poses[:, 3:])


def umeyama(src, dst):
    """Similarity (s, R, t) with dst ~ s R src + t (least squares)."""
    mu_s, mu_d = src.mean(0), dst.mean(0)
    a, b = src - mu_s, dst - mu_d
    U, D, Vt = np.linalg.svd(b.T @ a / len(src))
    S = np.eye(3)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        S[2, 2] = -1
    R = U @ S @ Vt
    s = np.trace(np.diag(D) @ S) / (a ** 2).sum(1).mean()
    return s, R, mu_d - s * R @ mu_s


def fd_jacobian(R, t, intr, X, h=1e-6):
    """Central differences of the oracle projection w.r.t. (dw left, dt) and X."""
    Jc = np.zeros((2, 6))
    Jx = np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3); e[a] = h
        up = oracle.project(Rotation.from_rotvec(e).as_matrix() @ R, t, intr, X)[0]
        um = oracle.project(Rotation.from_rotvec(-e).as_matrix() @ R, t, intr, X)[0]
        Jc[:, a] = (up - um) / (2 * h)
        up = oracle.project(R, t + e, intr, X)[0]
        um = oracle.project(R, t - e, intr, X)[0]
        Jc[:, 3 + a] = (up - um) / (2 * h)
        up = oracle.project(R, t, intr, X + e)[0]
        um = oracle.project(R, t, intr, X - e)[0]
        Jx[:, a] = (up - um) / (2 * h)
    return Jc, Jx


def sym6_full(s):
    return np.array([[s[0], s[1], s[2]], [s[1], s[3], s[4]], [s[2], s[4], s[5]]])


def winv_full(w):
    return np.array([[w[0], w[1]], [w[1], w[2]]])


def with_weights(prob, seed=3):
    """Random SPD 2x2 weights C^-1 per observation."""
    rng = np.random.default_rng(seed)
    K = prob["obs_cam"].size
    a = rng.uniform(0.5, 2.0, K)
    c = rng.uniform(0.5, 2.0, K)
    b = rng.uniform(-0.4, 0.4, K) * np.sqrt(a * c)
    p = dict(prob)
    p["obs_winv"] = np.stack([a, b, c], axis=1)
    return p


def dense_subblock_system(o, prob, l, lam, jac="analytic"):
    """Dense N + lam diag(N) and g = J^T W v of sub-block l at the oracle state.

    Unknowns: the cameras of l (6 each, oracle row order) then the instances
    of l (3 each, canonical order). Includes the TP control term of Eq. bact.
    """
    cams = o.sub_cameras(l)
    cam_pos = {int(c): n for n, c in enumerate(cams)}
    ip, isub = o.instances()
    inst = np.nonzero(isub == l)[0]
    inst_pos = {int(q): n for n, q in enumerate(inst)}
    inst_of = {(int(ip[q]), int(isub[q])): int(q) for q in range(o.P)}
    poses = o.cameras()
    X, act = o.points()
    Xl, Wl = o.instance_state()
    w = o.weights()
    winv = prob.get("obs_winv")
    nC, nX = 6 * len(cams), 3 * len(inst)
    n = nC + nX
    Nm = np.zeros((n, n))
    g = np.zeros(n)
    sub_of_cam = prob["cam_subblock"]
    for k in range(prob["obs_cam"].size):
        i, j = int(prob["obs_cam"][k]), int(prob["obs_point"][k])
        if sub_of_cam[i] != l or not act[j]:
            continue
        q = inst_of[(j, l)]
        R = pose_R(poses[i])
        uv, Jc, Jx, _ = oracle.project(R, poses[i, 3:], prob["cam_intr"][i], Xl[q])
        if jac == "fd":
            Jc, Jx = fd_jacobian(R, poses[i, 3:], prob["cam_intr"][i], Xl[q])
        v = uv - prob["obs_xy"][k]
        W = w[k] * (np.eye(2) if winv is None else winv_full(winv[k]))
        J = np.zeros((2, n))
        J[:, 6 * cam_pos[i]:6 * cam_pos[i] + 6] = Jc
        J[:, nC + 3 * inst_pos[q]:nC + 3 * inst_pos[q] + 3] = Jx
        Nm += J.T @ W @ J
        g += J.T @ W @ v
    for q in inst:
        j = int(ip[q])
        if not act[j]:
            continue
        a = nC + 3 * inst_pos[int(q)]
        Wq = sym6_full(Wl[q])
        Nm[a:a + 3, a:a + 3] += Wq
        g[a:a + 3] += Wq @ (Xl[q] - X[j])
    # inactive points: identity rows keep the dense system regular
    for q in inst:
        if not act[int(ip[q])]:
            a = nC + 3 * inst_pos[int(q)]
            Nm[a:a + 3, a:a + 3] = np.eye(3)
    Na = Nm + lam * np.diag(np.diag(Nm))
    return Na, g, nC


def sub_cost_numpy(o, prob, l, poses, Xl):
    """F_l (Eq. bact): sum w v^T W v over obs of l + TP terms, at given state."""
    X, act = o.points()
    _, Wl = o.instance_state()
    ip, isub = o.instances()
    inst_of = {(int(ip[q]), int(isub[q])): int(q) for q in range(o.P)}
    w = o.weights()
    winv = prob.get("obs_winv")
    F = 0.0
    for k in range(prob["obs_cam"].size):
        i, j = int(prob["obs_cam"][k]), int(prob["obs_point"][k])
        if prob["cam_subblock"][i] != l or not act[j]:
            continue
        q = inst_of[(j, l)]
        uv, _, _, _ = oracle.project(pose_R(poses[i]), poses[i, 3:], prob["cam_intr"][i], Xl[q])
        v = uv - prob["obs_xy"][k]
        W = np.eye(2) if winv is None else winv_full(winv[k])
        F += w[k] * v @ W @ v
    for q in np.nonzero(isub == l)[0]:
        j = int(ip[q])
        if act[j]:
            d = Xl[q] - X[j]
            F += d @ sym6_full(Wl[q]) @ d
    return F


# --------------------------------------------------------------------------
# rotations
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 1e-3, 0.3, 2.0, 3.1])
def test_rodrigues_matches_scipy(scale):
    rng = np.random.default_rng(1)
    for _ in range(20):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        np.testing.assert_allclose(oracle.rodrigues(w), Rotation.from_rotvec(w).as_matrix(),
                                   rtol=0, atol=1e-14)


def test_rotation_log_roundtrip():
    rng = np.random.default_rng(2)
    for scale in (1e-8, 1e-3, 0.5, 2.5, np.pi - 1e-2, np.pi - 2.5e-4, np.pi - 1e-7, np.pi - 1e-3):
        for _ in range(10):
            a = rng.normal(size=3)
            w = a / np.linalg.norm(a) * scale
            R = Rotation.from_rotvec(w).as_matrix()
            w2 = oracle.rotation_log(R)
            # exact to rounding, also near 180 degrees (nadir cameras are ~pi rotations)
            np.testing.assert_allclose(Rotation.from_rotvec(w2).as_matrix(), R, atol=2e-15)
            np.testing.assert_allclose(w2, Rotation.from_matrix(R).as_rotvec(), atol=1e-6)


# --------------------------------------------------------------------------
# projection and Jacobians (Sec. 2, Eq. ta)
# --------------------------------------------------------------------------
def _attitude(name):
    nadir_c2w = np.diag([1.0, -1.0, -1.0])
    if name == "nadir":
        return nadir_c2w
    if name == "oblique-north-30":
        q = Rotation.from_rotvec(np.deg2rad(30.0) * np.array([1.0, 0.0, 0.0])).as_matrix()
        return q @ nadir_c2w
    raise ValueError(name)


def test_projection_golden_cases():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "projection_cases.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 5
    for r in rows:
        c2w = _attitude(r[0])
        C = np.array(list(map(float, r[1:4])))
        X = np.array(list(map(float, r[4:7])))
        uv_exp = np.array(list(map(float, r[7:9])))
        R = c2w.T
        t = -R @ C
        uv, _, _, z = oracle.project(R, t, [1000.0, 1000.0, 750.0], X)
        assert z > 0
        np.testing.assert_allclose(uv, uv_exp, atol=1e-9)


def test_projection_behind_camera_has_negative_depth():
    R = np.diag([1.0, -1.0, -1.0])
    t = -R @ np.array([0.0, 0.0, 30.0])
    _, _, _, z = oracle.project(R, t, [1000.0, 1000.0, 750.0], [0.0, 0.0, 40.0])
    assert z < 0


def test_jacobians_match_finite_differences():
    rng = np.random.default_rng(4)
    for _ in range(50):
        R = Rotation.from_rotvec(rng.normal(size=3) * 0.8).as_matrix()
        X = rng.uniform(-5, 5, 3)
        t = -R @ X + np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(10, 40)])
        t = t  # camera sees X in front: X_c = R X + t has z in [10, 40]
        intr = [rng.uniform(500, 1500), 1000.0, 750.0]
        Xp = X + rng.normal(size=3)
        _, Jc, Jx, z = oracle.project(R, t, intr, Xp)
        assert z > 0
        Jc_fd, Jx_fd = fd_jacobian(R, t, intr, Xp)
        np.testing.assert_allclose(Jc, Jc_fd, rtol=1e-6, atol=1e-6 * np.abs(Jc_fd).max())
        np.testing.assert_allclose(Jx, Jx_fd, rtol=1e-6, atol=1e-6 * np.abs(Jx_fd).max())


def test_residuals_and_jacobian_arrays_are_per_observation():
    prob = synth.tiny(seed=5)
    o = oracle.Oracle(prob)
    v = o.residuals()
    Jc, Jx = o.jacobians()
    X, _ = o.points()
    for k in range(0, prob["obs_cam"].size, 7):
        i, j = prob["obs_cam"][k], prob["obs_point"][k]
        R = Rotation.from_rotvec(prob["cam_pose"][i, :3]).as_matrix()
        uv, jc, jx, _ = oracle.project(R, prob["cam_pose"][i, 3:], prob["cam_intr"][i], X[j])
        np.testing.assert_allclose(v[k], uv - prob["obs_xy"][k], atol=1e-9)
        np.testing.assert_allclose(Jc[k], jc, atol=1e-9)
        np.testing.assert_allclose(Jx[k], jx, atol=1e-12)


# --------------------------------------------------------------------------
# normal equations, Schur complement, LM step (Sec. 2, Sec. 5.5, Eq. bact)
# --------------------------------------------------------------------------
def _tiny_state(seed=11, runs=(3, 3), weights=True):
    prob = synth.tiny(seed=seed, nx=3, ny=2, n_points=30, opp=4, runs=list(runs))
    if weights:
        prob = with_weights(prob, seed)
    o = oracle.Oracle(prob)
    o.intersect()
    rng = np.random.default_rng(seed)
    w = np.where(rng.random(o.K) < 0.1, 1e-4, 1.0)
    o.set_weights(w)
    Xl, Wl = o.instance_state()
    o.set_instance_state(Xl + rng.normal(0, 0.05, Xl.shape), Wl)
    return prob, o


@pytest.mark.parametrize("lam", [0.0, 1e-4, 1e-2])
def test_rcs_equals_dense_schur_complement(lam):
    prob, o = _tiny_state()
    for l in range(o.L):
        Na, g, nC = dense_subblock_system(o, prob, l, lam)
        Ncc, Ncx, Nxx = Na[:nC, :nC], Na[:nC, nC:], Na[nC:, nC:]
        S_dense = Ncc - Ncx @ np.linalg.solve(Nxx, Ncx.T)
        y_dense = -g[:nC] + Ncx @ np.linalg.solve(Nxx, g[nC:])
        S, y = o.rcs(l, lam)
        scale = np.abs(S_dense).max()
        np.testing.assert_allclose(S, S_dense, atol=1e-10 * scale, rtol=0)
        np.testing.assert_allclose(y, y_dense, atol=1e-10 * np.abs(y_dense).max(), rtol=0)
        np.testing.assert_allclose(S, S.T, atol=1e-12 * scale)


def test_rcs_with_finite_difference_jacobians():
    prob, o = _tiny_state(seed=12)
    lam = 1e-4
    for l in range(o.L):
        Na, g, nC = dense_subblock_system(o, prob, l, lam, jac="fd")
        Ncc, Ncx, Nxx = Na[:nC, :nC], Na[:nC, nC:], Na[nC:, nC:]
        S_dense = Ncc - Ncx @ np.linalg.solve(Nxx, Ncx.T)
        S, _ = o.rcs(l, lam)
        np.testing.assert_allclose(S, S_dense, atol=2e-5 * np.abs(S_dense).max(), rtol=0)


@pytest.mark.parametrize("runs", [(3, 3), (6,), (2, 2, 2)])
def test_lm_step_equals_dense_solve_and_cost(runs):
    prob, o = _tiny_state(seed=13, runs=runs)
    lam = 1e-4
    for l in range(o.L):
        Na, g, nC = dense_subblock_system(o, prob, l, lam)
        delta = np.linalg.solve(Na, -g)
        poses0 = o.cameras()
        Xl0, _ = o.instance_state()
        F0 = sub_cost_numpy(o, prob, l, poses0, Xl0)
        r, Fb, Ft, dc, dx = o.lm_step(l, lam)
        assert r in (0, 1)
        np.testing.assert_allclose(Fb, F0, rtol=1e-9)
        np.testing.assert_allclose(dc, delta[:nC], atol=1e-9 * np.abs(delta).max() + 1e-12)
        np.testing.assert_allclose(dx.reshape(-1), delta[nC:],
                                   atol=1e-9 * np.abs(delta).max() + 1e-12)
        # trial state and its cost, independently
        cams = o.sub_cameras(l)
        poses_t = poses0.copy()
        for n, i in enumerate(cams):
            Rt = Rotation.from_rotvec(dc[6 * n:6 * n + 3]).as_matrix() @ pose_R(poses0[i])
            poses_t[i, :3] = Rotation.from_matrix(Rt).as_rotvec()
            poses_t[i, 3:] = poses0[i, 3:] + dc[6 * n + 3:6 * n + 6]
        _, isub = o.instances()
        Xl_t = Xl0.copy()
        Xl_t[isub == l] += dx
        Ft_np = sub_cost_numpy(o, prob, l, poses_t, Xl_t)
        np.testing.assert_allclose(Ft, Ft_np, rtol=1e-9)
        assert (r == 1) == (Ft_np < F0)
        if r == 1:
            np.testing.assert_allclose(o.cameras()[cams], poses_t[cams], atol=1e-10)
            np.testing.assert_allclose(o.instance_state()[0], Xl_t, atol=1e-12)


def test_lm_loop_decreases_cost_monotonically():
    prob, o = _tiny_state(seed=14, runs=(6,))
    F_prev = o.sub_cost(0)
    for _ in range(6):
        r, Fb, Ft, _, _ = o.lm_step(0, 1e-4)
        assert Fb == pytest.approx(F_prev, rel=1e-12)
        F_prev = Ft if r == 1 else Fb
        assert o.sub_cost(0) == pytest.approx(F_prev, rel=1e-12)


# --------------------------------------------------------------------------
# intersection, covariance, refined weights (Eq. bars, Sec. 5.1)
# --------------------------------------------------------------------------
def test_intersection_noise_free_two_cameras_is_exact():
    """Two views, no noise: the adjusted point equals linear (DLT) triangulation."""
    rng = np.random.default_rng(21)
    for trial in range(10):
        C1, C2 = np.array([0.0, 0.0, 30.0]), np.array([6.0, 1.0, 31.0])
        c2w = np.diag([1.0, -1.0, -1.0])
        Rs = [c2w.T, (Rotation.from_rotvec([0.05, -0.1, 0.02]).as_matrix() @ c2w).T]
        ts = [-Rs[0] @ C1, -Rs[1] @ C2]
        Xt = np.array([rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-2, 2)])
        intr = np.array([[1000.0, 1000.0, 750.0]] * 2)
        xy = np.array([oracle.project(Rs[a], ts[a], intr[a], Xt)[0] for a in range(2)])
        # DLT from the 3x4 projection matrices
        A = []
        for a in range(2):
            Kmat = np.array([[1000.0, 0, 1000.0], [0, 1000.0, 750.0], [0, 0, 1]])
            P = Kmat @ np.hstack([Rs[a], ts[a][:, None]])
            A.append(xy[a, 0] * P[2] - P[0])
            A.append(xy[a, 1] * P[2] - P[1])
        Xh = np.linalg.svd(np.array(A))[2][-1]
        X_dlt = Xh[:3] / Xh[3]
        prob = dict(cam_pose=np.array([np.r_[Rotation.from_matrix(Rs[a]).as_rotvec(), ts[a]] for a in range(2)]),
                    cam_intr=intr, points=(Xt + rng.normal(0, 0.3, 3))[None, :],
                    obs_cam=np.array([0, 1], np.int32), obs_point=np.array([0, 0], np.int32),
                    obs_xy=xy, obs_winv=None, cam_subblock=np.array([0, 1], np.int32))
        o = oracle.Oracle(prob)
        assert o.intersect() == 0
        X, act = o.points()
        assert act[0] == 1
        np.testing.assert_allclose(X[0], X_dlt, atol=1e-7)
        np.testing.assert_allclose(X[0], Xt, atol=1e-7)


def test_covariance_is_inverse_normal_matrix_and_refined_weights():
    prob = with_weights(synth.tiny(seed=22, runs=[2, 2, 2]), 22)
    o = oracle.Oracle(prob)
    o.intersect()
    X, act = o.points()
    _, Wl = o.instance_state()
    ip, isub = o.instances()
    poses = o.cameras()
    winv = prob["obs_winv"]
    ids = np.nonzero(act)[0]
    Cov = o.covariance(ids)
    for a, j in enumerate(ids):
        N = np.zeros((3, 3))
        Nsub = {}
        grad = np.zeros(3)
        for k in np.nonzero(prob["obs_point"] == j)[0]:
            i = prob["obs_cam"][k]
            R = pose_R(poses[i])
            uv = oracle.project(R, poses[i, 3:], prob["cam_intr"][i], X[j])[0]
            _, Jx = fd_jacobian(R, poses[i, 3:], prob["cam_intr"][i], X[j])
            part = Jx.T @ winv_full(winv[k]) @ Jx
            N += part
            grad += Jx.T @ winv_full(winv[k]) @ (uv - prob["obs_xy"][k])
            lsub = prob["cam_subblock"][i]
            Nsub[lsub] = Nsub.get(lsub, 0) + part
        # C_j N_j = I
        np.testing.assert_allclose(Cov[a] @ N, np.eye(3), atol=1e-6)
        # the adjusted point is stationary: J^T W v = 0
        assert np.abs(grad).max() < 1e-6 * np.abs(N).max()
        # W^l = N_j - N_j^(l) for every instance, zero for a single-instance point;
        # W^l comes from the last Gauss-Newton iteration, before its final step
        # (< 1e-3 px in the image), so it matches N at the final X to ~1e-5
        for q in np.nonzero(ip == j)[0]:
            Wexp = N - Nsub[isub[q]] if len(Nsub) >= 2 else np.zeros((3, 3))
            np.testing.assert_allclose(sym6_full(Wl[q]), Wexp, atol=2e-5 * np.abs(N).max())
            # invariant W^l + N^(l) = N
            if len(Nsub) >= 2:
                np.testing.assert_allclose(sym6_full(Wl[q]) + Nsub[isub[q]], N,
                                           atol=2e-5 * np.abs(N).max())


def test_intersection_drops_point_behind_camera():
    prob = synth.tiny(seed=23, runs=[3, 3])
    X = prob["points"].copy()
    X[0] = [0.0, 0.0, 60.0]  # above the 30 m cameras: behind all of them
    prob["points"] = X
    o = oracle.Oracle(prob)
    dropped = o.intersect()
    _, act = o.points()
    assert act[0] == 0 and dropped >= 1


# --------------------------------------------------------------------------
# robust scale (Sec. 5.3) and sigma_0 (Eq. sigma0)
# --------------------------------------------------------------------------
def test_median_even_and_odd():
    rng = np.random.default_rng(31)
    for n in (1, 2, 3, 10, 11, 1000, 1001):
        a = rng.normal(size=n)
        assert oracle.median(a) == pytest.approx(float(np.median(a)), abs=0)


def test_mad_factor_and_gaussian_scale():
    # 1.4826 is 1 / Phi^-1(3/4), the MAD-to-sigma factor of a normal distribution
    assert 1.0 / norm.ppf(0.75) == pytest.approx(1.4826, abs=5e-5)
    # one camera observing many points with known Gaussian pixel noise
    rng = np.random.default_rng(32)
    n = 20000
    sigma = 0.7
    R = np.diag([1.0, -1.0, -1.0])
    t = -R @ np.array([0.0, 0.0, 30.0])
    X = np.stack([rng.uniform(-20, 20, n), rng.uniform(-15, 15, n), np.zeros(n)], 1)
    uv = np.array([oracle.project(R, t, [1000.0, 1000.0, 750.0], x)[0] for x in X[:2000]])
    X = X[:2000]
    noise = rng.normal(0, sigma, uv.shape)
    # duplicate the camera so that every point has two observations (active)
    prob = dict(cam_pose=np.array([np.r_[Rotation.from_matrix(R).as_rotvec(), t]] * 2),
                cam_intr=np.array([[1000.0, 1000.0, 750.0]] * 2), points=X,
                obs_cam=np.r_[np.zeros(len(X)), np.ones(len(X))].astype(np.int32),
                obs_point=np.r_[np.arange(len(X)), np.arange(len(X))].astype(np.int32),
                obs_xy=np.r_[uv + noise, uv], obs_winv=None,
                cam_subblock=np.array([0, 0], np.int32))
    o = oracle.Oracle(prob)
    s = o.camera_scale()
    assert s[0] == pytest.approx(sigma, rel=0.05)
    assert s[1] == pytest.approx(0.0, abs=1e-6)
    # weighted residuals are whitened: scaling C^-1 by 4 doubles the scale
    prob4 = dict(prob)
    prob4["obs_winv"] = np.tile([4.0, 0.0, 4.0], (2 * len(X), 1))
    assert oracle.Oracle(prob4).camera_scale()[0] == pytest.approx(2 * s[0], rel=1e-9)


def test_sigma0_redundancy_and_noise_level():
    """Noise sigma 0.5 px, no outliers: the adjusted sigma_0 is ~0.5 (Sec. 6.2)."""
    prob = synth.config(1)
    keep = ~prob["outlier"]
    for k in ("obs_cam", "obs_point", "obs_xy"):
        prob[k] = prob[k][keep]
    o = oracle.Oracle(prob)
    rep = o.run()
    assert 0.48 < rep["sigma0"] < 0.53
    assert rep["outer"] <= 10
    # sigma_0^2 * redundancy equals the weighted residual sum
    v = o.residuals()
    X, act = o.points()
    m = act[prob["obs_point"]] == 1
    red = 2 * m.sum() - 6 * o.M - 3 * act.sum() + 7
    assert rep["sigma0"] ** 2 * red == pytest.approx(float(np.sum(v[m] ** 2)), rel=1e-9)
    # RMS over the same observations
    assert rep["rms"] == pytest.approx(np.sqrt(np.mean(v[m] ** 2)), rel=1e-9)


# --------------------------------------------------------------------------
# whole method
# --------------------------------------------------------------------------
@pytest.mark.parametrize("runs", [(6,), (3, 3), (2, 2, 2)])
def test_noise_free_block_converges_to_ground_truth(runs):
    """The bact/bars fixed point converges linearly to the exact solution."""
    prob = synth.tiny(seed=41, nx=3, ny=2, n_points=60, opp=4, runs=list(runs), sigma_px=0.0)
    o = oracle.Oracle(prob)
    rep = o.run(max_outer=60)
    assert rep["rms"] < 1e-7
    h = np.array(rep["sigma0_hist"])
    above_floor = h[:-1] > 1e-8
    assert np.all(h[1:][above_floor] < h[:-1][above_floor])
    X, act = o.points()
    assert act.all()
    est = np.r_[camera_centres(o.cameras()), X]
    gt = np.r_[camera_centres(prob["gt_cam_pose"]), prob["gt_points"]]
    s, R, t = umeyama(est, gt)
    aligned = s * est @ R.T + t
    assert np.abs(aligned - gt).max() < 1e-6


def test_single_subblock_is_ordinary_bundle_adjustment():
    """L = 1: no TPs, the LM loop minimises the plain weighted BA cost."""
    prob = with_weights(synth.tiny(seed=42, runs=[6], n_points=40), 42)
    o = oracle.Oracle(prob)
    o.intersect()
    _, Wl = o.instance_state()
    assert np.all(Wl == 0.0)
    for step in range(8):
        Na, g, nC = dense_subblock_system(o, prob, 0, 1e-4)
        r, Fb, Ft, dc, dx = o.lm_step(0, 1e-4)
        if step < 3:
            # later steps are rounding-level; L = 1 leaves the 7-DoF gauge to the
            # damping alone (cond ~ 1e8), so only the first steps are compared
            delta = np.linalg.solve(Na, -g)
            np.testing.assert_allclose(np.r_[dc, dx.reshape(-1)], delta,
                                       atol=1e-6 * np.abs(delta).max())
    # at the end the gradient of the plain BA cost vanishes
    Na, g, nC = dense_subblock_system(o, prob, 0, 0.0)
    assert np.abs(g).max() < 1e-6 * np.abs(Na).max()


def test_lambda_policy_hand_cases():
    """Reading of Sec. 5.5 (lambda fixed in the paper, silent on rejection):
    x10 after a rejected step, /10 after an accepted one, never below lambda0."""
    assert oracle.lambda_next(1e-4, 0, 1e-4) == pytest.approx(1e-3, rel=1e-15)
    assert oracle.lambda_next(1e-2, 0, 1e-4) == pytest.approx(1e-1, rel=1e-15)
    assert oracle.lambda_next(1e-2, 1, 1e-4) == pytest.approx(1e-3, rel=1e-15)
    assert oracle.lambda_next(1e-4, 1, 1e-4) == 1e-4
    assert oracle.lambda_next(5e-4, 1, 1e-4) == 1e-4  # 5e-5 is floored at lambda0
    assert oracle.lambda_next(1e-3, 1, 1e-3) == 1e-3


@pytest.mark.parametrize("values,grace,stop", [
    ([10.0, 5.0, 4.99, 4.98], 1, 3),          # one grace iteration, then stop
    ([10.0, 5.0, 4.99, 4.0, 3.99], 1, 4),     # the grace is not given back by a later improvement
    ([10.0, 9.95], 0, 1),                     # no grace: the first small ratio stops
    ([10.0, 10.5, 10.6], 1, 2),               # a worse value is a ratio below 1 (best stays 10)
    ([10.0, 10.5, 9.0, 8.95], 1, 3),          # ... and the best so far, not the last value, is the reference
    ([10.0, 9.0, 8.0, 7.0], 1, None),         # ratios of 1.11..1.14 never stop
    ([1.01, 1.0, 0.9999], 0, 2),              # a ratio of exactly 1.01 is not below 1.01; 1.0001 is
])
def test_ratio_rule_hand_sequences(values, grace, stop):
    """The stop rule of Sec. 5.5 for the inner (F_l) and the outer (sigma_0)
    loop on hand-worked sequences: ratio = best so far / new value, below
    1.01 spends the one grace iteration, then stops."""
    assert oracle.ratio_rule_sequence(values, 1.01, grace) == stop


def _dense_lm_loop(o2, prob, lambda0=1e-4, stop_ratio=1.01, grace=1, max_inner=20, max_reject=6):
    """An LM loop over one sub-block written with dense numpy algebra: the
    normal equations J^T W J of all unknowns (cameras and points), the damping
    lambda diag(N), np.linalg.solve, the trial update R <- exp([dw]x) R (scipy),
    the cost of Eq. bact in numpy, acceptance on a decrease, and the damping
    and stop rules of Sec. 5.5 as read (x10 on reject, /10 floored at lambda0
    on accept; best/current below 1.01 after one grace iteration). o2 only
    holds the state and projects points (its projection is pinned above)."""
    lam, best, g_left, rejects = lambda0, None, grace, 0
    F = sub_cost_numpy(o2, prob, 0, o2.cameras(), o2.instance_state()[0])
    best = F
    lams, accs, Fs = [], [], []
    it = 0
    while it < max_inner:
        it += 1
        Na, g, nC = dense_subblock_system(o2, prob, 0, lam)
        delta = np.linalg.solve(Na, -g)
        poses0 = o2.cameras()
        Xl0, Wl = o2.instance_state()
        poses_t = poses0.copy()
        for n, i in enumerate(o2.sub_cameras(0)):
            Rt = Rotation.from_rotvec(delta[6 * n:6 * n + 3]).as_matrix() @ pose_R(poses0[i])
            poses_t[i, :3] = Rotation.from_matrix(Rt).as_rotvec()
            poses_t[i, 3:] = poses0[i, 3:] + delta[6 * n + 3:6 * n + 6]
        Xl_t = Xl0 + delta[nC:].reshape(-1, 3)
        Ft = sub_cost_numpy(o2, prob, 0, poses_t, Xl_t)
        lams.append(lam)
        accepted = Ft < F
        accs.append(int(accepted))
        Fs.append(Ft if accepted else F)
        if not accepted:
            lam *= 10.0
            rejects += 1
            if rejects > max_reject:
                break
            continue
        rejects = 0
        o2.set_cameras(poses_t)
        o2.set_instance_state(Xl_t, Wl)
        F = Ft
        lam = max(lam / 10.0, lambda0)
        ratio = best / F
        best = min(best, F)
        if ratio < stop_ratio:
            if g_left > 0:
                g_left -= 1
            else:
                break
    return it, np.array(lams), np.array(accs), np.array(Fs)


@pytest.mark.parametrize("seed,rot_sigma,pos_sigma,lambda0,rejects", [
    (42, 0.01, 0.3, 1e-4, False),
    (43, 0.01, 0.3, 1e-4, False),
    # far from the minimum with little damping: rejected steps raise lambda
    # four times in a row, then accepted steps lower it again
    (50, 0.1, 2.0, 1e-6, True),
])
def test_single_subblock_lm_loop_equals_dense_lm(seed, rot_sigma, pos_sigma, lambda0, rejects):
    """L = 1 (no TPs): the oracle's whole LM loop (orc_sub_lm) is ordinary
    bundle adjustment. It takes the same number of iterations, the same
    damping sequence and the same accept/reject decisions as a dense numpy LM
    loop with the same policy, and its cost after every step agrees to 1e-10
    (at lambda0 = 1e-4; scaled by 1e-4 / lambda0 below it).
    Parameters are compared to 1e-6: with L = 1 the 7-DoF gauge is left to the
    damping alone (cond ~ 1e8), so rounding moves them along the gauge
    without changing the cost."""
    prob = with_weights(synth.tiny(seed=seed, runs=[6], n_points=40, rot_sigma=rot_sigma, pos_sigma=pos_sigma,
                                   pt_sigma=max(0.1, pos_sigma)), seed)
    o = oracle.Oracle(prob)
    o.intersect()
    o2 = oracle.Oracle(prob)
    o2.intersect()
    _, Wl = o.instance_state()
    assert o.L == 1 and np.all(Wl == 0.0)
    it, lam, acc, F = o.sub_lm_trace(0, lambda0=lambda0)
    it_d, lam_d, acc_d, F_d = _dense_lm_loop(o2, prob, lambda0=lambda0)
    assert it == it_d and it >= 3
    assert bool((acc != 1).any()) == rejects
    np.testing.assert_array_equal(acc == 1, acc_d == 1)
    np.testing.assert_allclose(lam, lam_d, rtol=1e-15)
    # the gauge's eigenvalues of the damped system scale with lambda0, so the
    # rounding in the step grows with 1 / lambda0: 1e-10 at the default 1e-4
    np.testing.assert_allclose(F, F_d, rtol=1e-10 * (1e-4 / lambda0))
    np.testing.assert_allclose(o.cameras(), o2.cameras(), atol=1e-6)
    np.testing.assert_allclose(o.instance_state()[0], o2.instance_state()[0], atol=1e-6)


def test_outer_loop_stops_where_the_ratio_rule_says():
    """The outer loop of orc_run (Sec. 5.5) stops at the first sigma_0 the
    stop rule rejects, counted on its own sigma_0 history from sigma_0 after
    the first intersection (robust stage off, so no restart)."""
    prob = synth.config(1)
    keep = ~prob["outlier"]
    for k in ("obs_cam", "obs_point", "obs_xy"):
        prob[k] = prob[k][keep]
    rep = oracle.Oracle(prob).run(robust=0)
    seq = [rep["sigma0_initial"]] + rep["sigma0_hist"]
    stop = oracle.ratio_rule_sequence(seq, 1.01, 1)
    assert stop == rep["outer"] and rep["outer"] < 30


def test_ablation_weights_all_cameras_and_scalar():
    """The ablation variants of Sec. 6.4 for the TPs' weight W^l. All cameras:
    the point's full normal matrix N_j for every instance; since the refined
    weights N_j - N_j^(l) of a point's n instances sum to (n - 1) N_j, it must
    equal that sum / (n - 1). Scalar: rho I, rho0 at the first intersection
    and 1.01 times more per outer iteration (the plain approach's schedule,
    Sec. 6.3); single-sub-block points get no weight in either."""
    prob = synth.tiny(seed=6, nx=4, ny=3, n_points=120, runs=[4, 4, 4], oblique_deg=30, nadir_every=3)
    o0 = oracle.Oracle(prob)
    o0.intersect()
    o1 = oracle.Oracle(prob)
    o1.intersect(weight_mode=1)
    ip, _ = o0.instances()
    _, W0 = o0.instance_state()
    _, W1 = o1.instance_state()
    n = np.bincount(ip, minlength=o0.N)
    tp = n[ip] >= 2
    assert tp.any() and (~tp).any()
    full = np.zeros((o0.N, 6))
    np.add.at(full, ip[tp], W0[tp])
    full[n >= 2] /= (n[n >= 2] - 1)[:, None]
    np.testing.assert_allclose(W1[tp], full[ip[tp]], rtol=1e-10, atol=1e-12 * np.abs(full).max())
    assert np.all(W1[~tp] == 0.0)
    o2 = oracle.Oracle(prob)
    o2.intersect(weight_mode=2, rho0=50.0)
    _, W2 = o2.instance_state()
    eye = np.array([1.0, 0, 0, 1.0, 0, 1.0])
    np.testing.assert_array_equal(W2[tp], np.tile(50.0 * eye, (int(tp.sum()), 1)))
    assert np.all(W2[~tp] == 0.0)
    o3 = oracle.Oracle(prob)
    rep = o3.run(weight_mode=2, rho0=50.0, max_outer=2)
    _, W3 = o3.instance_state()
    _, a3 = o3.points()
    live = tp & (a3[ip] == 1)
    np.testing.assert_allclose(W3[live], np.tile(50.0 * 1.01 ** rep["outer"] * eye, (int(live.sum()), 1)),
                               rtol=1e-15)


def test_robust_stage_finds_injected_outliers():
    prob = synth.config(1)
    o = oracle.Oracle(prob)
    rep = o.run(robust=1, robust_from_start=1)
    _, act = o.points()
    bad = np.unique(prob["obs_point"][prob["outlier"]])
    recall = (act[bad] == 0).mean()
    assert recall >= 0.95
    good = np.setdiff1d(np.arange(o.N), bad)
    assert (act[good] == 0).mean() < 0.06
    assert 0.45 < rep["sigma0"] < 0.55


@pytest.mark.parametrize("single_subblock", [True, False])
def test_serial_robust_stage_deletes_the_outliers(single_subblock):
    """Serial variant of Sec. 5.3 (t_v = 3): the down-weighted observations are
    deleted at the end and points left with fewer than two observations are
    eliminated. No injected outlier survives among the kept observations of
    the kept points, every kept point keeps at least two observations, and
    sigma_0 after the deletion is the noise level (0.5 px)."""
    prob = synth.config(1)
    if single_subblock:  # the serial case proper: one block, L = 1
        prob = dict(prob)
        prob["cam_subblock"] = np.zeros_like(prob["cam_subblock"])
    o = oracle.Oracle(prob)
    rep = o.run(robust=1, robust_from_start=1, robust_serial=1, t_v=3.0)
    _, act = o.points()
    w = o.weights()
    out = prob["outlier"]
    kept = (act[prob["obs_point"]] == 1) & (w == 1.0)
    assert set(np.unique(w)) <= {0.0, 1.0}  # deleted or kept, nothing in between
    assert not (kept & out).any()
    per_point = np.bincount(prob["obs_point"][kept], minlength=o.N)
    assert per_point[act == 1].min() >= 2
    assert 0.45 < rep["sigma0"] < 0.55
    # sigma_0 counts only the kept observations (a deleted one has weight 0)
    assert rep["active_points"] == int(act.sum())


def test_robust_stage_without_outliers_deletes_little():
    prob = synth.config(1)
    keep = ~prob["outlier"]
    for k in ("obs_cam", "obs_point", "obs_xy"):
        prob[k] = prob[k][keep]
    o = oracle.Oracle(prob)
    rep = o.run(robust=1)
    assert rep["robust_started_at"] >= 1
    assert rep["deleted_points"] / o.N < 0.01
