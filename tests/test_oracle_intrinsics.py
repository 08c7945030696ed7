"""Pins of the oracle's per-camera intrinsics (the Final data sets of Sec. 6:
focal length f and the first radial distortion parameter k1 estimated with
each camera's pose, 8 unknowns per camera) against facts that do not come from
the oracle: hand-worked projections, the pinhole special case, finite
differences, dense normal equations and a dense LM loop in numpy, recovery of
the true intrinsics from noise-free observations, and sigma_0's redundancy.
No GPU is used.
"""

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_1910_08138_gb300 import synth


def _rand_camera(rng):
    R = Rotation.from_rotvec(rng.normal(size=3) * 0.8).as_matrix()
    X = rng.uniform(-3, 3, 3)
    t = -R @ X + np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(4, 10)])
    intr = np.array([rng.uniform(600, 1400), 1000.0, 750.0])
    return R, t, intr, X + rng.normal(size=3)


# --------------------------------------------------------------------------
# the projection with k1
# --------------------------------------------------------------------------
def test_projection_hand_values():
    """(u, v) = f (1 + k1 |p|^2) p + c, worked by hand."""
    I, z0 = np.eye(3), np.zeros(3)
    intr = [1000.0, 1000.0, 750.0]
    # p = (0.5, 0), |p|^2 = 0.25, 1 + 0.1 * 0.25 = 1.025
    uv, _, _, z = oracle.project_k1(I, z0, intr, 0.1, [1.0, 0.0, 2.0])
    np.testing.assert_allclose(uv, [1512.5, 750.0], rtol=0, atol=1e-9)
    assert z == 2.0
    # p = (0.3, -0.4), |p|^2 = 0.25
    uv, _, _, _ = oracle.project_k1(I, z0, intr, 0.1, [0.6, -0.8, 2.0])
    np.testing.assert_allclose(uv, [1307.5, 340.0], rtol=0, atol=1e-9)
    # k1 = -0.2 at |p|^2 = 1: the radial factor is 0.8
    uv, _, _, _ = oracle.project_k1(I, z0, intr, -0.2, [3.0, 4.0, 5.0])
    np.testing.assert_allclose(uv, [1000.0 + 480.0, 750.0 + 640.0], rtol=0, atol=1e-9)
    # on the optical axis: the principal point whatever f and k1
    uv, _, _, _ = oracle.project_k1(I, [0.1, -0.2, 3.0], [777.0, 1000.0, 750.0], 0.3, [-0.1, 0.2, 2.0])
    np.testing.assert_allclose(uv, [1000.0, 750.0], rtol=0, atol=1e-12)


def test_projection_with_k1_zero_is_the_pinhole():
    rng = np.random.default_rng(1)
    for _ in range(20):
        R, t, intr, X = _rand_camera(rng)
        uv, Jc, Jx, z = oracle.project(R, t, intr, X)
        uv8, Jc8, Jx8, z8 = oracle.project_k1(R, t, intr, 0.0, X)
        assert z8 == z
        np.testing.assert_allclose(uv8, uv, rtol=1e-15, atol=1e-9)
        np.testing.assert_allclose(Jc8[:, :6], Jc, rtol=1e-14, atol=1e-10)
        np.testing.assert_allclose(Jx8, Jx, rtol=1e-14, atol=1e-10)
        # d/df of a pinhole is the normalised coordinate
        np.testing.assert_allclose(Jc8[:, 6], (uv - intr[1:]) / intr[0], rtol=1e-12)


def _fd_k1(R, t, intr, k1, X, h=1e-6):
    """Central differences of project_k1 w.r.t. (dw left, dt, df, dk1) and X."""
    P = lambda R_, t_, i_, k_, X_: oracle.project_k1(R_, t_, i_, k_, X_)[0]
    Jc, Jx = np.zeros((2, 8)), np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Jc[:, a] = (P(Rotation.from_rotvec(e).as_matrix() @ R, t, intr, k1, X) -
                    P(Rotation.from_rotvec(-e).as_matrix() @ R, t, intr, k1, X)) / (2 * h)
        Jc[:, 3 + a] = (P(R, t + e, intr, k1, X) - P(R, t - e, intr, k1, X)) / (2 * h)
        Jx[:, a] = (P(R, t, intr, k1, X + e) - P(R, t, intr, k1, X - e)) / (2 * h)
    hf = 1e-4 * intr[0]
    di = np.array([hf, 0.0, 0.0])
    Jc[:, 6] = (P(R, t, intr + di, k1, X) - P(R, t, intr - di, k1, X)) / (2 * hf)
    Jc[:, 7] = (P(R, t, intr, k1 + h, X) - P(R, t, intr, k1 - h, X)) / (2 * h)
    return Jc, Jx


def test_projection_k1_jacobians_match_finite_differences():
    rng = np.random.default_rng(2)
    for _ in range(50):
        R, t, intr, X = _rand_camera(rng)
        k1 = rng.uniform(-0.15, 0.15)
        _, Jc, Jx, z = oracle.project_k1(R, t, intr, k1, X)
        assert z > 0
        Jc_fd, Jx_fd = _fd_k1(R, t, intr, k1, X)
        np.testing.assert_allclose(Jc, Jc_fd, rtol=1e-6, atol=1e-6 * np.abs(Jc_fd).max())
        np.testing.assert_allclose(Jx, Jx_fd, rtol=1e-6, atol=1e-6 * np.abs(Jx_fd).max())


def test_residuals_and_jacobians_use_each_cameras_intrinsics():
    prob = synth.tiny_intrinsics(seed=3)
    o = oracle.Oracle(prob)
    assert o.cd == 8
    rng = np.random.default_rng(3)
    fk = np.stack([prob["cam_intr"][:, 0] * (1 + rng.normal(0, 0.01, o.M)), rng.uniform(-0.1, 0.1, o.M)], 1)
    o.set_intrinsics(fk)
    np.testing.assert_array_equal(o.intrinsics(), fk)
    v = o.residuals()
    Jc, Jx = o.jacobians()
    assert Jc.shape == (o.K, 2, 8)
    X, _ = o.points()
    for k in range(0, o.K, 11):
        i, j = prob["obs_cam"][k], prob["obs_point"][k]
        R = Rotation.from_rotvec(prob["cam_pose"][i, :3]).as_matrix()
        intr = np.array([fk[i, 0], prob["cam_intr"][i, 1], prob["cam_intr"][i, 2]])
        uv, jc, jx, _ = oracle.project_k1(R, prob["cam_pose"][i, 3:], intr, fk[i, 1], X[j])
        np.testing.assert_allclose(v[k], uv - prob["obs_xy"][k], atol=1e-9)
        np.testing.assert_allclose(Jc[k], jc, atol=1e-9)
        np.testing.assert_allclose(Jx[k], jx, atol=1e-12)


# --------------------------------------------------------------------------
# normal equations, Schur complement and LM with 8 unknowns per camera
# --------------------------------------------------------------------------
def _cam_state(o):
    poses = o.cameras()
    return poses, o.intrinsics()


def _project(prob, poses, fk, i, X, fd=False):
    R = Rotation.from_rotvec(poses[i, :3]).as_matrix()
    intr = np.array([fk[i, 0], prob["cam_intr"][i, 1], prob["cam_intr"][i, 2]])
    if fd:
        uv = oracle.project_k1(R, poses[i, 3:], intr, fk[i, 1], X)[0]
        return (uv,) + _fd_k1(R, poses[i, 3:], intr, fk[i, 1], X)
    uv, Jc, Jx, _ = oracle.project_k1(R, poses[i, 3:], intr, fk[i, 1], X)
    return uv, Jc, Jx


def _dense_system(o, prob, l, lam, fd=False):
    """Dense N + lam diag(N) and g = J^T W v of sub-block l: 8 unknowns per
    camera of l, then 3 per instance of l, with the TP term of Eq. bact."""
    cams = o.sub_cameras(l)
    cpos = {int(c): n for n, c in enumerate(cams)}
    ip, isub = o.instances()
    inst = np.nonzero(isub == l)[0]
    qpos = {int(q): n for n, q in enumerate(inst)}
    inst_of = {(int(ip[q]), int(isub[q])): int(q) for q in range(o.P)}
    poses, fk = _cam_state(o)
    X, act = o.points()
    Xl, Wl = o.instance_state()
    w = o.weights()
    nC, nX = 8 * len(cams), 3 * len(inst)
    n = nC + nX
    N, g = np.zeros((n, n)), np.zeros(n)
    for k in range(o.K):
        i, j = int(prob["obs_cam"][k]), int(prob["obs_point"][k])
        if prob["cam_subblock"][i] != l or not act[j]:
            continue
        q = inst_of[(j, l)]
        uv, Jc, Jx = _project(prob, poses, fk, i, Xl[q], fd)
        v = uv - prob["obs_xy"][k]
        J = np.zeros((2, n))
        J[:, 8 * cpos[i]:8 * cpos[i] + 8] = Jc
        J[:, nC + 3 * qpos[q]:nC + 3 * qpos[q] + 3] = Jx
        N += w[k] * J.T @ J
        g += w[k] * J.T @ v
    for q in inst:
        a = nC + 3 * qpos[int(q)]
        if act[int(ip[q])]:
            s = Wl[q]
            Wq = np.array([[s[0], s[1], s[2]], [s[1], s[3], s[4]], [s[2], s[4], s[5]]])
            N[a:a + 3, a:a + 3] += Wq
            g[a:a + 3] += Wq @ (Xl[q] - X[int(ip[q])])
        else:
            N[a:a + 3, a:a + 3] = np.eye(3)
    return N + lam * np.diag(np.diag(N)), g, nC


def _cost(o, prob, l, poses, fk, Xl):
    X, act = o.points()
    _, Wl = o.instance_state()
    ip, isub = o.instances()
    inst_of = {(int(ip[q]), int(isub[q])): int(q) for q in range(o.P)}
    w = o.weights()
    F = 0.0
    for k in range(o.K):
        i, j = int(prob["obs_cam"][k]), int(prob["obs_point"][k])
        if prob["cam_subblock"][i] != l or not act[j]:
            continue
        uv = _project(prob, poses, fk, i, Xl[inst_of[(j, l)]])[0]
        v = uv - prob["obs_xy"][k]
        F += w[k] * v @ v
    for q in np.nonzero(isub == l)[0]:
        if act[int(ip[q])]:
            s = Wl[q]
            Wq = np.array([[s[0], s[1], s[2]], [s[1], s[3], s[4]], [s[2], s[4], s[5]]])
            d = Xl[q] - X[int(ip[q])]
            F += d @ Wq @ d
    return F


def _prepared(seed=5, n_sub=3, **kw):
    prob = synth.tiny_intrinsics(seed=seed, n_cams=12, n_points=60, mean_track=5.0, n_sub=n_sub, **kw)
    # start from nonzero k1 (half the true values), so that every k1 term counts
    prob["cam_k1"] = 0.5 * prob["gt_cam_k1"]
    o = oracle.Oracle(prob)
    o.intersect()
    return prob, o


@pytest.mark.parametrize("lam", [0.0, 1e-4])
def test_rcs_with_intrinsics_equals_dense_schur_complement(lam):
    prob, o = _prepared()
    rng = np.random.default_rng(5)
    Xl, Wl = o.instance_state()
    o.set_instance_state(Xl + rng.normal(0, 0.02, Xl.shape), Wl)
    for l in range(o.L):
        Na, g, nC = _dense_system(o, prob, l, lam)
        Ncc, Ncx, Nxx = Na[:nC, :nC], Na[:nC, nC:], Na[nC:, nC:]
        S_dense = Ncc - Ncx @ np.linalg.solve(Nxx, Ncx.T)
        y_dense = -g[:nC] + Ncx @ np.linalg.solve(Nxx, g[nC:])
        S, y = o.rcs(l, lam)
        assert S.shape == (nC, nC)
        np.testing.assert_allclose(S, S_dense, atol=1e-9 * np.abs(S_dense).max(), rtol=0)
        np.testing.assert_allclose(y, y_dense, atol=1e-9 * np.abs(y_dense).max(), rtol=0)
        # and with finite-difference Jacobians
        Nf, _, _ = _dense_system(o, prob, l, lam, fd=True)
        S_fd = Nf[:nC, :nC] - Nf[:nC, nC:] @ np.linalg.solve(Nf[nC:, nC:], Nf[:nC, nC:].T)
        np.testing.assert_allclose(S, S_fd, atol=2e-5 * np.abs(S_fd).max(), rtol=0)


def test_lm_step_with_intrinsics_equals_dense_solve_and_cost():
    prob, o = _prepared(seed=6)
    lam = 1e-4
    for l in range(o.L):
        Na, g, nC = _dense_system(o, prob, l, lam)
        delta = np.linalg.solve(Na, -g)
        poses0, fk0 = _cam_state(o)
        Xl0, _ = o.instance_state()
        F0 = _cost(o, prob, l, poses0, fk0, Xl0)
        r, Fb, Ft, dc, dx = o.lm_step(l, lam)
        assert r in (0, 1)
        np.testing.assert_allclose(Fb, F0, rtol=1e-9)
        np.testing.assert_allclose(dc, delta[:nC], atol=1e-9 * np.abs(delta).max() + 1e-12)
        np.testing.assert_allclose(dx.reshape(-1), delta[nC:], atol=1e-9 * np.abs(delta).max() + 1e-12)
        poses_t, fk_t = poses0.copy(), fk0.copy()
        for n, i in enumerate(o.sub_cameras(l)):
            Rt = Rotation.from_rotvec(dc[8 * n:8 * n + 3]).as_matrix() @ Rotation.from_rotvec(poses0[i, :3]).as_matrix()
            poses_t[i, :3] = Rotation.from_matrix(Rt).as_rotvec()
            poses_t[i, 3:] = poses0[i, 3:] + dc[8 * n + 3:8 * n + 6]
            fk_t[i] = fk0[i] + dc[8 * n + 6:8 * n + 8]
        _, isub = o.instances()
        Xl_t = Xl0.copy()
        Xl_t[isub == l] += dx
        Ft_np = _cost(o, prob, l, poses_t, fk_t, Xl_t)
        np.testing.assert_allclose(Ft, Ft_np, rtol=1e-9)
        assert (r == 1) == (Ft_np < F0)
        if r == 1:
            np.testing.assert_allclose(o.intrinsics(), fk_t, rtol=1e-15, atol=1e-15)


def test_single_subblock_lm_loop_with_intrinsics_equals_dense_lm():
    """L = 1: the oracle's LM loop with 8 unknowns per camera takes the same
    steps, damping and decisions as a dense numpy LM loop of the same policy
    (x10 on reject, /10 floored at lambda0 on accept, best/current < 1.01
    after one grace iteration)."""
    prob, o = _prepared(seed=7, n_sub=1)
    _, o2 = _prepared(seed=7, n_sub=1)
    it, lam, acc, F = o.sub_lm_trace(0)
    lam0, F_cur = 1e-4, _cost(o2, prob, 0, *_cam_state(o2), o2.instance_state()[0])
    best, grace, lam_d, acc_d, F_d, l_cur = F_cur, 1, [], [], [], lam0
    while len(lam_d) < 20:
        Na, g, nC = _dense_system(o2, prob, 0, l_cur)
        delta = np.linalg.solve(Na, -g)
        poses0, fk0 = _cam_state(o2)
        Xl0, Wl = o2.instance_state()
        poses_t, fk_t = poses0.copy(), fk0.copy()
        for n, i in enumerate(o2.sub_cameras(0)):
            Rt = Rotation.from_rotvec(delta[8 * n:8 * n + 3]).as_matrix() @ Rotation.from_rotvec(poses0[i, :3]).as_matrix()
            poses_t[i, :3] = Rotation.from_matrix(Rt).as_rotvec()
            poses_t[i, 3:] = poses0[i, 3:] + delta[8 * n + 3:8 * n + 6]
            fk_t[i] = fk0[i] + delta[8 * n + 6:8 * n + 8]
        Xl_t = Xl0 + delta[nC:].reshape(-1, 3)
        Ft = _cost(o2, prob, 0, poses_t, fk_t, Xl_t)
        lam_d.append(l_cur)
        ok = Ft < F_cur
        acc_d.append(int(ok))
        F_d.append(Ft if ok else F_cur)
        if not ok:
            l_cur *= 10.0
            continue
        o2.set_cameras(poses_t)
        o2.set_intrinsics(fk_t)
        o2.set_instance_state(Xl_t, Wl)
        F_cur, l_cur = Ft, max(l_cur / 10.0, lam0)
        ratio, best = best / F_cur, min(best, F_cur)
        if ratio < 1.01:
            if grace > 0:
                grace -= 1
            else:
                break
    assert it == len(lam_d) and it >= 3
    np.testing.assert_array_equal(acc == 1, np.array(acc_d) == 1)
    np.testing.assert_allclose(lam, lam_d, rtol=1e-15)
    np.testing.assert_allclose(F, F_d, rtol=1e-9)
    np.testing.assert_allclose(o.intrinsics(), o2.intrinsics(), rtol=1e-6, atol=1e-8)


# --------------------------------------------------------------------------
# the whole method
# --------------------------------------------------------------------------
def test_noise_free_single_subblock_recovers_the_intrinsics():
    """Noise-free observations, one sub-block: ordinary bundle adjustment with
    intrinsics lands on the true focal lengths and k1 (they are invariant
    under the 7-DoF gauge) to rounding."""
    prob = synth.tiny_intrinsics(seed=2, sigma_px=0.0, n_sub=1)
    o = oracle.Oracle(prob)
    rep = o.run(max_outer=20)
    assert rep["rms"] < 1e-10
    fk = o.intrinsics()
    np.testing.assert_allclose(fk[:, 0], prob["gt_cam_intr"][:, 0], rtol=1e-12)
    np.testing.assert_allclose(fk[:, 1], prob["gt_cam_k1"], atol=1e-12)


def test_noise_free_subblocks_converge_toward_the_intrinsics():
    """Three sub-blocks: the bact/bars fixed point converges linearly; after
    80 outer iterations the residuals and the intrinsics are close to exact,
    and sigma_0 decreased at every iteration above its floor."""
    prob = synth.tiny_intrinsics(seed=2, sigma_px=0.0, n_sub=3)
    o = oracle.Oracle(prob)
    f0_err = np.abs(prob["cam_intr"][:, 0] - prob["gt_cam_intr"][:, 0]).max()
    rep = o.run(max_outer=80)
    h = np.array(rep["sigma0_hist"])
    assert np.all(h[1:] < h[:-1])
    assert rep["rms"] < 1e-4
    fk = o.intrinsics()
    assert np.abs(fk[:, 0] - prob["gt_cam_intr"][:, 0]).max() < 1e-5 * f0_err * 100
    assert np.abs(fk[:, 1] - prob["gt_cam_k1"]).max() < 1e-5


def test_sigma0_redundancy_with_intrinsics():
    """sigma_0^2 (2 K - 8 M - 3 N + 7) is the residual sum at the end, and
    sigma_0 lands at the pixel noise (0.5 px)."""
    prob = synth.tiny_intrinsics(seed=4, n_cams=24, n_points=600, mean_track=6.0, sigma_px=0.5)
    o = oracle.Oracle(prob)
    rep = o.run()
    v = o.residuals()
    X, act = o.points()
    m = act[prob["obs_point"]] == 1
    red = 2 * m.sum() - 8 * o.M - 3 * act.sum() + 7
    assert rep["sigma0"] ** 2 * red == pytest.approx(float(np.sum(v[m] ** 2)), rel=1e-9)
    assert 0.45 < rep["sigma0"] < 0.55
