"""Per-camera intrinsics (the Final data sets of Sec. 6: focal length and
first radial parameter estimated with each pose, 8 unknowns per camera) on
the GPU, through the C ABI, against the FP64 oracle at shared states.

Tolerances as for the pinhole blocks: FP64 form to rounding; FP32 form
Jacobians 1e-5 relative, covariance 1e-4, RCS 2e-5 of its largest entry,
costs and sigma_0 1e-6, final RMS within 1e-3 px of the oracle.
"""

import numpy as np
import pytest

import oracle
from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu


def _prob(seed=5, **kw):
    prob = synth.tiny_intrinsics(seed=seed, **kw)
    prob["cam_k1"] = 0.5 * prob["gt_cam_k1"]  # a nonzero k1 in the start state
    return prob


def _sync(o, g):
    g.set_cameras(o.cameras())
    g.set_intrinsics(o.intrinsics())
    X, a = o.points()
    g.set_points(X, a)
    Xl, Wl = o.instance_state()
    g.set_instance_state(Xl, Wl)
    g.set_weights(o.weights())


def _rel(a, b, axis):
    return np.linalg.norm(a - b, axis=axis) / np.maximum(np.linalg.norm(b, axis=axis), 1e-300)


def _state(precision, seed=5, **opts):
    prob = _prob(seed)
    o = oracle.Oracle(prob)
    g = rpba.Rpba(prob, precision=precision, **opts)
    o.intersect()
    rng = np.random.default_rng(seed)
    Xl, Wl = o.instance_state()
    o.set_instance_state(Xl + rng.normal(0, 0.01, Xl.shape), Wl)
    o.set_weights(np.where(rng.random(o.K) < 0.05, 1e-4, 1.0))
    fk = o.intrinsics()
    fk[:, 0] *= 1.0 + rng.normal(0, 0.003, o.M)
    o.set_intrinsics(fk)
    _sync(o, g)
    return prob, o, g


def test_intrinsics_state_options_and_refusals():
    prob = _prob()
    g = rpba.Rpba(prob, precision=1, solver=4)
    assert g.cd == 8 and g.resolved_options().solver == 1  # auto: PCG on 3 sub-blocks
    fk = g.intrinsics()
    np.testing.assert_array_equal(fk[:, 0], prob["cam_intr"][:, 0])
    np.testing.assert_array_equal(fk[:, 1], prob["cam_k1"])
    fk2 = fk * np.array([1.01, 1.5])
    g.set_intrinsics(fk2)
    np.testing.assert_array_equal(g.intrinsics(), fk2)
    with pytest.raises(rpba.RpbaError):
        g.set_intrinsics(fk2 * np.array([-1.0, 1.0]))  # a negative focal length
    g.close()
    with pytest.raises(rpba.RpbaError):  # the learned preconditioner is built on 6 x 6 camera blocks
        rpba.Rpba(prob, precision=1, solver=3)
    # without the option the intrinsics are fixed and k1 is 0
    g6 = rpba.Rpba(prob, precision=0, intrinsics=0)
    fk6 = g6.intrinsics()
    assert np.all(fk6[:, 1] == 0.0)
    g6.set_intrinsics(fk6)
    with pytest.raises(rpba.RpbaError):
        g6.set_intrinsics(fk6 * 1.01)
    g6.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_residuals_and_jacobians_with_intrinsics(precision):
    prob, o, g = _state(precision)
    np.testing.assert_allclose(g.residuals(), o.residuals(), rtol=0, atol=1e-9)
    Jc_o, Jx_o = o.jacobians()
    Jc_g, Jx_g = g.jacobians()
    assert Jc_g.shape == (o.K, 2, 8)
    tol = 1e-12 if precision == 0 else 1e-5
    assert _rel(Jc_g, Jc_o, (1, 2)).max() <= tol
    assert _rel(Jx_g, Jx_o, (1, 2)).max() <= tol
    # the intrinsic columns alone (they are small beside the pose columns)
    assert _rel(Jc_g[:, :, 6:], Jc_o[:, :, 6:], (1, 2)).max() <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_intersection_covariance_and_costs_with_intrinsics(precision):
    prob, o, g = _state(precision)
    # costs and sigma_0 at the shared state
    Fo = np.array([o.sub_cost(l) for l in range(o.L)])
    np.testing.assert_allclose(g.sub_costs(), Fo, rtol=1e-11 if precision == 0 else 1e-6)
    assert g.sigma0()[0] == pytest.approx(o.sigma0(), rel=1e-11 if precision == 0 else 1e-6)
    np.testing.assert_allclose(g.camera_scale(), o.camera_scale(), rtol=1e-9 if precision == 0 else 1e-6)
    # covariance of every active point at that state
    X, act = o.points()
    ids = np.nonzero(act)[0]
    assert _rel(g.covariance(ids), o.covariance(ids), (1, 2)).max() <= (1e-10 if precision == 0 else 1e-4)
    # the intersection from the same start
    o.intersect(tp_only=True)
    g.intersect_points(True)
    Xo, ao = o.points()
    Xg, ag = g.points()
    both = (ao == 1) & (ag == 1)
    assert (ao != ag).mean() <= (0.0 if precision == 0 else 0.01)
    err = np.abs(Xg[both] - Xo[both]).max(1)
    if precision == 0:
        assert err.max() <= 1e-9
    else:  # both stop once a step moves the image by < 1e-3 px per observation
        assert np.quantile(err, 0.99) <= 1e-4 and err.max() <= 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_rcs_with_intrinsics(precision):
    prob, o, g = _state(precision)
    for l in range(o.L):
        for lam in (1e-4, 1e-2):
            So, yo = o.rcs(l, lam)
            Sg, yg = g.rcs(l, lam)
            assert So.shape == Sg.shape == (8 * len(o.sub_cameras(l)),) * 2
            low = np.tril(np.ones_like(So, dtype=bool))
            tol = 1e-10 if precision == 0 else 2e-5
            assert np.abs(Sg[low] - So[low]).max() <= tol * np.abs(So).max()
            assert np.abs(yg - yo).max() <= tol * 10 * np.abs(yo).max()


@pytest.mark.parametrize("form", [(0, 0), (1, 0), (0, 2), (1, 2)])
def test_lm_step_with_intrinsics(form):
    precision, solver = form
    prob, o, g = _state(precision, solver=solver)
    acc, Fb, Ft, dc, dx = g.lm_step(1e-4)
    off = 0
    _, isub = o.instances()
    dk1 = 0.0
    for l in range(o.L):
        r, fb, ft, dco, dxo = o.lm_step(l, 1e-4)
        n = dco.size
        dk1 = max(dk1, np.abs(dco.reshape(-1, 8)[:, 7]).max())
        np.testing.assert_allclose(Fb[l], fb, rtol=1e-11 if precision == 0 else 1e-6)
        tol = 1e-7 if precision == 0 else 5e-3
        # the focal-length and k1 updates are compared on their own scale
        d_g, d_o = dc[off:off + n].reshape(-1, 8), dco.reshape(-1, 8)
        for cols in (slice(0, 6), slice(6, 7), slice(7, 8)):
            sc = max(np.abs(d_o[:, cols]).max(), 1e-12)
            assert np.abs(d_g[:, cols] - d_o[:, cols]).max() <= tol * sc
        sx = max(np.abs(dxo).max(), 1e-12)
        assert np.abs(dx[isub == l] - dxo).max() <= tol * sx
        np.testing.assert_allclose(Ft[l], ft, rtol=1e-8 if precision == 0 else 1e-4)
        assert acc[l] == r
        off += n
    np.testing.assert_allclose(g.cameras(), o.cameras(), atol=1e-8 if precision == 0 else 1e-4)
    # the applied steps agree as the steps do: f to 1e-5 relative, k1 to the
    # step tolerance times the largest k1 step
    fg, fo = g.intrinsics(), o.intrinsics()
    np.testing.assert_allclose(fg[:, 0], fo[:, 0], rtol=1e-9 if precision == 0 else 1e-5)
    assert np.abs(fg[:, 1] - fo[:, 1]).max() <= (1e-7 if precision == 0 else 5e-3) * dk1 + 1e-15


@pytest.mark.parametrize("form", [(1, 1), (1, 4), (0, 1)])
def test_lm_step_pcg_with_intrinsics(form):
    """Block-Jacobi PCG with 8 x 8 camera blocks: the returned camera step
    solves the GPU's own RCS to pcg_tol (plus the product's rounding), and
    matches the oracle's Cholesky step within the form's tolerance."""
    precision, solver = form
    prob, o, g = _state(precision, solver=solver)
    assert g.resolved_options().solver == 1
    lam = 1e-4
    systems = []
    for l in range(g.L):
        S, y = g.rcs(l, lam)
        systems.append((np.tril(S) + np.tril(S, -1).T, y))
    acc, Fb, Ft, dc, dx = g.lm_step(lam)
    it, rr = g.solver_stats()
    assert np.all(it > 0) and np.all(rr <= g.options.pcg_tol)
    off = 0
    _, isub = o.instances()
    for l in range(o.L):
        S, y = systems[l]
        n = y.size
        dcl = dc[off:off + n]
        res = np.linalg.norm(S @ dcl - y) / np.linalg.norm(y)
        fp = 1e-12 * np.linalg.norm(np.abs(S) @ np.abs(dcl)) / np.linalg.norm(y)
        assert res <= g.options.pcg_tol + fp, (l, res, fp)
        r, fb, ft, dco, dxo = o.lm_step(l, lam)
        tol = 1e-5 if precision == 0 else 5e-3
        d_g, d_o = dcl.reshape(-1, 8), dco.reshape(-1, 8)
        for cols in (slice(0, 6), slice(6, 7), slice(7, 8)):
            sc = max(np.abs(d_o[:, cols]).max(), 1e-12)
            assert np.abs(d_g[:, cols] - d_o[:, cols]).max() <= tol * sc
        np.testing.assert_allclose(Ft[l], ft, rtol=1e-6 if precision == 0 else 1e-4)
        off += n


@pytest.mark.parametrize("precision", [0, 1])
def test_whole_run_with_intrinsics(precision):
    """The whole method (robust stage from the start) on a ring block with
    1 % outliers: the final RMS within 1e-3 px of the oracle's, and the
    estimated focal lengths and radial parameters close to the oracle's."""
    prob = synth.tiny_intrinsics(seed=9, n_cams=30, n_points=800, mean_track=6.0, n_sub=3,
                                 outlier_frac=0.01)
    o = oracle.Oracle(prob)
    ro = o.run(robust=1, robust_from_start=1)
    g = rpba.Rpba(prob, precision=precision, solver=4, robust=1, robust_from_start=1)
    rg = g.iterate()
    assert abs(rg["rms"] - ro["rms"]) <= 1e-3
    if precision == 0:
        assert rg["outer"] == ro["outer"]
        np.testing.assert_allclose(rg["sigma0_hist"], ro["sigma0_hist"], rtol=1e-6)
    fo, fg = o.intrinsics(), g.intrinsics()
    np.testing.assert_allclose(fg[:, 0], fo[:, 0], rtol=1e-6 if precision == 0 else 1e-3)
    np.testing.assert_allclose(fg[:, 1], fo[:, 1], atol=1e-8 if precision == 0 else 1e-3)
    g.close()


def test_outer_iteration_with_intrinsics_fp32():
    """The benchmark's step in the FP32 form with intrinsics: sigma_0 of the
    tail equals the oracle's at the tail's state (1e-6)."""
    prob = _prob(seed=11)
    g = rpba.Rpba(prob, precision=1, solver=4, robust=1, robust_from_start=1)
    o = oracle.Oracle(prob)
    for _ in range(2):
        s, _ = g.outer_iteration(robust=True)
        o.set_camera_rt(g.camera_rt())
        o.set_intrinsics(g.intrinsics())
        X, a = g.points()
        o.set_points(X, a)
        Xl, Wl = g.instance_state()
        o.set_instance_state(Xl, Wl)
        o.set_weights(g.weights())
        assert s == pytest.approx(o.sigma0(), rel=1e-6)
    g.close()
