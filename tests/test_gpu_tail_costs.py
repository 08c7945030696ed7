"""The FP32 form's outer-iteration tail evaluates sigma_0 (Eq. sigma0) and every
sub-block's cost F_l (Eq. bact) in one pass over the observations: after the
exchange and the TP copies (Sec. 5) every X^l equals its point's X, so the TP
control terms vanish and F_l is the image part of sigma_0's sum over the
sub-block. The next bact starts from these costs instead of evaluating them
again, as long as no entry point has changed the state in between.

Checked here: sigma_0 of the tail against the FP64 oracle at the tail's state;
the reuse against runs that evaluate the costs afresh (an entry point that
changes nothing, the sub-block mask set to all sub-blocks, ends the reuse);
and that every entry point that changes the state ends it too.
"""

import numpy as np
import pytest

import oracle
from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu

OPTS = dict(precision=1, solver=4, robust=1, robust_from_start=1)


def _prob():
    return synth.config(1)


def _sync_oracle(o, g):
    o.set_camera_rt(g.camera_rt())
    X, a = g.points()
    o.set_points(X, a)
    Xl, Wl = g.instance_state()
    o.set_instance_state(Xl, Wl)
    o.set_weights(g.weights())


def test_tail_sigma0_matches_the_oracle_at_the_tail_state():
    prob = _prob()
    g = rpba.Rpba(prob, **OPTS)
    o = oracle.Oracle(prob)
    for _ in range(3):
        s, _ = g.outer_iteration(robust=True)
        _sync_oracle(o, g)
        # the FP32 form's sigma_0 tolerance (float-float residuals, FP32 terms)
        assert s == pytest.approx(o.sigma0(), rel=1e-6)
        # and the separate sigma_0 pass at the same state
        assert s == pytest.approx(g.sigma0()[0], rel=1e-12)
    g.close()


def _run(mutate=None, refresh=False, steps=3):
    prob = _prob()
    g = rpba.Rpba(prob, **OPTS)
    hist = [g.outer_iteration(robust=True)[0]]
    if mutate is not None:
        mutate(g)
    for _ in range(steps - 1):
        if refresh:
            g.set_subblock_mask(None)  # changes nothing, ends the reuse
        hist.append(g.outer_iteration(robust=True)[0])
    cams = g.cameras()
    g.close()
    return np.array(hist), cams


def test_reused_costs_equal_fresh_costs():
    h_reuse, c_reuse = _run()
    h_fresh, c_fresh = _run(refresh=True)
    # the two runs differ only in the order of the Schur atomics
    np.testing.assert_allclose(h_reuse, h_fresh, rtol=1e-7)
    np.testing.assert_allclose(c_reuse, c_fresh, rtol=0, atol=1e-7)


def _perturb_points(g):
    X, a = g.points()
    g.set_points(X + np.random.default_rng(1).normal(0, 0.05, X.shape), a)


def _perturb_cameras(g):
    c = g.cameras()
    c[:, 3:] += np.random.default_rng(2).normal(0, 0.02, (c.shape[0], 3))
    g.set_cameras(c)


def _halve_weights(g):
    w = g.weights()
    w[::7] *= 0.5
    g.set_weights(w)


def _move_instances(g):
    Xl, Wl = g.instance_state()
    g.set_instance_state(Xl + np.random.default_rng(3).normal(0, 0.05, Xl.shape), Wl)


def _intersect_all(g):
    g.intersect_points(tp_only=False)


@pytest.mark.parametrize("mutate", [_perturb_points, _perturb_cameras, _halve_weights, _move_instances,
                                    _intersect_all], ids=lambda f: f.__name__.strip("_"))
def test_state_changes_end_the_reuse(mutate):
    h_a, c_a = _run(mutate=mutate)
    h_b, c_b = _run(mutate=mutate, refresh=True)
    np.testing.assert_allclose(h_a, h_b, rtol=1e-7)
    np.testing.assert_allclose(c_a, c_b, rtol=0, atol=1e-7)
