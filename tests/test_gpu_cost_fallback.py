"""The FP32 form's cost pass stages a sub-block's camera records in shared
memory (k_cost_groups_f) when the largest sub-block's records fit 96 KB
(682 cameras); beyond that the records are read from global memory
(k_cost_chunks_f). This block has a sub-block of 720 cameras, so the
global-memory kernel runs: its sub-block costs (Eq. bact) and sigma_0
(Eq. sigma0) against the FP64 oracle at the same state, to the FP32 form's
1e-6.
"""

import numpy as np
import pytest

import oracle
from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu


def test_cost_pass_without_staging_matches_the_oracle():
    prob = synth.tiny(seed=3, nx=30, ny=25, n_points=6000, runs=[720, 30], extent=(-60.0, 60.0, -50.0, 50.0))
    assert np.bincount(prob["cam_subblock"]).max() == 720
    g = rpba.Rpba(prob, precision=1, solver=0)
    g.intersect()
    o = oracle.Oracle(prob)
    o.set_camera_rt(g.camera_rt())
    X, a = g.points()
    o.set_points(X, a)
    Xl, Wl = g.instance_state()
    rng = np.random.default_rng(4)
    Xl = Xl + rng.normal(0, 0.01, Xl.shape)  # sub-block copies off X: the TP terms count
    o.set_instance_state(Xl, Wl)
    g.set_instance_state(Xl, Wl)
    g.profile_enable(True)
    F = g.sub_costs()
    prof, _ = g.profile_read()
    g.profile_enable(False)
    assert "k_cost_chunks_f" in prof and "k_cost_groups_f" not in prof
    np.testing.assert_allclose(F, [o.sub_cost(l) for l in range(o.L)], rtol=1e-6)
    assert g.sigma0()[0] == pytest.approx(o.sigma0(), rel=1e-6)
    g.close()
