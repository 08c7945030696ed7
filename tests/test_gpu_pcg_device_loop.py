"""The FP32 form's block-Jacobi PCG inside the LM step's captured graph: the
refinement stages and the CG steps run as nested conditional while nodes, no
host read per solve. Checked against the host-driven loop of the same
kernels (taken while a loop kernel is being timed, since conditional bodies
hold no timing events): the same iterations, stages and LM trajectory; the
launch count from the device counters; and the bound on the loop when the
step cap ends it before convergence.
"""

import numpy as np
import pytest

from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu

OPTS = dict(precision=1, solver=1, robust=1, robust_from_start=1, max_inner=1)


def _run(host_loop, steps=3, **opts):
    g = rpba.Rpba(synth.config(1), **{**OPTS, **opts})
    g.intersect()
    g.profile_enable(True)
    # timing a loop kernel keeps the CG loop on the host; timing another
    # kernel leaves it on the device
    g.profile_select("k_pcg_symv32" if host_loop else "k_isect_fused_f")
    hist, its, stages = [], [], []
    for _ in range(steps):
        hist.append(g.outer_iteration(robust=True)[0])
        it, rr = g.solver_stats()
        its.append(it.copy())
        stages.append(g.solver_stages().copy())
    prof, total = g.profile_read()
    out = dict(hist=np.array(hist), its=np.array(its), stages=np.array(stages), rr=rr, cams=g.cameras(),
               prof=prof, total=total)
    g.close()
    return out


def test_device_loop_equals_host_loop():
    d, h = _run(False), _run(True)
    # the CG product is exact in the order of its atomics: the solves take the
    # same steps and stages; only the Schur atomics' order differs
    np.testing.assert_array_equal(d["its"], h["its"])
    np.testing.assert_array_equal(d["stages"], h["stages"])
    assert np.all(d["stages"] >= 1)
    np.testing.assert_allclose(d["hist"], h["hist"], rtol=1e-9)
    np.testing.assert_allclose(d["cams"], h["cams"], rtol=0, atol=1e-9)
    # launches counted from the loop's device counters: one product and one
    # step per lock-step CG step (at least the slowest sub-block's steps of
    # each solve); the host loop may add launches that find every sub-block
    # converged, as it reads the live count only every few steps
    n32 = d["prof"]["k_pcg_symv32"][0]
    assert n32 == d["prof"]["k_pcg_step32"][0]
    assert d["its"].max(axis=1).sum() <= n32 <= h["prof"]["k_pcg_symv32"][0]
    # one float-float product per stage in both
    assert d["prof"]["k_pcg_symv_ff"][0] == h["prof"]["k_pcg_symv_ff"][0] == d["stages"].max(axis=1).sum()
    assert "k_pcg_cond" in d["prof"] and "k_pcg_cond" not in h["prof"]


def test_step_cap_ends_the_device_loop():
    """pcg_max_iter bounds the CG steps of all stages together: with a cap of
    3 the loop ends after 3 steps, the solve is left unconverged (its true
    residual above pcg_tol) and the step completes."""
    d = _run(False, steps=1, pcg_max_iter=3)
    assert d["its"].max() <= 3
    assert np.all(d["rr"] > 1e-8)
    assert d["prof"]["k_pcg_symv32"][0] <= 3
    assert np.isfinite(d["hist"]).all()
