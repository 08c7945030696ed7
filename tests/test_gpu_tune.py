"""The autotuner (rpba_tune): launch shapes timed on the context's own data,
cached per workload. The tuned kernels give every thread one independent
item, so a run with the tuned shapes equals the run with the default ones
(FP64 form; to rounding, since the FP64 Schur assembly sums with atomics),
and a new context of the same workload reads the cached choice."""

import json

import numpy as np
import pytest

from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu

OPTS = dict(precision=0, solver=2, robust=1, robust_from_start=1)


def test_tuned_and_default_launch_shapes_give_the_same_run(tmp_path):
    prob = synth.config(3, n_blocks=8)  # 42 sub-blocks of 8 independent blocks, direct solver
    cache = tmp_path / "tune.jsonl"
    g = rpba.Rpba(prob, tune_cache=str(cache), **OPTS)
    g.intersect()
    chosen = g.tune()
    assert chosen["isect"] in (64, 128, 256) and chosen["lin"] in (64, 128, 256)
    assert chosen["backsub"] in (64, 128, 256) and chosen["robust"] in (128, 256, 512)
    assert chosen["chol_tc"] in (0, 1, 2)
    lines = [json.loads(ln) for ln in cache.read_text().splitlines() if ln.strip()]
    assert len(lines) == 1 and all(lines[0][k] == v for k, v in chosen.items())
    r_tuned = g.iterate()  # tuning left the state as it was
    g.close()
    r_default = rpba.Rpba(prob, **OPTS).iterate()
    g2 = rpba.Rpba(prob, tune_cache=str(cache), **OPTS)  # reads the cached shapes
    r_cached = g2.iterate()
    g2.close()
    for r in (r_tuned, r_cached):
        assert r["outer"] == r_default["outer"]
        np.testing.assert_allclose(r["sigma0_hist"], r_default["sigma0_hist"], rtol=1e-9)
        assert r["rms"] == pytest.approx(r_default["rms"], rel=1e-9)
    # tuning again for the same workload replaces its line
    g3 = rpba.Rpba(prob, **OPTS)
    g3.intersect()
    g3.tune(str(cache))
    assert len([ln for ln in cache.read_text().splitlines() if ln.strip()]) == 1
    g3.close()
