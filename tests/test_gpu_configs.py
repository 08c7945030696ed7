"""Every benchmark block, whole runs, against the FP64 oracle's stored result.

The oracle's final RMS on each block (tests/golden/oracle_targets.json,
written by oracle/make_targets.py, which calls only the oracle) is the target:
the chosen form (FP32 bulk, auto solver) and the plain all-FP64 form must each
end within 1e-3 px of it, run the way the benchmark's time-to-RMS leg runs
them (robust weights from the first intersection on, up to 20 LM iterations
per sub-block and outer iteration; a run that stops above the target may
continue for up to 10 more outer iterations).
"""

import json
import os

import pytest

from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu

TARGETS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_targets.json")))
FORMS = {"chosen": (1, 4), "plain": (0, 0)}


@pytest.fixture(scope="module", params=[2, 3, 4, 5, 6])
def block(request):
    return request.param, synth.config(request.param)


@pytest.mark.parametrize("form", list(FORMS))
def test_block_reaches_the_oracle_rms(block, form):
    c, prob = block
    target = TARGETS[f"config{c}"]
    precision, solver = FORMS[form]
    g = rpba.Rpba(prob, precision=precision, solver=solver, robust=1, robust_from_start=1, max_inner=20)
    rep = g.iterate()
    outer = rep["outer"]
    extra = 0
    while rep["rms"] > target["rms"] + 1e-3 and extra < 10:
        rep = g.iterate(1)
        extra += 1
    g.close()
    assert abs(rep["rms"] - target["rms"]) <= 1e-3, (c, form, rep["rms"], target["rms"], outer, extra)
