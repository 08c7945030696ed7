"""Writes tests/golden/oracle_targets.json: the FP64 oracle's final state
summary (RMS, sigma_0, iterations, deletions) on the benchmark blocks, with
the options the benchmark uses (robust stage from the first intersection).

Run: python -m oracle.make_targets [configs...]   (calls only the oracle)
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1910_08138_gb300 import synth  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "oracle_targets.json")
OPTIONS = dict(robust=1, robust_from_start=1)


def main(configs):
    for c in configs:
        prob = synth.config(c)
        t0 = time.perf_counter()
        rep = oracle.Oracle(prob).run(**OPTIONS)
        dt = time.perf_counter() - t0
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}  # written after every block
        data[f"config{c}"] = {"rms": rep["rms"], "sigma0": rep["sigma0"], "outer": rep["outer"],
                              "inner_total": rep["inner_total"], "deleted_points": rep["deleted_points"],
                              "active_obs": rep["active_obs"], "options": OPTIONS,
                              "oracle_seconds_single_thread": round(dt, 1),
                              "source": "oracle/make_targets.py (FP64 CPU oracle)"}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(c, data[f"config{c}"], flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2])
