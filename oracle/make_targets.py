"""Writes tests/golden/oracle_targets.json: the FP64 oracle's final state
summary (RMS, sigma_0, iterations, deletions) on the benchmark blocks, with
the options the benchmark uses (robust stage from the first intersection).

Run: python -m oracle.make_targets [config[@scale][/max_outer] ...]   (calls only the oracle)
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


def _parse(arg):
    """'4' -> (4, 1.0, 0); '4@0.1' -> block 4 with point counts scaled by 0.1;
    '4@0.1/4' -> the same, stopped after 4 outer iterations."""
    arg, _, outer = arg.partition("/")
    c, _, scale = arg.partition("@")
    return int(c), float(scale) if scale else 1.0, int(outer) if outer else 0


def key(c, scale=1.0, max_outer=0):
    k = f"config{c}" if scale == 1.0 else f"config{c}@{scale:g}"
    return k + (f"/outer{max_outer}" if max_outer else "")


def main(configs):
    for arg in configs:
        c, scale, max_outer = _parse(str(arg))
        prob = synth.config(c, scale=scale)
        t0 = time.perf_counter()
        opts = dict(OPTIONS, max_outer=max_outer) if max_outer else OPTIONS
        rep = oracle.Oracle(prob).run(**opts)
        dt = time.perf_counter() - t0
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}  # written after every block
        data[key(c, scale, max_outer)] = {"rms": rep["rms"], "sigma0": rep["sigma0"], "outer": rep["outer"],
                              "inner_total": rep["inner_total"], "deleted_points": rep["deleted_points"],
                              "active_obs": rep["active_obs"], "options": opts,
                              "oracle_seconds_single_thread": round(dt, 1),
                              "source": "oracle/make_targets.py (FP64 CPU oracle)"}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(arg, data[key(c, scale, max_outer)], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["1", "2"])
