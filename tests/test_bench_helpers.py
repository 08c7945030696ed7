"""Host-side pieces of the benchmark: the algorithmic work counts that its
roofline divides by, checked against brute force on a small block."""

import itertools
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1910_08138_gb300 import synth  # noqa: E402


def test_schur_pair_count_is_the_pairs_inside_each_point_instance():
    prob = synth.config(1)
    sub = prob["cam_subblock"][prob["obs_cam"]]
    pairs = 0
    for j in np.unique(prob["obs_point"]):
        subs = sub[prob["obs_point"] == j]
        for l in np.unique(subs):
            n = int((subs == l).sum())
            pairs += sum(1 for _ in itertools.combinations(range(n), 2))
    assert bench.schur_pairs(prob) == pairs


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
    assert bench.FP32_PEAK_TFLOPS == 152 * 128 * 2 * 2.070e9 / 1e12
