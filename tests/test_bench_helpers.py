"""Host-side pieces of the benchmark: the algorithmic work counts that its
roofline divides by and the observation count of its metric, checked against
brute force on small blocks; the clock summary; the threaded CPU baseline
(one host thread per sub-block gives the sequential result); the reference
arm's JSON line."""

import argparse
import contextlib
import io
import itertools
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import oracle  # noqa: E402
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


def test_counted_observations_are_those_of_active_points():
    prob = synth.config(1)
    rng = np.random.default_rng(0)
    act = (rng.random(prob["points"].shape[0]) < 0.7).astype(np.uint8)
    brute = sum(1 for j in prob["obs_point"] if act[j])
    assert bench.counted_obs(prob, act) == brute


class _Ctx:
    """solver_stats / solver_stages of a context, from given arrays."""

    def __init__(self, iters, stages):
        self.iters, self.stages = np.asarray(iters, np.int32), np.asarray(stages, np.int32)

    def solver_stats(self):
        return self.iters, np.zeros(self.iters.size)

    def solver_stages(self):
        return self.stages


def _brute_tiles(n):
    T = -(-n // 32)
    return sum(1 for a in range(T) for b in range(T) if b <= a)


def test_pcg_bytes_are_the_stored_lower_tiles_of_live_sub_blocks():
    """Every 32 x 32 lower tile (diagonal included) of the padded RCS of a
    sub-block is read once per CG step it ran (FP32 form: 4 B per entry, S
    rounded to FP32; FP64 form: 8 B) and, in the FP32 form, once per
    refinement stage in hi + lo (8 B per entry)."""
    n_sub = [6 * 25, 6 * 7, 8 * 40]
    iters, stages = [5, 2, 9], [2, 1, 3]
    ctx = _Ctx(iters, stages)
    w = bench.pcg_work(ctx, n_sub, 1)
    t32 = sum(i * _brute_tiles(n) for i, n in zip(iters, n_sub))
    tff = sum(s * _brute_tiles(n) for s, n in zip(stages, n_sub))
    assert w["k_pcg_symv32"] == (t32 * 32 * 32 * 4, t32)
    assert w["k_pcg_symv_ff"] == (tff * 32 * 32 * 8, tff)
    w64 = bench.pcg_work(ctx, n_sub, 0)
    assert w64 == {"k_pcg_symv": (t32 * 32 * 32 * 8, t32)}
    acc = {}
    bench.add_work(acc, w)
    bench.add_work(acc, w)
    assert acc["k_pcg_symv32"] == (2 * t32 * 32 * 32 * 4, 2 * t32)


def test_clock_summary_median_max_and_reasons():
    lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
             "1980, 2070, 1200.0, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 1000.0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    c = bench.summarise_clocks(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    c = bench.summarise_clocks(["1400, 2070, 500, Active, Not Active, Active, Not Active"])
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and c["sm_mhz"] == 1400.0


def test_threaded_oracle_lm_iteration_equals_sequential():
    """The CPU baseline runs one host thread per sub-block (the paper's
    scheme): the state after a threaded LM iteration of all sub-blocks is the
    sequential one, bit for bit."""
    prob = synth.tiny(seed=4, nx=4, ny=4, n_points=200, runs=[4, 4, 4, 4])
    a, per_a, k_a = bench.oracle_setup(prob)
    b, per_b, k_b = bench.oracle_setup(prob)
    assert k_a == k_b and a.L == 4
    for _ in range(3):
        bench.oracle_lm_iteration(a, list(range(a.L)), 1)
        bench.oracle_lm_iteration(b, list(range(b.L)), 4)
    np.testing.assert_array_equal(a.cameras(), b.cameras())
    np.testing.assert_array_equal(a.instance_state()[0], b.instance_state()[0])


def test_reference_arm_prints_one_line_with_the_contract_keys():
    args = argparse.Namespace(gpus=1, steps=2, warmup=1, impl="reference", config=1, precision=1, solver=4,
                              no_extras=False)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, 0, 1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "obs/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the reference arm counts the observations of the points the oracle keeps
    o = oracle.Oracle(synth.config(1))
    o.intersect()
    assert d["config"]["n_obs_block"] == bench.counted_obs(synth.config(1), o.points()[1])


def test_tie_point_counts_by_brute_force():
    prob = synth.config(1)
    rng = np.random.default_rng(1)
    act = (rng.random(prob["points"].shape[0]) < 0.8).astype(np.uint8)
    subs_of = {}
    for c, j in zip(prob["obs_cam"], prob["obs_point"]):
        subs_of.setdefault(int(j), set()).add(int(prob["cam_subblock"][c]))
    tps = {j for j, s in subs_of.items() if len(s) >= 2 and act[j]}
    n_obs = sum(1 for j in prob["obs_point"] if int(j) in tps)
    n_inst = sum(len(subs_of[j]) for j in tps)
    assert bench.tie_point_counts(prob, act) == (len(tps), n_obs, n_inst)
