#!/usr/bin/env python
"""Benchmark of the RPBA hot path on GB300 (one JSON line on stdout).

Workload (default): the 10,000-camera / 4M-point / 20M-observation block with
64 sub-blocks, nadir + 45 deg oblique wide-baseline views, 1 px noise, 5 %
outliers (seeded synthetic data; --config selects the smaller blocks).

A step is one pass of the whole hot path over that block: one steady-state
outer iteration of the method, i.e. one lock-step Levenberg-Marquardt
iteration of every sub-block (residuals, Jacobians, normal equations with the
TP control term, Schur complement, RCS solve, back-substitution, trial cost,
accept/reject), the exchange, the robust weights (per-camera MAD) and the
intersection of all tie points with their covariance-derived weights, and
sigma_0. value = observations per second per LM iteration, where the
observations counted are those active after the first (FP64) intersection,
the same number in both arms.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead (one LM iteration of as many sub-blocks as there are host
cores, one thread per sub-block, per step).
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to oracle-matched RMS (s) & obs/s per LM iter, chosen vs plain form"
WORKLOADS = {
    1: "rpba-50cam-2kpt-8kobs-2sub (10x5 nadir grid, 0.5px, 2% outliers)",
    2: "rpba-1000cam-100kpt-600kobs-8sub (25x40 grid, nadir+30deg oblique, 0.5px, 2% outliers)",
    3: "rpba-64blocks-7748cam-222kpt-1.0Mobs-304sub (20..400 cams/block, 2..8 sub-blocks, 0.5px, 2% outliers)",
    4: "rpba-5000cam-1Mpt-3.4Mobs-32sub (50x100 strips, 60% forward / 30% side overlap, 0.5px, 5% outliers)",
    5: "rpba-10000cam-4Mpt-20Mobs-64sub (100x100 grid, nadir+45deg oblique wide baseline, 1px, 5% outliers)",
    6: "rpba-961cam-187kpt-3.4Mobs-12sub-intrinsics (ring around an object, focal length and k1 per camera, "
       "18 obs/point, 1px, 2% outliers; stand-in for Final 961)",
}
DEFAULT_CONFIG = 5
TARGETS = os.path.join(ROOT, "tests", "golden", "oracle_targets.json")
FORMS = {"chosen": (1, 4), "plain": (0, 0)}  # (precision, solver); solver 4 = auto
TTR_REPEATS = 3  # fresh runs per form for the time to the oracle's RMS (median reported)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=DEFAULT_CONFIG)
    p.add_argument("--precision", type=int, default=1)
    p.add_argument("--solver", type=int, default=4)
    p.add_argument("--chol-tc", type=int, default=0,
                   help="direct solver's FP32 factorisation: 0 CUDA cores, 1 tensor cores per step, 2 persistent")
    p.add_argument("--tune", action="store_true", help="autotune the launch shapes on the block before timing")
    p.add_argument("--no-extras", action="store_true", help="skip e2e / time-to-RMS / cpu legs")
    p.add_argument("--clock-ms", type=int, default=50,
                   help="nvidia-smi sampling interval during the timed region (0: no sampling)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# host description
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, interval_ms=10):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []  # (host time, line)

    def start(self):
        """Starts the query loop and returns once its first sample arrived
        (nvidia-smi takes a moment to start), so that the timed region that
        follows is sampled from its beginning."""
        if self.interval_ms <= 0:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < t_end:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.perf_counter(), ln.strip()))

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between host times t0 and t1 (all
        when not given)."""
        if self.proc is None:
            why = "not sampled" if self.interval_ms <= 0 else "nvidia-smi unavailable"
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lo = -np.inf if t0 is None else t0
        hi = np.inf if t1 is None else t1 + self.interval_ms / 1e3
        return summarise_clocks([ln for t, ln in self.lines if lo <= t <= hi])


def summarise_clocks(lines):
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 7:
            continue
        try:
            sm.append(float(f[0]))
            smax.append(float(f[1]))
        except ValueError:
            continue
        for n, v in zip(names, f[3:7]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": float(np.median(sm)) if sm else None,
            "sm_max_mhz": float(max(smax)) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock
FP32_PEAK_SOURCE = "FP32 CUDA-core rate from 152 SMs x 128 lanes x 2 flops x 2070 MHz"

# DRAM bytes per unit of work from the ncu captures summarised under profiles/
# (dram__bytes_read.sum + dram__bytes_write.sum); a kernel is removed from this
# table when it changes after its capture
NCU_TRAFFIC_PER_UNIT = {
    # profiles/k_pcg_symv32_cfg4_5000cam.md: 60.673 + 0.210 MB over 14,688 lower tiles
    "k_pcg_symv32": ((60.673280 + 0.209920) * 1e6 / 14688, "tile", "profiles/k_pcg_symv32_cfg4_5000cam.md"),
}


def schur_pairs(prob):
    """Point pairs of the Schur complement: sum over point instances (point,
    sub-block) of n (n - 1) / 2, n the instance's observations."""
    sub = np.asarray(prob["cam_subblock"])[np.asarray(prob["obs_cam"])].astype(np.int64)
    key = np.asarray(prob["obs_point"]).astype(np.int64) * (int(sub.max()) + 1) + sub
    _, n = np.unique(key, return_counts=True)
    return float(np.sum(n * (n - 1) // 2))


def tie_point_counts(prob, active):
    """Active tie points (points seen in two or more sub-blocks), their
    observations and their instances: what the TP intersection reads."""
    cam_sub = np.asarray(prob["cam_subblock"]).astype(np.int64)
    op = np.asarray(prob["obs_point"]).astype(np.int64)
    sub = cam_sub[np.asarray(prob["obs_cam"])]
    N = int(np.asarray(prob["points"]).shape[0])
    key = np.unique(op * (int(sub.max()) + 1) + sub)
    n_inst = np.bincount(key // (int(sub.max()) + 1), minlength=N)
    tp = (n_inst >= 2) & (np.asarray(active) == 1)
    return int(tp.sum()), int(tp[op].sum()), int(n_inst[tp].sum())


def obs_stream_bytes(has_winv):
    """Bytes per observation every FP32-form per-observation pass streams: the
    point and camera indices (4 + 4), the position hi + lo (8 + 8), the robust
    weight (4) and C^-1 when given (12)."""
    return 28 + (12 if has_winv else 0)


def kernel_models(K, N, P, M, has_winv, pairs, tps=None, cd=6):
    """Algorithmic bytes (HBM-bound kernels) or flops (ALU-bound) of one launch
    of each FP32-form kernel of the step, from the data it must read and write
    once: K observations, N points, P instances, M cameras with cd unknowns
    each (6, or 8 with per-camera intrinsics). Camera records are 128 B each.
    Lower bounds: a kernel that gathers the same word twice is charged once."""
    ob = obs_stream_bytes(has_winv)
    return {
        "k_obs_sigma_f": ("hbm", K * ob + N * 25 + M * 128),
        "k_cost_chunks_f": ("hbm", K * ob + P * 72 + M * 128),
        # the same with the sub-block's records staged: plus a 16-bit local camera index per observation
        "k_cost_groups_f": ("hbm", K * (ob + 2) + P * 72 + M * 128),
        "k_robust_weights_f": ("hbm", K * (ob + 12) + N * 25 + M * 132),
        "k_camera_mad_u32": ("hbm", K * ob + N * 25 + M * 136),
        # the TP intersection: the tie points' observations, positions and instances
        "k_isect_fused_f": ("hbm", (tps[1] * ob + tps[0] * 48 + tps[2] * 24 if tps else K * ob + N * 48 + P * 24)
                            + M * 128),
        "k_camera_blocks_f32": ("hbm", K * ob + P * 60 + M * (128 + 12 * cd * cd)),
        "k_linearize_f32": ("hbm", K * ob + P * 132 + M * 128),
        "k_backsub_f32": ("hbm", K * ob + P * 72 + M * (128 + 4 * cd)),
        # cd x cd product N_XC,a^T (Ninv N_XC,b) per point pair, Z = Ninv N_XC once per observation
        "k_schur_seg": ("alu", 6.0 * cd * cd * pairs + 18.0 * cd * K),
    }


def roofline_entry(name, launches, ms, bound, work, peaks, traffic=None, traffic_note=None):
    per_launch_s = ms / 1e3 / max(launches, 1)
    if bound == "alu":
        achieved = work / per_launch_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "peak_source": FP32_PEAK_SOURCE,
                "launches": launches, "avg_launch_ms": per_launch_s * 1e3}
    achieved = work / per_launch_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_note": traffic_note,
            "algorithmic_bytes": work,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if not peaks.get("fallback") else "fallback",
            "launches": launches, "avg_launch_ms": per_launch_s * 1e3}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def bench_options(precision, solver, max_inner):
    return dict(precision=precision, solver=solver, robust=1, robust_from_start=1, max_inner=max_inner)


def train_preconditioner(stream):
    """The learned preconditioner's weights, trained by the library's own
    kernels on the reduced camera systems of configs 1 and 2 (every sub-block
    after 0 and 1 outer iterations, damping 1e-4 and 1e-2), 300 Adam steps
    with new probes every step. Returns (weights, seconds)."""
    import torch

    from paper_1910_08138_gb300 import rpba, synth
    t0 = time.perf_counter()
    G = rpba.Gnn(seed=0)
    for cfg in (1, 2):
        c = rpba.Rpba(synth.config(cfg), stream=stream, precision=0, solver=0, robust=1, robust_from_start=1)
        c.intersect()
        for k in range(2):
            for lam in (1e-4, 1e-2):
                G.add_rcs(c, lam, n_probes=4, seed=100 * cfg + 10 * k + int(lam * 1e4))
            c.iterate(1)
        c.close()
    G.train(300, lr=3e-4, probe_seed=7)
    w = G.weights()
    G.close()
    torch.cuda.synchronize()
    return w, time.perf_counter() - t0


def counted_obs(prob, active):
    """Observations of active points: the work unit of the metric."""
    return int(np.asarray(active)[np.asarray(prob["obs_point"])].astype(bool).sum())


# ---------------------------------------------------------------------------
# the FP64 CPU oracle (reference arm and CPU baseline)
# ---------------------------------------------------------------------------
def oracle_setup(prob):
    """The oracle after its first intersection (untimed) and the observations
    of active points per sub-block."""
    import oracle
    o = oracle.Oracle(prob)
    o.intersect()
    _, act = o.points()
    sub_of_obs = np.asarray(prob["cam_subblock"])[np.asarray(prob["obs_cam"])]
    active_obs = act[np.asarray(prob["obs_point"])] == 1
    per_sub = np.bincount(sub_of_obs[active_obs], minlength=o.L)
    return o, per_sub, int(active_obs.sum())


def oracle_lm_iteration(o, subs, threads, lam=1e-4):
    """One LM iteration of the listed sub-blocks, one host thread per
    sub-block (the paper's scheme; the oracle's step of sub-block l touches
    only l's cameras and instances, so the result equals the sequential
    run's). Returns seconds."""
    t0 = time.perf_counter()
    if threads <= 1 or len(subs) <= 1:
        for l in subs:
            o.lm_step(int(l), lam)
    else:
        with cf.ThreadPoolExecutor(max_workers=min(threads, len(subs))) as ex:
            list(ex.map(lambda l: o.lm_step(int(l), lam), subs))
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    from paper_1910_08138_gb300 import synth
    if rank != 0:
        return
    prob = synth.config(args.config)
    o, per_sub, k_work = oracle_setup(prob)
    threads = host_cores()
    # each step: one LM iteration of `threads` sub-blocks in parallel, cycling
    # through the block's sub-blocks from step to step
    order = [l for l in range(o.L) if per_sub[l] > 0]
    pos = 0

    def step():
        nonlocal pos
        subs = [order[(pos + a) % len(order)] for a in range(min(threads, len(order)))]
        pos = (pos + len(subs)) % len(order)
        return oracle_lm_iteration(o, subs, threads), int(sum(per_sub[l] for l in subs))

    for _ in range(max(args.warmup, 0)):
        step()
    times, kk = [], []
    for _ in range(args.steps):
        dt, k = step()
        times.append(dt)
        kk.append(k)
    ms = 1e3 * float(np.mean(times))
    value = float(np.sum(kk)) / float(np.sum(times))
    sample = (f"per step one LM iteration of {min(threads, len(order))} of the {len(order)} sub-blocks "
              f"(one host thread each, cycling through the block), FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "obs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "n_obs_block": k_work, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "obs/s", "cores": min(threads, len(order)), "kind": "oracle",
                             "sample": sample, "nproc": host_cores(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "obs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_full_step(prob, threads):
    """The CPU baseline in our arm: the oracle's whole step on the same block
    (one LM iteration of every sub-block, one host thread per sub-block up to
    the core count; then the robust weights, the TP intersection and sigma_0,
    single-threaded as the oracle is written). Returns (seconds, observations,
    description)."""
    o, per_sub, k_work = oracle_setup(prob)
    subs = [l for l in range(o.L) if per_sub[l] > 0]
    t0 = time.perf_counter()
    oracle_lm_iteration(o, subs, threads)
    t_lm = time.perf_counter() - t0
    o.robust_weights()
    o.intersect(tp_only=True)
    o.sigma0()
    dt = time.perf_counter() - t0
    what = (f"one whole step of the FP64 oracle: LM iteration of all {len(subs)} sub-blocks on "
            f"{min(threads, len(subs))} threads ({t_lm:.1f} s), then robust weights, TP intersection and "
            f"sigma_0 on one thread ({dt - t_lm:.1f} s)")
    return dt, k_work, what


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def replicas_aggregate(total_ms, obs_per_step, steps, world, device):
    """N independent replicas of the block (weak scaling, no collective on the
    data path): the job's time is the slowest rank's, its work that of all
    ranks. Returns (total_ms, obs/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return total_ms, world * obs_per_step * steps / (total_ms / 1e3)


def pcg_work(ctx, n_sub, precision):
    """Algorithmic bytes of the RCS products in the context's last PCG solve,
    per kernel: {kernel: (bytes, lower-tile reads)}. In the FP32 form the CG
    product reads S rounded to FP32 (4 B per stored lower-tile entry) of every
    live sub-block once per CG step, and the refinement product reads the hi
    and lo planes (8 B) once per stage; the FP64 form's product reads the FP64
    S (8 B) once per CG step."""
    npad = [32 * ((n + 31) // 32) for n in n_sub]
    tiles = np.array([(n // 32) * (n // 32 + 1) // 2 for n in npad], dtype=np.float64)
    it = ctx.solver_stats()[0].astype(np.float64)
    if precision == 1:
        t32 = float(np.dot(it, tiles))
        tff = float(np.dot(ctx.solver_stages().astype(np.float64), tiles))
        return {"k_pcg_symv32": (t32 * 1024 * 4, t32), "k_pcg_symv_ff": (tff * 1024 * 8, tff)}
    t = float(np.dot(it, tiles))
    return {"k_pcg_symv": (t * 1024 * 8, t)}


def add_work(acc, work):
    for k, (b, t) in work.items():
        b0, t0 = acc.get(k, (0.0, 0.0))
        acc[k] = (b0 + b, t0 + t)


def run_ours(args, rank, world):
    import torch

    from paper_1910_08138_gb300 import rpba, synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    prob = synth.config(args.config)
    peaks = load_peaks()
    gnn_w, gnn_s = (train_preconditioner(stream) if args.solver == 3 else (None, None))
    ctx = rpba.Rpba(prob, stream=stream, chol_tc=args.chol_tc, **bench_options(args.precision, args.solver, 1))
    if gnn_w is not None:
        ctx.set_gnn_weights(gnn_w)
    ctx.intersect()
    tuned = ctx.tune() if args.tune else None
    _, act0 = ctx.points()
    K = counted_obs(prob, act0)  # the same count as the oracle's after its first intersection
    n_sub = [ctx.cd * len(ctx.sub_cameras(l)) for l in range(ctx.L)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        return ctx.outer_iteration(robust=True)

    # the last warm-up step times every kernel (the breakdown and the dominant
    # kernel); the timed steps time only the dominant kernel, so that event
    # records stay out of the rest of the step
    for _ in range(max(args.warmup - 2, 0)):
        step()
    ctx.profile_enable(True)
    flush.fill_(-1.0)
    step()
    prof_all, _ = ctx.profile_read()
    ctx.profile_enable(False)
    solver = ctx.resolved_options().solver
    work_warm = pcg_work(ctx, n_sub, args.precision) if solver in (1, 3) else {}
    dominant = max(prof_all.items(), key=lambda kv: kv[1][1])[0]
    # the next warm-up step already runs with the timed steps' profiling, so
    # that the graphs it captures (event nodes for the dominant kernel only)
    # are the ones the timed steps replay
    ctx.profile_enable(True)
    ctx.profile_select(dominant)
    if args.warmup >= 2:
        flush.fill_(-2.0)
        step()
    solver = ctx.resolved_options().solver
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctx.profile_enable(True)  # resets the counters; the selection stays
    ctx.profile_select(dominant)
    clocks = ClockSampler(dev, args.clock_ms)
    clocks.start()
    times = []
    work_timed = {}
    t_timed0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        if solver in (1, 3):
            add_work(work_timed, pcg_work(ctx, n_sub, args.precision))
            solver = ctx.resolved_options().solver
    clk = clocks.stop(t_timed0, time.perf_counter())
    prof, launches = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.profile_select(None)
    total_ms, value = replicas_aggregate(float(np.sum(times)), K, args.steps, world, "cuda")
    ms = total_ms / args.steps

    # rooflines: the dominant kernel over the timed region; the other hot
    # kernels from the fully event-timed last warm-up step
    has_winv = prob.get("obs_winv") is not None
    models = (kernel_models(K, ctx.N, ctx.P, ctx.M, has_winv, schur_pairs(prob), tie_point_counts(prob, act0),
                            cd=ctx.cd)
              if args.precision == 1 else {})

    def entry(name, launches_, ms_, work=None):
        # work: {kernel: (bytes, tile reads)} of the PCG products over the
        # launches timed (their bytes per launch follow from the launch count)
        if work and name in work:
            b, t = work[name]
            model, tiles_per = ("hbm", b / max(launches_, 1)), t / max(launches_, 1)
        else:
            model, tiles_per = models.get(name), None
        if model is None:
            return {"kernel": name, "bound": None, "achieved": None, "frac": None, "launches": launches_,
                    "avg_launch_ms": ms_ / max(launches_, 1)}
        bound, per_launch = model
        traffic, note = None, None
        if name in NCU_TRAFFIC_PER_UNIT and tiles_per:
            per, unit, src = NCU_TRAFFIC_PER_UNIT[name]
            traffic = per * tiles_per
            note = f"ncu DRAM bytes per {unit} ({src}) x {tiles_per:.0f} live tiles per launch"
        return roofline_entry(name, launches_, ms_, bound, per_launch, peaks, traffic, note)

    roof = entry(dominant, *prof.get(dominant, (0, 0.0)), work=work_timed)
    step_ms_all = sum(v[1] for v in prof_all.values())
    hot = []
    for name, (la, kms) in sorted(prof_all.items(), key=lambda kv: -kv[1][1]):
        if kms < 0.02 * step_ms_all:
            continue
        e = entry(name, la, kms, work=work_warm)
        e["share"] = kms / step_ms_all
        hot.append(e)
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4)}
               for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1][1])}
    solver_names = {0: "FP64 Cholesky", 1: "block-Jacobi PCG" + (" (FP32 CG stages, float-float refinement)" if args.precision == 1 else " (FP64)"),
                    2: "FP32 Cholesky + FP64 refinement", 3: "PCG, learned preconditioner"}
    line = {"metric": METRIC, "value": value, "unit": "obs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == 1 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config],
                       "precision": "mixed FP32/FP64" if args.precision == 1 else "FP64",
                       "solver": solver_names.get(solver)
                       + (" (auto: PCG for up to 64 sub-blocks while a solve takes at most 48 CG iterations,"
                          " else the direct solve)" if args.solver == 4 else ""),
                       "l2": "flushed between steps (256 MB write)", "n_obs": K,
                       "n_obs_note": "observations of points active after the first (FP64) intersection; the "
                                     "reference arm counts the same",
                       "subblocks": ctx.L,
                       "step": "1 steady-state outer iteration: 1 LM iteration of all sub-blocks + exchange + "
                               "robust weights + TP intersection + sigma_0",
                       "parallelism": f"replicas x{world}"},
            "step_ms_spread": {"min": float(np.min(times)), "median": float(np.median(times)),
                               "max": float(np.max(times))},
            "roofline": roof, "hot_kernels": hot, "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps, "clocks": clk,
            "kernels_last_warmup_step": kernels}
    if gnn_w is not None:
        line["config"]["preconditioner_training_s"] = round(gnn_s, 2)
    if tuned is not None:
        line["config"]["tuned_launch_shapes"] = tuned
    if rank == 0 and not args.no_extras:
        line.update(extras(args, prob, ctx, stream, K, gnn_w))
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def extras(args, prob, ctx, stream, K, gnn_w=None):
    import torch

    from paper_1910_08138_gb300 import rpba
    out = {}
    # e2e through the C ABI with host buffers in pinned memory: the state (poses,
    # points, active flags) H2D, one step, the state D2H
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    cams = pin((ctx.M, 6), torch.float64)
    X, act = pin((ctx.N, 3), torch.float64), pin((ctx.N,), torch.uint8)
    ctx.cameras(out=cams)
    ctx.points(out=(X, act))
    times = []
    for s in range(max(3, min(args.steps, 20) // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_cameras(cams)
        ctx.set_points(X, act)
        ctx.outer_iteration(robust=True)
        ctx.cameras(out=cams)
        ctx.points(out=(X, act))
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    h2d = cams.nbytes + X.nbytes + act.nbytes
    d2h = h2d
    out["e2e"] = {"value": K / float(np.mean(times)), "unit": "obs/s", "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * float(np.mean(times)),
                  "host_buffers": "pinned"}
    # time to the oracle's final RMS, chosen form vs plain all-FP64 form
    target = None
    try:
        target = json.load(open(TARGETS))[f"config{args.config}"]["rms"]
    except Exception:
        pass
    ttr = {}
    if target is None:
        out["time_to_oracle_rms"] = {"skipped": "no stored oracle RMS for this block"}
    for form, (prec, solver) in (() if target is None else
                                 (("chosen", (args.precision, args.solver)), ("plain", FORMS["plain"]))):
        runs = []
        for _ in range(TTR_REPEATS):  # a wall-clock time: the median of fresh runs
            g = rpba.Rpba(prob, stream=stream, **bench_options(prec, solver, 20))
            if solver == 3:
                g.set_gnn_weights(gnn_w)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.intersect()
            rep = g.iterate()
            own_rms, outer, lm = rep["rms"], rep["outer"], rep["lm_launches"]
            extra = 0
            # keep iterating the same process until the oracle's final RMS is met
            while target is not None and rep["rms"] > target + 1e-3 and extra < 10:
                rep = g.iterate(1)
                extra += 1
                outer += rep["outer"]
                lm += rep["lm_launches"]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            runs.append((dt, rep, own_rms, outer, lm, extra))
            g.close()
        runs.sort(key=lambda x: x[0])
        dt, rep, own_rms, outer, lm, extra = runs[len(runs) // 2]
        ttr[form] = {"seconds": dt, "seconds_all_runs": [round(x[0], 4) for x in runs], "final_rms": rep["rms"],
                     "own_convergence_rms": own_rms, "outer": outer,
                     "lm_iterations": lm, "deleted_points": rep["deleted_points"],
                     "extra_outer_after_own_convergence": extra,
                     "matches_oracle": (target is not None and rep["rms"] <= target + 1e-3)}
    if target is not None:
        ttr["oracle_final_rms"] = target
        if ttr["plain"]["seconds"] > 0:
            ttr["chosen_speedup_vs_plain"] = ttr["plain"]["seconds"] / ttr["chosen"]["seconds"]
        out["time_to_oracle_rms"] = ttr
    # CPU oracle: one whole step of the same block on the host cores
    threads = host_cores()
    dt, kk, what = oracle_full_step(prob, threads)
    out["cpu_baseline"] = {"value": kk / dt, "unit": "obs/s", "cores": min(threads, ctx.L), "kind": "oracle",
                           "sample": f"{what}; {kk} observations, {dt:.1f} s",
                           "nproc": host_cores(), "cpu_model": cpu_model()}
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
