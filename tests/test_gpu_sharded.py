"""The sharded loop (paper_1910_08138_gb300/sharding.py) over this library's
contexts on the GPU.

One rank: the loop with a single context equals rpba_iterate's run (FP64 form,
to rounding: the FP64 Schur assembly sums with atomics). Two ranks: two
contexts on the one GPU, each adjusting its share of the sub-blocks under the
sub-block and point masks, driven by two host threads that exchange cameras,
TP records and weights through queues between launches (no kernel waits on
another); the result follows the FP64 oracle's single-process trajectory.
"""

import queue
import threading

import numpy as np
import pytest

import oracle
from paper_1910_08138_gb300 import sharding, synth

pytestmark = pytest.mark.gpu


class ThreadComm:
    """The sharded loop's collectives between ranks that are threads of one
    process: point-to-point messages through queues, the all-reduce summed in
    rank order."""

    def __init__(self, rank, world, shared):
        self.rank, self.world, self.sh = rank, world, shared

    def exchange(self, send, recv_sizes):
        for d, a in send.items():
            self.sh["q"][(self.rank, d)].put(np.array(a, dtype=np.float64))
        out = {}
        for s, n in recv_sizes.items():
            a = self.sh["q"][(s, self.rank)].get(timeout=120)
            assert a.size == n
            out[s] = a
        return out

    def _reduce(self, a, op):
        self.sh["slots"][self.rank] = np.asarray(a, dtype=np.float64)
        self.sh["barrier"].wait(timeout=120)
        vals = [self.sh["slots"][r] for r in range(self.world)]
        res = vals[0].copy()
        for v in vals[1:]:
            res = op(res, v)
        self.sh["barrier"].wait(timeout=120)
        return res

    def allreduce_sum(self, a):
        return self._reduce(a, np.add)

    def allreduce_max(self, a):
        return self._reduce(a, np.maximum)


def test_one_rank_equals_the_library_loop():
    prob = synth.config(1)
    ref = sharding.RpbaEngine(prob, precision=0, solver=0, robust=1, robust_from_start=1)
    r_ref = ref.ctx.iterate()
    eng = sharding.RpbaEngine(prob, precision=0, solver=0, robust=1, robust_from_start=1)
    rep = sharding.run_sharded(eng, sharding.ShardPlan(prob, 1, 0), sharding.SoloComm())
    assert rep["outer"] == r_ref["outer"]
    np.testing.assert_allclose(rep["sigma0_hist"], r_ref["sigma0_hist"], rtol=1e-9)
    assert rep["sigma0"] == pytest.approx(r_ref["sigma0"], rel=1e-9)
    np.testing.assert_allclose(eng.ctx.cameras(), ref.ctx.cameras(), rtol=0, atol=1e-8)
    for e in (ref, eng):
        e.close()


def test_two_ranks_on_one_gpu_follow_the_oracle():
    prob = synth.tiny(seed=8, nx=6, ny=4, n_points=300, opp=4, runs=[8, 6, 6, 4], oblique_deg=30,
                      nadir_every=3, outlier_frac=0.03, extent=(-12.0, 12.0, -8.0, 8.0))
    ref = oracle.Oracle(prob).run(robust=1, robust_from_start=1)
    world = 2
    shared = {"q": {(a, b): queue.Queue() for a in range(world) for b in range(world)},
              "slots": [None] * world, "barrier": threading.Barrier(world)}
    engines = [sharding.RpbaEngine(prob, precision=0, solver=0, robust=1, robust_from_start=1)
               for _ in range(world)]
    plans = [sharding.ShardPlan(prob, world, r) for r in range(world)]
    reps, errs = [None] * world, []

    def rank_main(r):
        try:
            reps[r] = sharding.run_sharded(engines[r], plans[r], ThreadComm(r, world, shared))
        except Exception as e:  # surfaced by the main thread
            errs.append(e)

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    for rep in reps:
        assert rep["outer"] == ref["outer"]
        np.testing.assert_allclose(rep["sigma0_hist"], ref["sigma0_hist"], rtol=1e-6)
    # each rank adjusted only its own sub-blocks: its cameras are the ones the
    # other rank received
    rt = [e.cameras() for e in engines]
    for r in range(world):
        own = plans[r].own_cams
        np.testing.assert_array_equal(rt[0][own], rt[1][own])
    for e in engines:
        e.close()
