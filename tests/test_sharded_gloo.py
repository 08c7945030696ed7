"""The method sharded by sub-block over CPU ranks (gloo), against the
single-process FP64 oracle.

Each rank holds the whole block in an oracle context but adjusts only its
sub-blocks, intersects only the points it owns and computes the robust
weights only of its cameras; the exchange of Sec. 5 connects them: an
all-gather of the camera poses, the owners' (X_TP, active, W^l) records to the
ranks holding the TPs' sub-blocks, the TP observations' robust weights to the
TPs' owners, and sigma_0 as an all-reduce of partial sums. The cameras, the
points and the active flags must equal the single-process run's bit for bit;
sigma_0 (summed in another order) to 1e-13.
"""

import os
import socket
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1910_08138_gb300 import sharding, synth  # noqa: E402


class OracleEngine:
    """The sharded loop's engine over one FP64 oracle context."""

    def __init__(self, prob):
        self.o = oracle.Oracle(prob)
        self.obs_point = np.asarray(prob["obs_point"], dtype=np.int64)
        w = prob.get("obs_winv")
        self.winv = None if w is None else np.asarray(w, dtype=np.float64)
        ip, _ = self.o.instances()
        self.inst_point = ip.astype(np.int64)

    def intersect(self, ids, tp_only):
        self.o.intersect_points(np.asarray(ids, dtype=np.int32), tp_only)

    def bact(self, subs):
        for l in subs:
            self.o.sub_lm(int(l))

    def robust_weights(self, cams, t_v, downweight):
        self.o.robust_weights_cams(np.asarray(cams, dtype=np.int32), t_v, downweight)

    def cameras(self):
        rt = self.o.camera_rt()
        if self.o.cd == 8:  # per-camera intrinsics travel with the camera
            rt = np.concatenate([rt, self.o.intrinsics()], axis=1)
        return rt

    def set_cameras(self, rt):
        self.o.set_camera_rt(rt[:, :12])
        if rt.shape[1] == 14:
            self.o.set_intrinsics(rt[:, 12:])

    def points(self):
        return self.o.points()

    def set_points(self, X, act):
        self.o.set_points(X, act)

    def instance_state(self):
        return self.o.instance_state()

    def set_instance_state(self, Xl, Wl):
        self.o.set_instance_state(Xl, Wl)

    def weights(self):
        return self.o.weights()

    def set_weights(self, w):
        self.o.set_weights(w)

    def residuals(self):
        return self.o.residuals()


PROBS = {
    "cfg1": lambda: synth.config(1),
    # four uneven sub-blocks, oblique views and 3 % outliers
    "tiny4": lambda: synth.tiny(seed=8, nx=6, ny=4, n_points=300, opp=4, runs=[8, 6, 6, 4], oblique_deg=30,
                                nadir_every=3, outlier_frac=0.03, extent=(-12.0, 12.0, -8.0, 8.0)),
    # per-camera intrinsics (8 unknowns per camera), 4 arcs of a ring
    "ring4": lambda: synth.tiny_intrinsics(seed=8, n_cams=20, n_points=250, mean_track=5.0, n_sub=4,
                                           outlier_frac=0.02),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, opts, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = PROBS[name]()
    eng = OracleEngine(prob)
    plan = sharding.ShardPlan(prob, world, rank)
    rep = sharding.run_sharded(eng, plan, sharding.Comm(), **opts)
    X, act = eng.points()
    np.savez(os.path.join(out, f"rank{rank}.npz"), cams=eng.cameras(), X=X, act=act, own_pts=plan.own_pts,
             own_cams=plan.own_cams, hist=np.array(rep["sigma0_hist"]), s0=rep["sigma0"],
             outer=rep["outer"], sent=plan.exchange_bytes())
    dist.destroy_process_group()


def _run_ranks(world, name, opts):
    import torch.multiprocessing as mp
    out = tempfile.mkdtemp()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, opts, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return [dict(np.load(os.path.join(out, f"rank{r}.npz"))) for r in range(world)]


def _assemble(res):
    """Each rank's cameras and owned points make up the global state."""
    cams = res[0]["cams"].copy()
    X = res[0]["X"].copy()
    act = res[0]["act"].copy()
    for r in res:
        cams[r["own_cams"]] = r["cams"][r["own_cams"]]
        X[r["own_pts"]] = r["X"][r["own_pts"]]
        act[r["own_pts"]] = r["act"][r["own_pts"]]
    return cams, X, act


@pytest.mark.parametrize("name,world", [("cfg1", 2), ("tiny4", 2), ("tiny4", 3), ("ring4", 2)])
def test_sharded_run_equals_single_process_run(name, world):
    opts = dict(robust=True, robust_from_start=True)
    prob = PROBS[name]()
    o = oracle.Oracle(prob)
    ref = o.run(robust=1, robust_from_start=1)
    Xo, ao = o.points()
    res = _run_ranks(world, name, opts)
    cams, X, act = _assemble(res)
    exp = o.camera_rt() if o.cd == 6 else np.concatenate([o.camera_rt(), o.intrinsics()], axis=1)
    np.testing.assert_array_equal(cams, exp)
    np.testing.assert_array_equal(act, ao)
    np.testing.assert_array_equal(X[ao == 1], Xo[ao == 1])
    for r in res:
        # every rank ran the same loop: same outer count, same sigma_0 history
        assert int(r["outer"]) == ref["outer"]
        np.testing.assert_allclose(r["hist"], ref["sigma0_hist"], rtol=1e-13)
        assert float(r["s0"]) == pytest.approx(ref["sigma0"], rel=1e-13)
        assert int(r["sent"]) > 0


def test_plan_partitions_everything_once():
    prob = PROBS["tiny4"]()
    plans = [sharding.ShardPlan(prob, 3, r) for r in range(3)]
    for attr, n in (("own_subs", 4), ("own_cams", prob["cam_pose"].shape[0]),
                    ("own_obs", prob["obs_cam"].size), ("own_pts", prob["points"].shape[0])):
        allv = np.concatenate([getattr(p, attr) for p in plans])
        assert allv.size == n and np.unique(allv).size == n, attr
    # what one rank sends is what its peer expects
    for a in plans:
        for b in plans:
            if a.rank == b.rank:
                continue
            np.testing.assert_array_equal(a.tp_send[b.rank], b.tp_recv[a.rank])
            np.testing.assert_array_equal(a.tpi_send[b.rank], b.tpi_recv[a.rank])
            np.testing.assert_array_equal(a.w_send[b.rank], b.w_recv[a.rank])
    # the loop's exchange moves only tie points and their instances and
    # observations (Sec. 5: all cameras, only the TPs)
    for a in plans:
        for d in a.tp_send:
            assert a.is_tp[a.tp_send[d]].all() and a.is_tp[a.inst_point[a.tpi_send[d]]].all()
            assert a.is_tp[np.asarray(prob["obs_point"])[a.w_send[d]]].all()
    # a single rank owns everything and sends nothing
    solo = sharding.ShardPlan(prob, 1, 0)
    assert solo.exchange_bytes() == 0 and solo.own_subs.size == 4


def test_world_one_equals_single_process_run():
    prob = PROBS["tiny4"]()
    o = oracle.Oracle(prob)
    ref = o.run(robust=1, robust_from_start=1)
    eng = OracleEngine(prob)
    rep = sharding.run_sharded(eng, sharding.ShardPlan(prob, 1, 0), sharding.SoloComm())
    np.testing.assert_array_equal(eng.cameras(), o.camera_rt())
    assert rep["outer"] == ref["outer"]
