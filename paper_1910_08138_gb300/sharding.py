"""RPBA sharded by sub-block over several ranks (one process per GPU).

The method's parallel structure (Sec. 5): every sub-block's adjustment
(Eq. bact) depends only on its own cameras, its point copies X^l and, for the
tie points (TPs), their current position X_TP and refined weight W^l. One
exchange step per outer iteration connects the sub-blocks: the cameras of all
sub-blocks go to every rank, only the TPs are intersected again (Eq. bars)
and their positions and weights go back to the ranks that adjust them. This
module runs that loop with the sub-blocks partitioned over the ranks:

* ShardPlan: sub-blocks to ranks (largest estimated cost first, to the least
  loaded rank), each point to an owner rank (the rank of its first sub-block),
  and the static routing of every exchange (which cameras, TP records and
  robust weights each rank sends to each other rank). Every rank computes the
  same plan from the problem's topology, so message sizes need not be sent.
* run_sharded: the outer loop of the method over an engine that holds the
  whole problem but advances only its rank's share:
    bact of the own sub-blocks -> exchange of the single-sub-block points ->
    all-gather of the cameras -> robust weights of the own cameras, the TP
    observations' weights to the TPs' owners -> owners intersect their TPs ->
    (X_TP, active, W^l) to the ranks holding the TPs' sub-blocks -> sigma_0 as
    an all-reduce of partial sums -> the stop rule of Sec. 5.5.
  The collectives are point-to-point sends and receives of float64 tensors
  (torch.distributed: gloo on the CPU, NCCL on GPUs) and one all-reduce.
* RpbaEngine: the engine over one GPU context of this library.

With the same engine arithmetic on every rank the result equals the
single-process run's: each sub-block's adjustment, each point's intersection
and each camera's robust scale see the same inputs as there. Only sigma_0 is
summed in a different order (partial sums per rank).
"""

from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# the plan
# ---------------------------------------------------------------------------
class ShardPlan:
    """Static partition and routing of one block over `world` ranks."""

    def __init__(self, prob, world: int, rank: int, inst_point=None, inst_sub=None):
        self.world, self.rank = int(world), int(rank)
        # camera unknowns: 6, or 8 with per-camera intrinsics (f and k1 travel
        # with each camera's rotation and translation)
        self.cd = 8 if prob.get("intrinsics", False) else 6
        cam_sub = np.asarray(prob["cam_subblock"], dtype=np.int64)
        obs_cam = np.asarray(prob["obs_cam"], dtype=np.int64)
        obs_pt = np.asarray(prob["obs_point"], dtype=np.int64)
        self.M, self.N, self.K = cam_sub.size, int(np.asarray(prob["points"]).shape[0]), obs_cam.size
        self.L = int(cam_sub.max()) + 1 if cam_sub.size else 0
        obs_sub = cam_sub[obs_cam]
        # sub-blocks to ranks: cost ~ observations + (6 M_l)^3 / 3 of its solve
        m_l = np.bincount(cam_sub, minlength=self.L).astype(np.float64)
        k_l = np.bincount(obs_sub, minlength=self.L).astype(np.float64)
        cost = k_l * 1000.0 + (float(self.cd) * m_l) ** 3 / 3.0
        load = np.zeros(self.world)
        self.sub_rank = np.zeros(self.L, dtype=np.int64)
        for l in sorted(range(self.L), key=lambda x: (-cost[x], x)):
            r = int(np.argmin(load))
            self.sub_rank[l] = r
            load[r] += cost[l]
        self.cam_rank = self.sub_rank[cam_sub]
        self.obs_rank = self.cam_rank[obs_cam]
        # instances (point, sub-block) in canonical order (sub-block, point)
        if inst_point is None:
            key = np.unique(obs_sub * self.N + obs_pt)
            inst_sub, inst_point = key // self.N, key % self.N
        self.inst_point = np.asarray(inst_point, dtype=np.int64)
        self.inst_sub = np.asarray(inst_sub, dtype=np.int64)
        self.P = self.inst_point.size
        n_inst = np.bincount(self.inst_point, minlength=self.N)
        self.is_tp = n_inst >= 2
        # owner of a point: the rank of its first (smallest id) sub-block
        first_sub = np.full(self.N, np.iinfo(np.int64).max)
        np.minimum.at(first_sub, self.inst_point, self.inst_sub)
        seen = first_sub < np.iinfo(np.int64).max
        self.pt_owner = np.where(seen, self.sub_rank[np.where(seen, first_sub, 0)], 0)
        r = self.rank
        self.own_subs = np.nonzero(self.sub_rank == r)[0]
        self.own_cams = np.nonzero(self.cam_rank == r)[0]
        self.own_obs = np.nonzero(self.obs_rank == r)[0]
        # points no sub-block sees belong to rank 0, which drops them in the
        # first intersection as the single-process run does
        self.own_pts = np.nonzero(self.pt_owner == r)[0]
        self.own_tps = self.own_pts[self.is_tp[self.own_pts]]
        inst_rank = self.sub_rank[self.inst_sub]
        self.own_inst = np.nonzero(inst_rank == r)[0]
        # points seen by each rank's sub-blocks
        seen_by = [np.unique(self.inst_point[inst_rank == d]) for d in range(self.world)]
        self.cams_of = [np.nonzero(self.cam_rank == d)[0] for d in range(self.world)]
        # point records (X, active, W^l of the receiver's instances): owner -> holders
        self.pt_send, self.pt_recv, self.inst_send, self.inst_recv = {}, {}, {}, {}
        self.tp_send, self.tp_recv, self.tpi_send, self.tpi_recv = {}, {}, {}, {}
        self.w_send, self.w_recv = {}, {}
        tp_obs = self.is_tp[obs_pt]
        for d in range(self.world):
            if d == r:
                continue
            # everything I own that d sees, and what d owns that I see
            self.pt_send[d] = seen_by[d][self.pt_owner[seen_by[d]] == r]
            self.pt_recv[d] = seen_by[r][self.pt_owner[seen_by[r]] == d]
            self.inst_send[d] = np.nonzero((inst_rank == d) & (self.pt_owner[self.inst_point] == r))[0]
            self.inst_recv[d] = np.nonzero((inst_rank == r) & (self.pt_owner[self.inst_point] == d))[0]
            # the TP subset (the loop's exchange)
            self.tp_send[d] = self.pt_send[d][self.is_tp[self.pt_send[d]]]
            self.tp_recv[d] = self.pt_recv[d][self.is_tp[self.pt_recv[d]]]
            self.tpi_send[d] = self.inst_send[d][self.is_tp[self.inst_point[self.inst_send[d]]]]
            self.tpi_recv[d] = self.inst_recv[d][self.is_tp[self.inst_point[self.inst_recv[d]]]]
            # robust weights of TP observations: camera's rank -> TP's owner
            self.w_send[d] = np.nonzero(tp_obs & (self.obs_rank == r) & (self.pt_owner[obs_pt] == d))[0]
            self.w_recv[d] = np.nonzero(tp_obs & (self.obs_rank == d) & (self.pt_owner[obs_pt] == r))[0]
        # instances of my sub-blocks whose point is a TP / a single-sub-block point
        self.own_tp_inst = self.own_inst[self.is_tp[self.inst_point[self.own_inst]]]
        self.own_single_inst = self.own_inst[~self.is_tp[self.inst_point[self.own_inst]]]

    def exchange_bytes(self):
        """Bytes this rank sends per outer iteration: its cameras (rotation
        matrix and translation, 12 doubles, with intrinsics also f and k1) to
        every other rank, its TPs' records (X_TP and the active flag: 4
        doubles, W^l: 6 per receiving instance) and the robust weights of TP
        observations (1 double each)."""
        b = 8 * (12 + self.cd - 6) * self.own_cams.size * (self.world - 1)
        for d in self.tp_send:
            b += 8 * (4 * self.tp_send[d].size + 6 * self.tpi_send[d].size + self.w_send[d].size)
        return b


# ---------------------------------------------------------------------------
# collectives
# ---------------------------------------------------------------------------
class Comm:
    """The exchange as torch.distributed point-to-point messages of float64
    tensors (sizes known to both sides from the plan) and an all-reduce.
    device: 'cpu' for gloo, a CUDA device for NCCL."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = device

    def exchange(self, send: dict, recv_sizes: dict) -> dict:
        """send: {dest: float64 array}; recv_sizes: {src: element count}.
        Returns {src: float64 array}."""
        import torch
        dist = self.dist
        ops, bufs = [], {}
        for s, n in sorted(recv_sizes.items()):
            if n:
                bufs[s] = torch.empty(int(n), dtype=torch.float64, device=self.device)
                ops.append(dist.P2POp(dist.irecv, bufs[s], s, self.group))
        for d, a in sorted(send.items()):
            if a.size:
                t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)
                ops.append(dist.P2POp(dist.isend, t, d, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return {s: (bufs[s].cpu().numpy() if s in bufs else np.zeros(0)) for s in recv_sizes}

    def allreduce_sum(self, a):
        import torch
        t = torch.as_tensor(np.asarray(a, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def allreduce_max(self, a):
        import torch
        t = torch.as_tensor(np.asarray(a, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t.cpu().numpy()


class SoloComm:
    """world size 1: no messages."""

    def exchange(self, send, recv_sizes):
        return {}

    def allreduce_sum(self, a):
        return np.asarray(a, dtype=np.float64)

    def allreduce_max(self, a):
        return np.asarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# the loop
# ---------------------------------------------------------------------------
def _exchange_cameras(engine, plan, comm):
    """All-gather of the cameras as held: rotation matrix and translation
    (12 doubles each; with intrinsics 14: f and k1 too), so that every rank
    holds the same bits."""
    rt = engine.cameras()
    width = rt.shape[1]
    send = {d: rt[plan.own_cams].reshape(-1) for d in range(plan.world) if d != plan.rank}
    sizes = {s: width * plan.cams_of[s].size for s in range(plan.world) if s != plan.rank}
    got = comm.exchange(send, sizes)
    for s, a in got.items():
        if a.size:
            rt[plan.cams_of[s]] = a.reshape(-1, width)
    engine.set_cameras(rt)


def _exchange_points(engine, plan, comm, pts_send, pts_recv, inst_send, inst_recv):
    """Owner -> holders: X (3), active (1) per point, W^l (6) per instance."""
    X, act = engine.points()
    Xl, Wl = engine.instance_state()
    send = {}
    for d in pts_send:
        p, q = pts_send[d], inst_send[d]
        send[d] = np.concatenate([X[p].reshape(-1), act[p].astype(np.float64), Wl[q].reshape(-1)])
    sizes = {s: 4 * pts_recv[s].size + 6 * inst_recv[s].size for s in pts_recv}
    got = comm.exchange(send, sizes)
    for s, a in got.items():
        p, q = pts_recv[s], inst_recv[s]
        if not a.size:
            continue
        X[p] = a[:3 * p.size].reshape(-1, 3)
        act[p] = a[3 * p.size:4 * p.size].astype(np.uint8)
        Wl[q] = a[4 * p.size:].reshape(-1, 6)
    engine.set_points(X, act)
    engine.set_instance_state(Xl, Wl)


def _exchange_weights(engine, plan, comm):
    """Robust weights of TP observations: camera's rank -> TP's owner."""
    w = engine.weights()
    send = {d: w[plan.w_send[d]] for d in plan.w_send}
    got = comm.exchange(send, {s: plan.w_recv[s].size for s in plan.w_recv})
    for s, a in got.items():
        if a.size:
            w[plan.w_recv[s]] = a
    engine.set_weights(w)


def _copies_from_points(engine, inst):
    """X^l = X_j for the listed instances (the TP copies restart at X_TP)."""
    X, _ = engine.points()
    Xl, Wl = engine.instance_state()
    Xl[inst] = X[engine.inst_point[inst]]
    engine.set_instance_state(Xl, Wl)


def _points_from_single_copies(engine, plan):
    """Points seen by one sub-block take that sub-block's copy (exchange)."""
    X, act = engine.points()
    Xl, _ = engine.instance_state()
    q = plan.own_single_inst
    j = engine.inst_point[q]
    keep = act[j] == 1
    X[j[keep]] = Xl[q[keep]]
    engine.set_points(X, act)


def _sigma0(engine, plan, comm):
    """sigma_0 (Eq. sigma0, weights C^-1): the weighted square sum over the
    observations of active points and their count, each rank over the
    observations of its cameras, the active points counted by their owners;
    r = 2 K - 6 M - 3 N + 7 (8 M with per-camera intrinsics)."""
    v = engine.residuals()
    w = engine.weights()
    _, act = engine.points()
    k = plan.own_obs
    a = act[engine.obs_point[k]] == 1
    k = k[a]
    W = engine.winv
    vv = v[k]
    if W is None:
        q = vv[:, 0] * vv[:, 0] + vv[:, 1] * vv[:, 1]
    else:
        Wk = W[k]
        q = Wk[:, 0] * vv[:, 0] * vv[:, 0] + 2.0 * Wk[:, 1] * vv[:, 0] * vv[:, 1] + Wk[:, 2] * vv[:, 1] * vv[:, 1]
    part = np.array([float(np.sum(w[k] * q)), float(k.size), float(np.sum(act[plan.own_pts] == 1))])
    tot = comm.allreduce_sum(part)
    red = max(2.0 * tot[1] - float(plan.cd) * plan.M - 3.0 * tot[2] + 7.0, 1.0)
    return float(np.sqrt(tot[0] / red))


def run_sharded(engine, plan, comm, robust=True, robust_from_start=True, stop_ratio=1.01, grace=1,
                max_outer=30, t_v=4.0, downweight=1e-4):
    """The RPBA outer loop (Sec. 5) over the rank's share of the block; the
    same sequence as the single-process loop: initial intersection, then per
    outer iteration bact, exchange, robust weights (when on), TP intersection
    and sigma_0 with the best/current stop rule (Sec. 5.5, one grace
    iteration); after the robust stage the points with a down-weighted
    observation are eliminated (Sec. 5.3). Returns a report dict."""
    rep = {"sigma0_hist": [], "outer": 0, "robust_started_at": -1}
    # initial intersection of every point by its owner, records to the holders
    engine.intersect(plan.own_pts, tp_only=False)
    _exchange_points(engine, plan, comm, plan.pt_send, plan.pt_recv, plan.inst_send, plan.inst_recv)
    _copies_from_points(engine, plan.own_inst)
    s = _sigma0(engine, plan, comm)
    rep["sigma0_initial"] = s
    best, g, robust_on = s, grace, False

    def robust_update():
        engine.robust_weights(plan.own_cams, t_v, downweight)
        _exchange_weights(engine, plan, comm)

    def tp_intersection():
        engine.intersect(plan.own_tps, tp_only=True)
        _exchange_points(engine, plan, comm, plan.tp_send, plan.tp_recv, plan.tpi_send, plan.tpi_recv)
        _copies_from_points(engine, plan.own_tp_inst)

    for _ in range(max_outer):
        engine.bact(plan.own_subs)
        _points_from_single_copies(engine, plan)
        _exchange_cameras(engine, plan, comm)
        if robust and robust_from_start and not robust_on:
            robust_on = True
            rep["robust_started_at"] = rep["outer"]
        if robust_on:
            robust_update()
        tp_intersection()
        s = _sigma0(engine, plan, comm)
        rep["sigma0_hist"].append(s)
        rep["outer"] += 1
        ratio = best / max(s, 1e-300)
        best = min(best, s)
        if ratio < stop_ratio:
            if g > 0:
                g -= 1
                continue
            if robust and not robust_on:
                robust_on = True
                rep["robust_started_at"] = rep["outer"]
                robust_update()
                tp_intersection()
                best = _sigma0(engine, plan, comm)
                g = grace
                continue
            break
    if robust_on:
        # a point with any down-weighted observation is eliminated; its
        # observations may sit on several ranks
        w = engine.weights()
        X, act = engine.points()
        k = plan.own_obs[(w[plan.own_obs] != 1.0) & (act[engine.obs_point[plan.own_obs]] == 1)]
        flag = np.zeros(plan.N)
        flag[engine.obs_point[k]] = 1.0
        flag = comm.allreduce_max(flag)
        act[flag > 0] = 0
        engine.set_points(X, act)
    rep["sigma0"] = _sigma0(engine, plan, comm)
    return rep


# ---------------------------------------------------------------------------
# the engine over one GPU context
# ---------------------------------------------------------------------------
class RpbaEngine:
    """One library context holding the whole block; the loop above tells it
    which sub-blocks to adjust (a sub-block mask) and which points to
    intersect (a point mask). State moves through the context's host get/set
    entry points."""

    def __init__(self, prob, **options):
        from . import rpba
        self.ctx = rpba.Rpba(prob, **options)
        self.obs_point = np.asarray(prob["obs_point"], dtype=np.int64)
        w = prob.get("obs_winv")
        self.winv = None if w is None else np.asarray(w, dtype=np.float64)
        ip, _ = self.ctx.instances()
        self.inst_point = np.asarray(ip, dtype=np.int64)

    def close(self):
        self.ctx.close()

    def intersect(self, ids, tp_only):
        mask = np.zeros(self.ctx.N, np.uint8)
        mask[np.asarray(ids, dtype=np.int64)] = 1
        self.ctx.set_point_mask(mask)
        if tp_only:
            self.ctx.intersect_points(True)
        else:
            self.ctx.intersect()  # the first intersection: FP64 in every form
        self.ctx.set_point_mask(None)

    def bact(self, subs):
        mask = np.zeros(self.ctx.L, np.uint8)
        mask[np.asarray(subs, dtype=np.int64)] = 1
        self.ctx.set_subblock_mask(mask)
        self.ctx.bact()
        self.ctx.set_subblock_mask(None)

    def robust_weights(self, cams, t_v, downweight):
        # the context computes every camera's scale and weights; the loop
        # replaces those of other ranks' observations before they are used
        self.ctx.robust_weights()

    def cameras(self):
        """(M, 12) rotation and translation as held; (M, 14) with f and k1
        when the context estimates intrinsics."""
        rt = self.ctx.camera_rt()
        if self.ctx.options.intrinsics:
            rt = np.concatenate([rt, self.ctx.intrinsics()], axis=1)
        return rt

    def set_cameras(self, rt):
        self.ctx.set_camera_rt(np.ascontiguousarray(rt[:, :12]))
        if rt.shape[1] == 14:
            self.ctx.set_intrinsics(np.ascontiguousarray(rt[:, 12:]))

    def points(self):
        return self.ctx.points()

    def set_points(self, X, act):
        self.ctx.set_points(X, act)

    def instance_state(self):
        return self.ctx.instance_state()

    def set_instance_state(self, Xl, Wl):
        self.ctx.set_instance_state(Xl, Wl)

    def weights(self):
        return self.ctx.weights()

    def set_weights(self, w):
        self.ctx.set_weights(w)

    def residuals(self):
        return self.ctx.residuals().reshape(-1, 2)
