"""Seeded synthetic bundle-adjustment blocks (inputs only).

This module makes the inputs that both the CUDA path and the CPU oracle are
fed: camera poses, 3D points, image observations and the camera -> sub-block
assignment. It holds none of the adjustment's arithmetic (no residual
weighting, no Jacobian, no normal equations). To create image observations it
has to image the synthetic scene with a pinhole camera; that projection is
written here on its own (scipy rotations, numpy algebra) and is shared with
nothing else.

The scenes follow the paper's simulated aerial block (Sec. 6: strips of nadir
cameras with fore/side overlap, points only where images overlap, Gaussian
pixel noise, perturbed initial poses) and the oblique multi-view blocks of its
other data sets, whose files are not available; these seeded scenes stand in
for them.

Conventions
-----------
* world: x east, y north, z up (metres); points near z = 0.
* camera: X_c = R X + t, the camera looks along +z_c, image u to the right
  (+x_c), v downwards (+y_c); pinhole f = 1000 px, 2000 x 1500 image,
  principal point (1000, 750).
* pose vector per camera: (omega, t), omega the angle-axis vector of R.
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

F_PX = 1000.0
IMG_W = 2000.0
IMG_H = 1500.0
CX = 1000.0
CY = 750.0

SEED_BASE = 8138


# --------------------------------------------------------------------------
# camera rigs
# --------------------------------------------------------------------------
def _nadir_c2w() -> np.ndarray:
    """Camera-to-world rotation of a camera looking straight down, image-up north."""
    return np.diag([1.0, -1.0, -1.0])


def _tilted_c2w(tilt_rad: float, azimuth_idx: int) -> np.ndarray:
    """Nadir camera tilted by `tilt_rad` toward N/E/S/W (azimuth_idx 0..3)."""
    d = [np.array([0.0, 1.0, 0.0]), np.array([1.0, 0.0, 0.0]),
         np.array([0.0, -1.0, 0.0]), np.array([-1.0, 0.0, 0.0])][azimuth_idx % 4]
    axis = np.cross(d, np.array([0.0, 0.0, 1.0]))  # rotates -z toward d
    q = Rotation.from_rotvec(tilt_rad * axis).as_matrix()
    return q @ _nadir_c2w()


def _rig(centers: np.ndarray, c2w: np.ndarray):
    """World-to-camera R and t for camera centres and camera-to-world rotations."""
    R = np.transpose(c2w, (0, 2, 1)).copy()
    t = -np.einsum("mab,mb->ma", R, centers)
    return R, t


def _footprint_centres(centers: np.ndarray, R: np.ndarray) -> np.ndarray:
    fwd = R[:, 2, :]  # optical axis in world coordinates
    s = -centers[:, 2] / fwd[:, 2]
    return centers[:, :2] + s[:, None] * fwd[:, :2]


# --------------------------------------------------------------------------
# imaging
# --------------------------------------------------------------------------
def _image(R, t, X):
    """Pinhole imaging of X (n,3) by cameras (R (n,3,3), t (n,3)); returns uv, depth."""
    xc = np.einsum("nab,nb->na", R, X) + t
    z = xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = F_PX * xc[:, 0] / z + CX
        v = F_PX * xc[:, 1] / z + CY
    return np.stack([u, v], axis=1), z


def _assign_observations(rng, R, t, foot, X, opp, chunk=200_000):
    """For each point pick up to opp[j] cameras that see it (random subset)."""
    M = R.shape[0]
    tree = cKDTree(foot)
    kq = int(min(M, max(32, 8 * int(np.max(opp)))))
    obs_cam, obs_pt, obs_uv = [], [], []
    for s in range(0, X.shape[0], chunk):
        Xs = X[s:s + chunk]
        n = Xs.shape[0]
        _, idx = tree.query(Xs[:, :2], k=kq, workers=-1)  # parallel over query points; same result
        idx = np.asarray(idx).reshape(n, kq)
        Rc = R[idx.reshape(-1)]
        tc = t[idx.reshape(-1)]
        Xr = np.repeat(Xs, kq, axis=0)
        uv, z = _image(Rc, tc, Xr)
        vis = (z > 0.5) & (uv[:, 0] >= 0) & (uv[:, 0] < IMG_W) & (uv[:, 1] >= 0) & (uv[:, 1] < IMG_H)
        vis = vis.reshape(n, kq)
        key = rng.random((n, kq))
        key[~vis] = 2.0
        order = np.argsort(key, axis=1)
        nvis = vis.sum(axis=1)
        take = np.minimum(nvis, opp[s:s + n])
        rank = np.empty_like(order)
        np.put_along_axis(rank, order, np.arange(kq)[None, :].repeat(n, 0), axis=1)
        sel = rank < take[:, None]
        rows, cols = np.nonzero(sel)
        obs_cam.append(idx[rows, cols])
        obs_pt.append(rows + s)
        obs_uv.append(uv.reshape(n, kq, 2)[rows, cols])
    return (np.concatenate(obs_cam).astype(np.int32), np.concatenate(obs_pt).astype(np.int64),
            np.concatenate(obs_uv))


def _finish_block(rng, R_gt, t_gt, centers_gt, X_gt, obs_cam, obs_pt, uv, sigma_px,
                  outlier_frac, rot_sigma, pos_sigma, pt_sigma, min_obs=2, n_points=None):
    # keep points with >= min_obs observations (points only in the overlap area)
    cnt = np.bincount(obs_pt, minlength=X_gt.shape[0])
    keep = cnt >= min_obs
    keep_idx = np.nonzero(keep)[0]
    if n_points is not None:
        keep_idx = keep_idx[:n_points]
    newid = -np.ones(X_gt.shape[0], dtype=np.int64)
    newid[keep_idx] = np.arange(keep_idx.size)
    m = newid[obs_pt] >= 0
    obs_cam, obs_pt, uv = obs_cam[m], newid[obs_pt[m]], uv[m]
    X_gt = X_gt[keep_idx]
    K = obs_cam.size
    xy = uv + rng.normal(0.0, sigma_px, size=(K, 2))
    outlier = rng.random(K) < outlier_frac
    n_out = int(outlier.sum())
    xy[outlier] = np.stack([rng.uniform(0, IMG_W, n_out), rng.uniform(0, IMG_H, n_out)], axis=1)
    M = R_gt.shape[0]
    # perturbed initial values: left-multiplied small rotation, moved centre, moved points
    dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, size=(M, 3))).as_matrix()
    R0 = np.einsum("mab,mbc->mac", dR, R_gt)
    C0 = centers_gt + rng.normal(0.0, pos_sigma, size=(M, 3))
    t0 = -np.einsum("mab,mb->ma", R0, C0)
    X0 = X_gt + rng.normal(0.0, pt_sigma, size=X_gt.shape)
    pose0 = np.concatenate([Rotation.from_matrix(R0).as_rotvec(), t0], axis=1)
    pose_gt = np.concatenate([Rotation.from_matrix(R_gt).as_rotvec(), t_gt], axis=1)
    return dict(
        cam_pose=np.ascontiguousarray(pose0), points=np.ascontiguousarray(X0),
        obs_cam=obs_cam.astype(np.int32), obs_point=obs_pt.astype(np.int32),
        obs_xy=np.ascontiguousarray(xy), obs_winv=None,
        gt_cam_pose=pose_gt, gt_points=X_gt, outlier=outlier,
    )


def grid_block(rng, nx, ny, spacing, height, n_points, opp, sigma_px, outlier_frac,
               oblique_deg=0.0, nadir_every=1, extent=None, z_range=(-2.0, 2.0),
               runs=None, rot_sigma=0.01, pos_sigma=0.1, pt_sigma=0.1, n_cams=None):
    """Cameras on an nx-by-ny grid (column-major numbering: i = ix*ny + iy).

    Camera i is nadir when i % nadir_every == 0, otherwise tilted by oblique_deg
    toward N/E/S/W in turn. `runs` splits the column-major index range into
    contiguous sub-blocks of the given sizes.
    """
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ix, iy = ix.reshape(-1), iy.reshape(-1)
    if n_cams is not None:
        ix, iy = ix[:n_cams], iy[:n_cams]
    M = ix.size
    cxs = (ix - (nx - 1) / 2.0) * spacing
    cys = (iy - (ny - 1) / 2.0) * spacing
    centers = np.stack([cxs, cys, np.full(M, height)], axis=1)
    c2w = np.empty((M, 3, 3))
    for i in range(M):
        if nadir_every <= 1 or i % nadir_every == 0:
            c2w[i] = _nadir_c2w()
        else:
            c2w[i] = _tilted_c2w(np.deg2rad(oblique_deg), (i % nadir_every) - 1)
    R, t = _rig(centers, c2w)
    foot = _footprint_centres(centers, R)
    if extent is None:
        extent = (cxs.min(), cxs.max(), cys.min(), cys.max())
    x0, x1, y0, y1 = extent
    n_try = int(n_points * 1.3) + 16
    X = np.stack([rng.uniform(x0, x1, n_try), rng.uniform(y0, y1, n_try),
                  rng.uniform(z_range[0], z_range[1], n_try)], axis=1)
    opp_arr = opp(rng, n_try) if callable(opp) else np.full(n_try, int(opp))
    oc, op, uv = _assign_observations(rng, R, t, foot, X, opp_arr)
    blk = _finish_block(rng, R, t, centers, X, oc, op, uv, sigma_px, outlier_frac,
                        rot_sigma, pos_sigma, pt_sigma, n_points=n_points)
    blk["cam_intr"] = np.tile(np.array([F_PX, CX, CY]), (M, 1))
    if runs is None:
        runs = [M]
    assert sum(runs) == M, (runs, M)
    blk["cam_subblock"] = np.repeat(np.arange(len(runs)), runs).astype(np.int32)
    blk["cam_block"] = np.zeros(M, dtype=np.int32)
    return blk


def _even_runs(M, L):
    base = [M // L + (1 if r < M % L else 0) for r in range(L)]
    return [b for b in base if b > 0]


def merge_blocks(blocks):
    """Concatenate independent blocks into one problem (ids offset per block)."""
    out = {k: [] for k in ("cam_pose", "cam_intr", "points", "obs_cam", "obs_point", "obs_xy",
                           "gt_cam_pose", "gt_points", "outlier", "cam_subblock", "cam_block")}
    moff = noff = loff = 0
    for b, blk in enumerate(blocks):
        out["cam_pose"].append(blk["cam_pose"]); out["cam_intr"].append(blk["cam_intr"])
        out["points"].append(blk["points"]); out["obs_xy"].append(blk["obs_xy"])
        out["obs_cam"].append(blk["obs_cam"] + moff); out["obs_point"].append(blk["obs_point"] + noff)
        out["gt_cam_pose"].append(blk["gt_cam_pose"]); out["gt_points"].append(blk["gt_points"])
        out["outlier"].append(blk["outlier"])
        out["cam_subblock"].append(blk["cam_subblock"] + loff)
        out["cam_block"].append(np.full(blk["cam_pose"].shape[0], b, dtype=np.int32))
        moff += blk["cam_pose"].shape[0]; noff += blk["points"].shape[0]
        loff += int(blk["cam_subblock"].max()) + 1
    res = {k: np.concatenate(v) for k, v in out.items()}
    for k in ("obs_cam", "obs_point", "cam_subblock", "cam_block"):
        res[k] = res[k].astype(np.int32)
    res["obs_winv"] = None
    return res


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def multi_block_member(b: int, scale: float = 1.0):
    """Block b of the 64-block workload (config 3), on its own: 20..400 cameras
    (log-uniform), 50..200 points per camera, 3..6 obs/point, 2..8 sub-blocks."""
    rb = np.random.Generator(np.random.PCG64(SEED_BASE + 100 * 3 + 1 + b))
    Mb = int(round(np.exp(rb.uniform(np.log(20), np.log(400)))))
    ppc = rb.uniform(50, 200)
    Lb = int(rb.integers(2, 9))
    ny = int(np.ceil(np.sqrt(Mb)))
    nx = int(np.ceil(Mb / ny))
    Nb = max(8, int(round(Mb * ppc / 4.5 * scale)))
    return grid_block(rb, nx, ny, 4.0, 30.0, Nb, lambda r, n: r.integers(3, 7, size=n), 0.5, 0.02,
                      oblique_deg=30.0, nadir_every=5, n_cams=Mb, runs=_even_runs(Mb, Lb))


def config(c: int, scale: float = 1.0, n_blocks: int = 64):
    """The five benchmark blocks (c = 1..5); `scale` < 1 shrinks point counts.

    1: 50 nadir cameras (10x5 grid, 4 m, 30 m high), 2,000 points, 4 obs/point,
       2 sub-blocks of 25; sigma 0.5 px, 2 % outliers.
    2: 1,000 cameras (25x40 grid, every 5th nadir, others 30 deg oblique),
       100k points, 6 obs/point, 8 uneven sub-blocks (60..200 cameras).
    3: 64 independent blocks, 20..400 cameras (log-uniform), 50..200 points per
       camera, 3..6 obs/point, 2..8 sub-blocks each (`n_blocks` keeps the first ones).
    4: 50 strips x 100 cameras, 60 % forward / 30 % side overlap, 1M points,
       5 obs/point, 32 sub-blocks, 5 % outliers.
    5: 100x100 positions, nadir and 45 deg obliques, 4M points, 5 obs/point,
       64 sub-blocks, sigma 1 px, 5 % outliers.
    6: the photo-collection block with per-camera intrinsics (bal_config):
       961 cameras on a ring, 187,103 points, 18 obs/point, 12 sub-blocks,
       focal length and k1 estimated per camera, sigma 1 px, 2 % outliers.
    """
    if c == 6:
        return bal_config(scale)
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 100 * c))
    if c == 1:
        return grid_block(rng, 10, 5, 4.0, 30.0, int(2000 * scale), 4, 0.5, 0.02,
                          extent=(-10.0, 10.0, -10.0, 10.0), runs=[25, 25])
    if c == 2:
        return grid_block(rng, 25, 40, 4.0, 30.0, int(100_000 * scale), 6, 0.5, 0.02,
                          oblique_deg=30.0, nadir_every=5,
                          runs=[60, 80, 100, 120, 140, 160, 140, 200])
    if c == 3:
        return merge_blocks([multi_block_member(b, scale) for b in range(n_blocks)])
    if c == 4:
        # strips run along y; 60 % forward overlap of the 45 m along-track footprint
        # (18 m base), 30 % side overlap of the 60 m across-track footprint (42 m).
        nx, ny = 50, 100
        sub = np.empty(nx * ny, dtype=np.int32)
        ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
        band = np.minimum(ix.reshape(-1) * 4 // nx, 3)
        seg = np.minimum(iy.reshape(-1) * 8 // ny, 7)
        sub[:] = band * 8 + seg
        blk = _grid_strips(rng, nx, ny, 42.0, 18.0, 30.0, int(1_000_000 * scale), 5, 0.5, 0.05)
        blk["cam_subblock"] = sub
        return blk
    if c == 5:
        nx = ny = 100
        ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
        sub = (np.minimum(ix.reshape(-1) * 8 // nx, 7) * 8 + np.minimum(iy.reshape(-1) * 8 // ny, 7))
        blk = grid_block(rng, nx, ny, 10.0, 30.0, int(4_000_000 * scale), 5, 1.0, 0.05,
                         oblique_deg=45.0, nadir_every=5)
        blk["cam_subblock"] = sub.astype(np.int32)
        return blk
    raise ValueError(f"unknown config {c}")


def _grid_strips(rng, nx, ny, dx, dy, height, n_points, opp, sigma_px, outlier_frac):
    """Nadir strip block: nx strips (x spacing dx) of ny cameras (y spacing dy)."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ix, iy = ix.reshape(-1), iy.reshape(-1)
    M = ix.size
    centers = np.stack([(ix - (nx - 1) / 2.0) * dx, (iy - (ny - 1) / 2.0) * dy,
                        np.full(M, height)], axis=1)
    c2w = np.repeat(_nadir_c2w()[None], M, axis=0)
    R, t = _rig(centers, c2w)
    foot = _footprint_centres(centers, R)
    x0, x1 = centers[:, 0].min(), centers[:, 0].max()
    y0, y1 = centers[:, 1].min(), centers[:, 1].max()
    n_try = int(n_points * 1.6) + 16
    X = np.stack([rng.uniform(x0, x1, n_try), rng.uniform(y0, y1, n_try),
                  rng.uniform(-2.0, 2.0, n_try)], axis=1)
    oc, op, uv = _assign_observations(rng, R, t, foot, X, np.full(n_try, opp))
    blk = _finish_block(rng, R, t, centers, X, oc, op, uv, sigma_px, outlier_frac,
                        0.01, 0.1, 0.1, n_points=n_points)
    blk["cam_intr"] = np.tile(np.array([F_PX, CX, CY]), (M, 1))
    blk["cam_block"] = np.zeros(M, dtype=np.int32)
    return blk


def tiny(seed=0, nx=3, ny=2, n_points=30, opp=4, runs=None, sigma_px=0.5, outlier_frac=0.0,
         oblique_deg=0.0, nadir_every=1, spacing=4.0, rot_sigma=0.01, pos_sigma=0.1,
         pt_sigma=0.1, extent=(-6.0, 6.0, -6.0, 6.0)):
    """A small block for brute-force checks (M = nx*ny cameras)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7 + seed))
    return grid_block(rng, nx, ny, spacing, 30.0, n_points, opp, sigma_px, outlier_frac,
                      oblique_deg=oblique_deg, nadir_every=nadir_every, extent=extent,
                      runs=runs, rot_sigma=rot_sigma, pos_sigma=pos_sigma, pt_sigma=pt_sigma)


# --------------------------------------------------------------------------
# photo-collection blocks with per-camera intrinsics (the Final data sets of
# Sec. 6: focal length and first radial parameter estimated per camera)
# --------------------------------------------------------------------------
def _image_radial(R, t, f, k1, X):
    """Imaging with a radial polynomial on the normalised coordinates:
    p = (x_c, y_c)/z_c, (u, v) = f (1 + k1 |p|^2) p + (CX, CY)."""
    xc = np.einsum("nab,nb->na", R, X) + t
    z = xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        p = xc[:, :2] / z[:, None]
    d = 1.0 + k1 * np.sum(p * p, axis=1)
    uv = (f * d)[:, None] * p + np.array([CX, CY])
    return uv, z


def ring_block(rng, n_cams, n_points, mean_track, n_sub, sigma_px=1.0, outlier_frac=0.02,
               radius=9.0, f_range=(850.0, 1250.0), k1_range=(-0.08, 0.08), f_sigma_rel=0.01,
               rot_sigma=0.002, pos_sigma=0.03, pt_sigma=0.03):
    """Cameras on a ring around an object, each with its own focal length and
    radial parameter; points on the object, each seen by a random subset of
    the cameras facing its side (track lengths 2 + geometric, mean
    `mean_track`); sub-blocks are contiguous arcs of the ring. The initial
    values perturb the poses and points and the focal lengths (relative
    sigma `f_sigma_rel`) and start every k1 at 0."""
    M = n_cams
    az = 2.0 * np.pi * (np.arange(M) + rng.uniform(-0.3, 0.3, M)) / M
    centers = np.stack([radius * np.cos(az), radius * np.sin(az), rng.uniform(1.0, 4.0, M)], axis=1)
    target = np.array([0.0, 0.0, 2.5]) + rng.normal(0.0, 0.3, (M, 3))
    c2w = np.empty((M, 3, 3))
    for i in range(M):
        zc = target[i] - centers[i]
        zc /= np.linalg.norm(zc)
        xc = np.cross(zc, np.array([0.0, 0.0, 1.0]))
        xc /= np.linalg.norm(xc)
        yc = np.cross(zc, xc)
        roll = Rotation.from_rotvec(zc * rng.normal(0.0, 0.05)).as_matrix()
        c2w[i] = roll @ np.stack([xc, yc, zc], axis=1)
    R, t = _rig(centers, c2w)
    f = rng.uniform(*f_range, M)
    k1 = rng.uniform(*k1_range, M)
    # points on the object (a cylinder of radius 4.5, 0..5 high), each facing outward
    n_try = int(n_points * 1.2) + 16
    paz = rng.uniform(0.0, 2.0 * np.pi, n_try)
    pr = 4.5 * np.sqrt(rng.uniform(0.3, 1.0, n_try))
    X = np.stack([pr * np.cos(paz), pr * np.sin(paz), rng.uniform(0.0, 5.0, n_try)], axis=1)
    want = 2 + rng.geometric(1.0 / max(mean_track - 1.0, 1.0), n_try) - 1
    half = int(M * 65 / 360)  # cameras within 65 degrees of the point's side
    centre_cam = np.round(paz / (2.0 * np.pi) * M).astype(np.int64)
    oc, op, ouv = [], [], []
    for j in range(n_try):
        cand = (centre_cam[j] + np.arange(-half, half + 1)) % M
        take = rng.permutation(cand)[:min(int(want[j]), cand.size)]
        uv, z = _image_radial(R[take], t[take], f[take], k1[take], np.repeat(X[j][None], take.size, 0))
        ok = (z > 0.5) & (uv[:, 0] >= 0) & (uv[:, 0] < IMG_W) & (uv[:, 1] >= 0) & (uv[:, 1] < IMG_H)
        if ok.sum() >= 2:
            oc.append(take[ok])
            op.append(np.full(int(ok.sum()), j))
            ouv.append(uv[ok])
    oc, op, ouv = np.concatenate(oc).astype(np.int32), np.concatenate(op), np.concatenate(ouv)
    blk = _finish_block(rng, R, t, centers, X, oc, op, ouv, sigma_px, outlier_frac,
                        rot_sigma, pos_sigma, pt_sigma, n_points=n_points)
    f0 = f * (1.0 + rng.normal(0.0, f_sigma_rel, M))
    blk["cam_intr"] = np.stack([f0, np.full(M, CX), np.full(M, CY)], axis=1)
    blk["cam_k1"] = np.zeros(M)
    blk["intrinsics"] = True
    blk["gt_cam_intr"] = np.stack([f, np.full(M, CX), np.full(M, CY)], axis=1)
    blk["gt_cam_k1"] = k1
    blk["cam_subblock"] = (np.arange(M) * n_sub // M).astype(np.int32)
    blk["cam_block"] = np.zeros(M, dtype=np.int32)
    return blk


def bal_config(scale: float = 1.0):
    """Stand-in for the Final 961 data set of Sec. 6 (Table datasets: 961
    cameras, 187,103 points, 3,385,950 observations, focal length and k1 per
    camera): a seeded ring block of the same size, 18 observations per point
    on average, 12 sub-blocks of about 80 cameras (the paper's minimum is 70),
    sigma 1 px, 2 % outliers."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 961))
    return ring_block(rng, 961, int(187_103 * scale), 18.1, 12)


def tiny_intrinsics(seed=0, n_cams=24, n_points=300, mean_track=6.0, n_sub=3, sigma_px=0.5,
                    outlier_frac=0.0, **kw):
    """A small ring block with per-camera intrinsics for brute-force checks."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 29 + seed))
    return ring_block(rng, n_cams, n_points, mean_track, n_sub, sigma_px=sigma_px,
                      outlier_frac=outlier_frac, **kw)


PROBLEM_KEYS = ("cam_pose", "cam_intr", "points", "obs_cam", "obs_point", "obs_xy",
                "obs_winv", "cam_subblock", "cam_block")


# --------------------------------------------------------------------------
# RCS-shaped matrices for the learned preconditioner
# --------------------------------------------------------------------------
def rcs_like_systems(seed: int, sizes=(12, 20, 7), points_per_cam: int = 6, n_probes: int = 4):
    """Random symmetric positive definite 6n x 6n matrices with the block
    structure of a reduced camera system: cameras on a strip, each "point"
    couples 2..4 neighbouring cameras through a rank-3 term, camera scales
    spread over two decades. Returns a list of (S, z) with z the Gaussian
    probe vectors (n_probes x 6n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for n in sizes:
        scale = np.repeat(np.exp(rng.uniform(0.0, np.log(100.0), n)), 6) * rng.uniform(0.5, 2.0, 6 * n)
        S = np.zeros((6 * n, 6 * n))
        for _ in range(points_per_cam * n):
            c0 = int(rng.integers(0, n))
            k = int(rng.integers(2, 5))
            cams = sorted({min(n - 1, max(0, c0 + int(d))) for d in rng.integers(-2, 3, size=k)} | {c0})
            idx = np.concatenate([np.arange(6 * c, 6 * c + 6) for c in cams])
            G = rng.normal(size=(3, idx.size)) * np.sqrt(scale[idx])
            S[np.ix_(idx, idx)] += G.T @ G
        S += np.diag(1e-3 * np.diag(S).mean() + 1e-2 * np.diag(S))
        z = rng.normal(size=(n_probes, 6 * n))
        out.append((S, z))
    return out
