"""Thin Python binding of the RPBA C ABI (include/rpba.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of librpba.so. The functions keep the C names (rpba_create,
rpba_intersect, rpba_iterate, rpba_covariance, ...); `Rpba` wraps a context.
PyTorch supplies the CUDA stream (and optionally device memory through its
caching allocator). There is no CPU fallback: if the library or a GPU is
missing, the calls raise.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u8 = C.POINTER(C.c_uint8)
_fp = C.POINTER(C.c_float)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Problem(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("n_points", C.c_int32), ("n_obs", C.c_int32),
                ("cam_pose", _dp), ("cam_intr", _dp), ("points", _dp), ("obs_cam", _ip),
                ("obs_point", _ip), ("obs_xy", _dp), ("obs_winv", _dp), ("cam_subblock", _ip),
                ("cam_block", _ip), ("cam_k1", _dp)]


class Options(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("t_v", C.c_double), ("downweight", C.c_double),
                ("stop_ratio", C.c_double), ("grace", C.c_int32), ("max_outer", C.c_int32),
                ("max_inner", C.c_int32), ("max_reject", C.c_int32), ("robust", C.c_int32),
                ("robust_from_start", C.c_int32), ("weight_mode", C.c_int32), ("rho0", C.c_double),
                ("robust_serial", C.c_int32), ("isect_max_iter", C.c_int32),
                ("isect_tol", C.c_double), ("isect_px_tol", C.c_double), ("cond_max", C.c_double),
                ("precision", C.c_int32),
                ("solver", C.c_int32), ("pcg_tol", C.c_double), ("pcg_max_iter", C.c_int32),
                ("ir_steps", C.c_int32), ("chol_tc", C.c_int32), ("intrinsics", C.c_int32),
                ("tune_cache", C.c_char_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", C.c_void_p)]


class Report(C.Structure):
    _fields_ = [("sigma0", C.c_double), ("rms", C.c_double), ("sigma0_initial", C.c_double),
                ("outer", C.c_int32), ("inner_total", C.c_int32), ("lm_launches", C.c_int32),
                ("deleted_points", C.c_int32), ("active_points", C.c_int32),
                ("active_obs", C.c_int32), ("robust_started_at", C.c_int32),
                ("sigma0_hist", C.c_double * 128)]


STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED",
          5: "DEVICE_TIMEOUT", 6: "NUMERIC", 7: "STATE"}


class RpbaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rpba status {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librpba.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    vp = C.c_void_p
    sigs = {
        "rpba_default_options": (None, [C.POINTER(Options)]),
        "rpba_create": (C.c_int, [C.POINTER(Problem), C.POINTER(Options), vp, C.POINTER(vp)]),
        "rpba_destroy": (None, [vp]),
        "rpba_last_error": (C.c_char_p, [vp]),
        "rpba_intersect": (C.c_int, [vp]),
        "rpba_iterate": (C.c_int, [vp, C.c_int32, C.POINTER(Report)]),
        "rpba_covariance": (C.c_int, [vp, _ip, C.c_int32, _dp]),
        "rpba_get_cameras": (C.c_int, [vp, _dp]),
        "rpba_get_points": (C.c_int, [vp, _dp, _u8]),
        "rpba_info": (C.c_int, [vp, _ip, _ip]),
        "rpba_get_options": (C.c_int, [vp, C.POINTER(Options)]),
        "rpba_sub_cameras": (C.c_int, [vp, C.c_int32, _ip, _ip]),
        "rpba_set_cameras": (C.c_int, [vp, _dp]),
        "rpba_set_points": (C.c_int, [vp, _dp, _u8]),
        "rpba_get_instances": (C.c_int, [vp, _ip, _ip, _dp, _dp]),
        "rpba_set_instances": (C.c_int, [vp, _dp, _dp]),
        "rpba_get_weights": (C.c_int, [vp, _dp]),
        "rpba_set_weights": (C.c_int, [vp, _dp]),
        "rpba_residuals": (C.c_int, [vp, _dp]),
        "rpba_jacobians": (C.c_int, [vp, _dp, _dp]),
        "rpba_sigma0": (C.c_int, [vp, _dp, _dp]),
        "rpba_camera_scale": (C.c_int, [vp, _dp]),
        "rpba_robust_weights": (C.c_int, [vp, _ip]),
        "rpba_intersect_points": (C.c_int, [vp, C.c_int32, _ip]),
        "rpba_sub_costs": (C.c_int, [vp, _dp]),
        "rpba_rcs": (C.c_int, [vp, C.c_int32, C.c_double, _dp, _dp]),
        "rpba_lm_step": (C.c_int, [vp, C.c_double, _ip, _dp, _dp, _dp, _dp]),
        "rpba_bact": (C.c_int, [vp, _ip]),
        "rpba_profile_enable": (C.c_int, [vp, C.c_int32]),
        "rpba_profile_select": (C.c_int, [vp, C.c_char_p]),
        "rpba_tune": (C.c_int, [vp, C.c_char_p, _ip]),
        "rpba_partition": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _ip, _ip, C.c_int32, _ip, _dp,
                                     C.POINTER(C.c_double)]),
        "rpba_get_camera_rt": (C.c_int, [vp, _dp, _dp]),
        "rpba_get_intrinsics": (C.c_int, [vp, _dp]),
        "rpba_set_intrinsics": (C.c_int, [vp, _dp]),
        "rpba_set_camera_rt": (C.c_int, [vp, _dp, _dp]),
        "rpba_set_subblock_mask": (C.c_int, [vp, C.c_void_p]),
        "rpba_set_point_mask": (C.c_int, [vp, C.c_void_p]),
        "rpba_outer_iteration": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
        "rpba_profile_read": (C.c_int, [vp, C.c_int32, C.c_char_p, _dp, C.POINTER(C.c_int64), _ip,
                                        C.POINTER(C.c_int64)]),
        "rpba_solver_stats": (C.c_int, [vp, _ip, _dp]),
        "rpba_solver_stages": (C.c_int, [vp, _ip]),
        "rpba_solver_fallbacks": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "rpba_gnn_param_count": (C.c_int32, []),
        "rpba_set_gnn_weights": (C.c_int, [vp, _fp, C.c_int32]),
        "rpba_gnn_create": (C.c_int, [C.c_uint64, C.POINTER(vp)]),
        "rpba_gnn_destroy": (None, [vp]),
        "rpba_gnn_last_error": (C.c_char_p, [vp]),
        "rpba_gnn_get_weights": (C.c_int, [vp, _fp]),
        "rpba_gnn_set_weights": (C.c_int, [vp, _fp]),
        "rpba_gnn_add_system": (C.c_int, [vp, C.c_int32, _dp, C.c_int32, C.c_int32, _dp]),
        "rpba_gnn_add_rcs": (C.c_int, [vp, vp, C.c_double, C.c_int32, C.c_uint64]),
        "rpba_gnn_dataset_size": (C.c_int, [vp, _ip, _ip, _ip]),
        "rpba_gnn_graph": (C.c_int, [vp, _fp, _ip, _ip, _fp]),
        "rpba_gnn_precondition": (C.c_int, [vp, _dp, _dp]),
        "rpba_gnn_loss_grad": (C.c_int, [vp, _dp, _fp]),
        "rpba_gnn_train": (C.c_int, [vp, C.c_int32, C.c_float, C.c_uint64, _dp]),
        "rpba_sigma0_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32] + [vp] * 10 + [vp, _dp, _dp, _dp]),
        "rpba_check_formats": (C.c_int, [_dp, _fp, C.c_int32, _fp, _fp, _dp, _dp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/rpba.h that the library must export."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "rpba.h")
    import re
    names = re.findall(r"^\s*(?:rpba_status|void|int32_t|const char\s*\*)\s*\*?\s*(rpba_\w+)\s*\(",
                       open(hdr).read(), flags=re.M)
    return sorted(set(names))


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _f(a):
    return a.ctypes.data_as(_fp) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def rpba_sigma0_noalloc(n_cams, n_points, n_obs, R, t, intr, X, active, obs_cam, obs_point, obs_xy,
                        obs_winv=None, obs_w=None, stream=None):
    """sigma_0 and RMS of device arrays (integer device addresses, e.g. a
    torch tensor's data_ptr(); None for the optional ones) without any device
    allocation by the library. Returns (sigma0, rms, sums5)."""
    ptr = lambda a: None if a is None else C.c_void_p(int(a))
    sums = np.zeros(5)
    s0, rms = C.c_double(), C.c_double()
    st = load().rpba_sigma0_noalloc(int(n_cams), int(n_points), int(n_obs), ptr(R), ptr(t), ptr(intr), ptr(X),
                                    ptr(active), ptr(obs_cam), ptr(obs_point), ptr(obs_xy), ptr(obs_winv),
                                    ptr(obs_w), ptr(getattr(stream, "cuda_stream", stream)), _d(sums),
                                    C.byref(s0), C.byref(rms))
    if st != 0:
        raise RpbaError(st, "rpba_sigma0_noalloc failed")
    return s0.value, rms.value, sums


def rpba_partition(n_cams, n_points, obs_cam, obs_point, n_parts):
    """Sub-blocks from the visibility graph (Sec. 5.2): returns (cam_subblock,
    node_weight, edge_cut)."""
    oc = np.ascontiguousarray(obs_cam, dtype=np.int32)
    op = np.ascontiguousarray(obs_point, dtype=np.int32)
    part = np.zeros(int(n_cams), np.int32)
    w = np.zeros(int(n_cams))
    cut = C.c_double()
    st = load().rpba_partition(int(n_cams), int(n_points), int(oc.size), _i(oc), _i(op), int(n_parts), _i(part),
                               _d(w), C.byref(cut))
    if st != 0:
        raise RpbaError(st, "rpba_partition failed")
    return part, w, cut.value


def rpba_check_formats(x, f):
    """The FP32 form's device format changes: x (float64) -> (hi, lo, hi + lo)
    and f (float32) -> float64 (rpba_check_formats)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float32)
    assert x.size == f.size
    n = x.size
    hi, lo = np.zeros(n, np.float32), np.zeros(n, np.float32)
    back, fd = np.zeros(n), np.zeros(n)
    st = load().rpba_check_formats(_d(x), _f(f), n, _f(hi), _f(lo), _d(back), _d(fd))
    if st != 0:
        raise RpbaError(st, "rpba_check_formats failed")
    return hi, lo, back, fd


def rpba_default_options(**overrides) -> Options:
    o = Options()
    load().rpba_default_options(C.byref(o))
    for k, v in overrides.items():
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def _check(handle, status):
    if status != 0:
        msg = load().rpba_last_error(handle)
        raise RpbaError(status, msg.decode() if msg else "")


def _torch_allocator(device):
    """Allocator hooks backed by PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, user):
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=device)

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def rpba_create(problem: dict, options: Options | None = None, stream=None, torch_alloc: bool = False):
    """Returns (handle, keepalive). `stream`: a torch.cuda.Stream, an int handle or None."""
    L = load()
    keep = {}
    M = int(problem["cam_pose"].shape[0])
    N = int(problem["points"].shape[0])
    K = int(problem["obs_cam"].shape[0])
    arrs = dict(cam_pose=_f64(problem["cam_pose"], (M, 6)), cam_intr=_f64(problem["cam_intr"], (M, 3)),
                points=_f64(problem["points"], (N, 3)), obs_cam=_i32(problem["obs_cam"]),
                obs_point=_i32(problem["obs_point"]), obs_xy=_f64(problem["obs_xy"], (K, 2)),
                cam_subblock=_i32(problem["cam_subblock"]))
    winv = problem.get("obs_winv")
    arrs["obs_winv"] = None if winv is None else _f64(winv, (K, 3))
    blk = problem.get("cam_block")
    arrs["cam_block"] = None if blk is None else _i32(blk)
    k1 = problem.get("cam_k1")
    arrs["cam_k1"] = None if k1 is None else _f64(k1, (M,))
    keep["arrs"] = arrs
    pb = Problem(M, N, K, _d(arrs["cam_pose"]), _d(arrs["cam_intr"]), _d(arrs["points"]),
                 _i(arrs["obs_cam"]), _i(arrs["obs_point"]), _d(arrs["obs_xy"]), _d(arrs["obs_winv"]),
                 _i(arrs["cam_subblock"]), _i(arrs["cam_block"]), _d(arrs["cam_k1"]))
    opt = options if options is not None else rpba_default_options()
    if torch_alloc:
        import torch
        dev = torch.cuda.current_device()
        a, f = _torch_allocator(dev)
        keep["alloc"] = (a, f)
        opt.dev_alloc, opt.dev_free = a, f
    s = None
    if stream is not None:
        s = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    h = C.c_void_p()
    st = L.rpba_create(C.byref(pb), C.byref(opt), s, C.byref(h))
    if st != 0:
        msg = L.rpba_last_error(h) if h.value else b"create failed"
        if h.value:
            L.rpba_destroy(h)
        raise RpbaError(st, msg.decode() if msg else "")
    keep["opt"] = opt
    return h, keep


class Rpba:
    """One library context over a problem dict (same keys as the C struct).
    The intrinsics option defaults to the problem's "intrinsics" entry."""

    def __init__(self, problem, stream=None, torch_alloc=False, **options):
        options.setdefault("intrinsics", int(bool(problem.get("intrinsics", False))))
        self.options = rpba_default_options(**options)
        self.cd = 8 if self.options.intrinsics else 6
        self._h, self._keep = rpba_create(problem, self.options, stream=stream, torch_alloc=torch_alloc)
        self.M = int(problem["cam_pose"].shape[0])
        self.N = int(problem["points"].shape[0])
        self.K = int(problem["obs_cam"].shape[0])
        Lp, Pp = C.c_int32(), C.c_int32()
        _check(self._h, load().rpba_info(self._h, C.byref(Lp), C.byref(Pp)))
        self.L, self.P = Lp.value, Pp.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().rpba_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(self._h, st)

    # main calls
    def intersect(self):
        self._c(load().rpba_intersect(self._h))

    def iterate(self, max_outer=0):
        r = Report()
        self._c(load().rpba_iterate(self._h, int(max_outer), C.byref(r)))
        return {"sigma0": r.sigma0, "rms": r.rms, "sigma0_initial": r.sigma0_initial, "outer": r.outer,
                "inner_total": r.inner_total, "lm_launches": r.lm_launches,
                "deleted_points": r.deleted_points, "active_points": r.active_points,
                "active_obs": r.active_obs, "robust_started_at": r.robust_started_at,
                "sigma0_hist": list(r.sigma0_hist[:min(r.outer, 128)])}

    def outer_iteration(self, robust=True):
        """One steady-state outer iteration (bact, exchange, robust weights,
        TP intersection, sigma_0); returns (sigma_0, lock-step LM iterations)."""
        s, n = C.c_double(), C.c_int32()
        self._c(load().rpba_outer_iteration(self._h, int(bool(robust)), C.byref(s), C.byref(n)))
        return s.value, n.value

    def covariance(self, ids):
        ids = _i32(ids)
        out = np.zeros((ids.size, 9))
        self._c(load().rpba_covariance(self._h, _i(ids), ids.size, _d(out)))
        return out.reshape(-1, 3, 3)

    def cameras(self, out=None):
        """Poses (n_cams x 6); into `out` (C-contiguous float64) when given."""
        out = np.zeros((self.M, 6)) if out is None else out
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 6 * self.M
        self._c(load().rpba_get_cameras(self._h, _d(out)))
        return out

    def points(self, out=None):
        """(X n_points x 3, active); into `out` = (X, active) when given."""
        X, a = (np.zeros((self.N, 3)), np.zeros(self.N, np.uint8)) if out is None else out
        assert X.dtype == np.float64 and X.flags.c_contiguous and X.size == 3 * self.N
        assert a.dtype == np.uint8 and a.flags.c_contiguous and a.size == self.N
        self._c(load().rpba_get_points(self._h, _d(X), a.ctypes.data_as(_u8)))
        return X, a

    # state access (parity tests)
    def sub_cameras(self, l):
        out = np.zeros(self.M, np.int32)
        n = C.c_int32()
        self._c(load().rpba_sub_cameras(self._h, l, _i(out), C.byref(n)))
        return out[:n.value]

    def set_cameras(self, pose):
        self._c(load().rpba_set_cameras(self._h, _d(_f64(pose, (self.M, 6)))))

    def intrinsics(self):
        """(n_cams x 2): focal length and radial parameter k1 of every camera."""
        fk = np.zeros((self.M, 2))
        self._c(load().rpba_get_intrinsics(self._h, _d(fk)))
        return fk

    def set_intrinsics(self, fk):
        self._c(load().rpba_set_intrinsics(self._h, _d(_f64(fk, (self.M, 2)))))

    def set_points(self, X, active=None):
        a = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        self._c(load().rpba_set_points(self._h, _d(_f64(X, (self.N, 3))),
                                       None if a is None else a.ctypes.data_as(_u8)))

    def instances(self):
        ip, isb = np.zeros(self.P, np.int32), np.zeros(self.P, np.int32)
        self._c(load().rpba_get_instances(self._h, _i(ip), _i(isb), None, None))
        return ip, isb

    def instance_state(self):
        Xl, Wl = np.zeros((self.P, 3)), np.zeros((self.P, 6))
        self._c(load().rpba_get_instances(self._h, None, None, _d(Xl), _d(Wl)))
        return Xl, Wl

    def set_instance_state(self, Xl, Wl):
        self._c(load().rpba_set_instances(self._h, _d(_f64(Xl, (self.P, 3))), _d(_f64(Wl, (self.P, 6)))))

    def weights(self):
        w = np.zeros(self.K)
        self._c(load().rpba_get_weights(self._h, _d(w)))
        return w

    def set_weights(self, w):
        self._c(load().rpba_set_weights(self._h, _d(_f64(w))))

    def residuals(self):
        v = np.zeros((self.K, 2))
        self._c(load().rpba_residuals(self._h, _d(v)))
        return v

    def jacobians(self):
        Jc, Jx = np.zeros((self.K, 2 * self.cd)), np.zeros((self.K, 6))
        self._c(load().rpba_jacobians(self._h, _d(Jc), _d(Jx)))
        return Jc.reshape(self.K, 2, self.cd), Jx.reshape(self.K, 2, 3)

    def sigma0(self):
        s, r = C.c_double(), C.c_double()
        self._c(load().rpba_sigma0(self._h, C.byref(s), C.byref(r)))
        return s.value, r.value

    def camera_scale(self):
        s = np.zeros(self.M)
        self._c(load().rpba_camera_scale(self._h, _d(s)))
        return s

    def robust_weights(self):
        n = C.c_int32()
        self._c(load().rpba_robust_weights(self._h, C.byref(n)))
        return n.value

    def intersect_points(self, tp_only=False):
        n = C.c_int32()
        self._c(load().rpba_intersect_points(self._h, int(tp_only), C.byref(n)))
        return n.value

    def sub_costs(self):
        F = np.zeros(self.L)
        self._c(load().rpba_sub_costs(self._h, _d(F)))
        return F

    def rcs(self, l, lam):
        n = self.cd * len(self.sub_cameras(l))
        S, y = np.zeros((n, n)), np.zeros(n)
        self._c(load().rpba_rcs(self._h, l, float(lam), _d(S), _d(y)))
        return S, y

    def lm_step(self, lam):
        acc = np.zeros(self.L, np.int32)
        Fb, Ft = np.zeros(self.L), np.zeros(self.L)
        dc, dx = np.zeros(self.cd * self.M), np.zeros((self.P, 3))
        self._c(load().rpba_lm_step(self._h, float(lam), _i(acc), _d(Fb), _d(Ft), _d(dc), _d(dx)))
        return acc, Fb, Ft, dc, dx

    def tune(self, cache_path=None):
        """Autotune the launch shapes on this context's data; returns the
        choice {isect, lin, backsub, robust, chol_tc} (written to cache_path,
        or to the context's tune_cache, when given)."""
        out = np.zeros(5, np.int32)
        self._c(load().rpba_tune(self._h, None if cache_path is None else str(cache_path).encode(), _i(out)))
        return dict(zip(("isect", "lin", "backsub", "robust", "chol_tc"), (int(x) for x in out)))

    def camera_rt(self):
        """(M, 12): rotation matrix (row-major) and translation per camera, as held."""
        R, t = np.zeros((self.M, 9)), np.zeros((self.M, 3))
        self._c(load().rpba_get_camera_rt(self._h, _d(R), _d(t)))
        return np.concatenate([R, t], axis=1)

    def set_camera_rt(self, Rt):
        Rt = _f64(Rt, (self.M, 12))
        self._c(load().rpba_set_camera_rt(self._h, _d(np.ascontiguousarray(Rt[:, :9])),
                                          _d(np.ascontiguousarray(Rt[:, 9:]))))

    def set_subblock_mask(self, mask=None):
        """LM adjustment only of the sub-blocks with mask[l] != 0 (None: all)."""
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        assert m is None or m.size == self.L
        self._c(load().rpba_set_subblock_mask(self._h, None if m is None else m.ctypes.data_as(C.c_void_p)))

    def set_point_mask(self, mask=None):
        """Intersections only of the points with mask[j] != 0 (None: all)."""
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        assert m is None or m.size == self.N
        self._c(load().rpba_set_point_mask(self._h, None if m is None else m.ctypes.data_as(C.c_void_p)))

    def bact(self):
        it = np.zeros(self.L, np.int32)
        self._c(load().rpba_bact(self._h, _i(it)))
        return it

    def resolved_options(self):
        """The context's options, with solver 4 (auto) resolved."""
        o = Options()
        self._c(load().rpba_get_options(self._h, C.byref(o)))
        return o

    def solver_stats(self):
        it, rr = np.zeros(self.L, np.int32), np.zeros(self.L)
        self._c(load().rpba_solver_stats(self._h, _i(it), _d(rr)))
        return it, rr

    def solver_stages(self):
        """Refinement stages of every sub-block in the last FP32-form
        block-Jacobi PCG solve (zeros for the other solvers)."""
        n = np.zeros(self.L, np.int32)
        self._c(load().rpba_solver_stages(self._h, _i(n)))
        return n

    def solver_fallbacks(self):
        n = C.c_int64()
        self._c(load().rpba_solver_fallbacks(self._h, C.byref(n)))
        return int(n.value)

    def set_gnn_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        self._c(load().rpba_set_gnn_weights(self._h, _f(w), int(w.size)))

    # measurement
    def profile_enable(self, enable=True):
        self._c(load().rpba_profile_enable(self._h, int(bool(enable))))

    def profile_select(self, kernel=None):
        """Time only this kernel's launches while profiling (None: all)."""
        self._c(load().rpba_profile_select(self._h, kernel.encode() if kernel else None))

    def profile_read(self):
        """{kernel: (launches, ms)}, total launches since profile_enable."""
        cap = 128
        names = C.create_string_buffer(48 * cap)
        ms = np.zeros(cap)
        la = np.zeros(cap, np.int64)
        n = C.c_int32()
        tot = C.c_int64()
        self._c(load().rpba_profile_read(self._h, cap, names, _d(ms), la.ctypes.data_as(C.POINTER(C.c_int64)),
                                         C.byref(n), C.byref(tot)))
        raw = names.raw
        out = {}
        for a in range(min(n.value, cap)):
            nm = raw[48 * a:48 * a + 48].split(b"\0", 1)[0].decode()
            out[nm] = (int(la[a]), float(ms[a]))
        return out, int(tot.value)


def gnn_param_count() -> int:
    return int(load().rpba_gnn_param_count())


class Gnn:
    """The learned block preconditioner's trainer (rpba_gnn_*): network,
    dataset of systems and Adam, on the current CUDA device."""

    def __init__(self, seed=0):
        L = load()
        self._h = C.c_void_p()
        st = L.rpba_gnn_create(int(seed), C.byref(self._h))
        self._c(st)
        self.n_params = gnn_param_count()

    def _c(self, st):
        if st != 0:
            msg = load().rpba_gnn_last_error(self._h) if self._h.value else b""
            raise RpbaError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().rpba_gnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self):
        w = np.zeros(self.n_params, np.float32)
        self._c(load().rpba_gnn_get_weights(self._h, _f(w)))
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        assert w.size == self.n_params
        self._c(load().rpba_gnn_set_weights(self._h, _f(w)))

    def add_system(self, S, z):
        S = _f64(S)
        z = _f64(z)
        n = S.shape[0] // 6
        self._c(load().rpba_gnn_add_system(self._h, n, _d(S), S.shape[1], z.shape[0], _d(z)))

    def add_rcs(self, ctx, lam=1e-4, n_probes=4, seed=0):
        self._c(load().rpba_gnn_add_rcs(self._h, ctx._h, float(lam), int(n_probes), int(seed)))

    def size(self):
        n, e, s = C.c_int32(), C.c_int32(), C.c_int32()
        self._c(load().rpba_gnn_dataset_size(self._h, C.byref(n), C.byref(e), C.byref(s)))
        return n.value, e.value, s.value

    def graph(self):
        n, ne, _ = self.size()
        x = np.zeros((n, 21), np.float32)
        ptr = np.zeros(n + 1, np.int32)
        adj = np.zeros(max(ne, 1), np.int32)
        e = np.zeros(max(ne, 1), np.float32)
        self._c(load().rpba_gnn_graph(self._h, _f(x), _i(ptr), _i(adj), _f(e)))
        return x, ptr, adj[:ne], e[:ne]

    def precondition(self, r):
        """z = P^-1 r for every dataset system (r: n_nodes x 6 values)."""
        r = _f64(r).reshape(-1)
        z = np.zeros_like(r)
        self._c(load().rpba_gnn_precondition(self._h, _d(r), _d(z)))
        return z

    def loss_grad(self):
        loss = C.c_double()
        g = np.zeros(self.n_params, np.float32)
        self._c(load().rpba_gnn_loss_grad(self._h, C.byref(loss), _f(g)))
        return loss.value, g

    def train(self, steps, lr=1e-3, probe_seed=0):
        """Adam steps; probe_seed != 0 draws new probes before every step."""
        hist = np.zeros(max(int(steps), 1))
        self._c(load().rpba_gnn_train(self._h, int(steps), float(lr), int(probe_seed), _d(hist)))
        return hist[:int(steps)]
