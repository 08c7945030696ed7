"""Python access to the FP64 CPU oracle (rpba_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark load this module to check or time against the CUDA path.
Nothing in the library package imports it.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpba_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librpba_oracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


class Options(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("t_v", C.c_double), ("downweight", C.c_double),
                ("stop_ratio", C.c_double), ("grace", C.c_int), ("max_outer", C.c_int),
                ("max_inner", C.c_int), ("max_reject", C.c_int), ("robust", C.c_int),
                ("robust_from_start", C.c_int), ("isect_max_iter", C.c_int),
                ("isect_tol", C.c_double), ("isect_px_tol", C.c_double), ("cond_max", C.c_double),
                ("robust_serial", C.c_int), ("weight_mode", C.c_int), ("rho0", C.c_double),
                ("rho", C.c_double)]


class Report(C.Structure):
    _fields_ = [("sigma0", C.c_double), ("rms", C.c_double), ("sigma0_initial", C.c_double),
                ("outer", C.c_int), ("inner_total", C.c_int), ("deleted_points", C.c_int),
                ("active_points", C.c_int), ("active_obs", C.c_int),
                ("robust_started_at", C.c_int), ("sigma0_hist", C.c_double * 128)]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, no -march flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rpba_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _ip, _ip, _dp,
                                 C.c_void_p, _ip]
        L.orc_destroy.argtypes = [C.c_void_p]
        for name in ("orc_num_subblocks", "orc_num_instances"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = C.c_int
        L.orc_instances.argtypes = [C.c_void_p, _ip, _ip]
        L.orc_sub_cameras.argtypes = [C.c_void_p, C.c_int, _ip]
        L.orc_sub_cameras.restype = C.c_int
        L.orc_get_cameras.argtypes = [C.c_void_p, _dp]
        L.orc_set_cameras.argtypes = [C.c_void_p, _dp]
        L.orc_get_camera_rt.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_set_camera_rt.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_get_points.argtypes = [C.c_void_p, _dp, _up]
        L.orc_set_points.argtypes = [C.c_void_p, _dp, C.c_void_p]
        L.orc_get_instances.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_set_instances.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_get_weights.argtypes = [C.c_void_p, _dp]
        L.orc_set_weights.argtypes = [C.c_void_p, _dp]
        L.orc_rodrigues.argtypes = [_dp, _dp]
        L.orc_rotation_log.argtypes = [_dp, _dp]
        L.orc_project.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_project.restype = C.c_double
        L.orc_project_k1.argtypes = [_dp, _dp, _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.orc_project_k1.restype = C.c_double
        L.orc_enable_intrinsics.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_camera_dim.argtypes = [C.c_void_p]
        L.orc_camera_dim.restype = C.c_int
        L.orc_get_intrinsics.argtypes = [C.c_void_p, _dp]
        L.orc_set_intrinsics.argtypes = [C.c_void_p, _dp]
        L.orc_residuals.argtypes = [C.c_void_p, _dp]
        L.orc_jacobians.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_sigma0.argtypes = [C.c_void_p]
        L.orc_sigma0.restype = C.c_double
        L.orc_rms.argtypes = [C.c_void_p]
        L.orc_rms.restype = C.c_double
        L.orc_covariance.argtypes = [C.c_void_p, _ip, C.c_int, _dp]
        L.orc_camera_scale.argtypes = [C.c_void_p, _dp]
        L.orc_median.argtypes = [_dp, C.c_int]
        L.orc_median.restype = C.c_double
        L.orc_robust_weights.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_robust_weights.restype = C.c_int
        L.orc_intersect.argtypes = [C.c_void_p, C.POINTER(Options), C.c_int]
        L.orc_intersect.restype = C.c_int
        L.orc_intersect_points.argtypes = [C.c_void_p, C.POINTER(Options), _ip, C.c_int, C.c_int]
        L.orc_intersect_points.restype = C.c_int
        L.orc_robust_weights_cams.argtypes = [C.c_void_p, _ip, C.c_int, C.c_double, C.c_double]
        L.orc_robust_weights_cams.restype = C.c_int
        L.orc_sub_cost.argtypes = [C.c_void_p, C.c_int]
        L.orc_sub_cost.restype = C.c_double
        L.orc_rcs.argtypes = [C.c_void_p, C.c_int, C.c_double, _dp, _dp]
        L.orc_rcs.restype = C.c_int
        L.orc_lm_step.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), _dp, _dp]
        L.orc_lm_step.restype = C.c_int
        L.orc_sub_lm.argtypes = [C.c_void_p, C.c_int, C.POINTER(Options)]
        L.orc_sub_lm.restype = C.c_int
        L.orc_sub_lm_trace.argtypes = [C.c_void_p, C.c_int, C.POINTER(Options), _dp, _dp, _ip, C.c_int]
        L.orc_sub_lm_trace.restype = C.c_int
        L.orc_lambda_next.argtypes = [C.c_double, C.c_int, C.c_double]
        L.orc_lambda_next.restype = C.c_double
        L.orc_ratio_rule.argtypes = [C.POINTER(C.c_double), C.c_double, C.c_double, C.POINTER(C.c_int)]
        L.orc_ratio_rule.restype = C.c_int
        L.orc_run.argtypes = [C.c_void_p, C.POINTER(Options), C.POINTER(Report)]
        L.orc_default_options.argtypes = [C.POINTER(Options)]
        _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    lib().orc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    if "rho0" in kw and "rho" not in kw:
        o.rho = o.rho0
    return o


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def rodrigues(w):
    R = np.zeros(9)
    lib().orc_rodrigues(_f64(w), R)
    return R.reshape(3, 3)


def rotation_log(R):
    w = np.zeros(3)
    lib().orc_rotation_log(_f64(R).reshape(-1), w)
    return w


def project(R, t, intr, X):
    """Returns (uv, Jc 2x6, Jx 2x3, depth)."""
    uv, Jc, Jx = np.zeros(2), np.zeros(12), np.zeros(6)
    z = lib().orc_project(_f64(R).reshape(-1), _f64(t), _f64(intr), _f64(X), uv, Jc, Jx)
    return uv, Jc.reshape(2, 6), Jx.reshape(2, 3), z


def project_k1(R, t, intr, k1, X):
    """With the radial parameter k1: returns (uv, Jc 2x8, Jx 2x3, depth)."""
    uv, Jc, Jx = np.zeros(2), np.zeros(16), np.zeros(6)
    z = lib().orc_project_k1(_f64(R).reshape(-1), _f64(t), _f64(intr), float(k1), _f64(X), uv, Jc, Jx)
    return uv, Jc.reshape(2, 8), Jx.reshape(2, 3), z


def lambda_next(lam, accepted, lambda0):
    return lib().orc_lambda_next(float(lam), int(accepted), float(lambda0))


def ratio_rule_sequence(values, stop_ratio=1.01, grace=1):
    """Feeds values[1:] to the oracle's stop rule, starting from best =
    values[0]; returns the index (into values) of the value that stopped the
    loop, or None."""
    best, g = C.c_double(float(values[0])), C.c_int(int(grace))
    for i, v in enumerate(values[1:], start=1):
        if lib().orc_ratio_rule(C.byref(best), float(v), float(stop_ratio), C.byref(g)):
            return i
    return None


def median(a):
    a = _f64(a).copy()
    return lib().orc_median(a, a.size)


class Oracle:
    """One oracle context over a problem dict (see paper_1910_08138_gb300.synth).
    With intrinsics (default: the problem's "intrinsics" entry) the focal
    length and the radial parameter of every camera are unknowns too, starting
    from cam_intr's f and the problem's "cam_k1" (0 when absent)."""

    def __init__(self, prob, intrinsics=None):
        L = lib()
        self.M = int(prob["cam_pose"].shape[0])
        self.N = int(prob["points"].shape[0])
        self.K = int(prob["obs_cam"].shape[0])
        winv = prob.get("obs_winv")
        self._winv = None if winv is None else _f64(winv, (self.K, 3))
        self._h = L.orc_create(self.M, self.N, self.K, _f64(prob["cam_pose"]), _f64(prob["cam_intr"]),
                               _f64(prob["points"]), _i32(prob["obs_cam"]), _i32(prob["obs_point"]),
                               _f64(prob["obs_xy"]),
                               None if self._winv is None else self._winv.ctypes.data_as(C.c_void_p),
                               _i32(prob["cam_subblock"]))
        self.L = L.orc_num_subblocks(self._h)
        self.P = L.orc_num_instances(self._h)
        if intrinsics is None:
            intrinsics = bool(prob.get("intrinsics", False))
        if intrinsics:
            k1 = prob.get("cam_k1")
            self._k1 = None if k1 is None else _f64(k1, (self.M,))
            L.orc_enable_intrinsics(self._h, None if self._k1 is None else self._k1.ctypes.data_as(C.c_void_p))
        self.cd = L.orc_camera_dim(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    # topology
    def instances(self):
        p, s = np.zeros(self.P, np.int32), np.zeros(self.P, np.int32)
        lib().orc_instances(self._h, p, s)
        return p, s

    def sub_cameras(self, l):
        out = np.zeros(self.M, np.int32)
        n = lib().orc_sub_cameras(self._h, l, out)
        return out[:n]

    # state
    def cameras(self):
        out = np.zeros((self.M, 6))
        lib().orc_get_cameras(self._h, out)
        return out

    def set_cameras(self, pose):
        lib().orc_set_cameras(self._h, _f64(pose, (self.M, 6)))

    def camera_rt(self):
        """(M, 12): the rotation matrix (row-major) and translation of every
        camera, as held."""
        R, t = np.zeros((self.M, 9)), np.zeros((self.M, 3))
        lib().orc_get_camera_rt(self._h, R, t)
        return np.concatenate([R, t], axis=1)

    def set_camera_rt(self, Rt):
        Rt = _f64(Rt, (self.M, 12))
        lib().orc_set_camera_rt(self._h, np.ascontiguousarray(Rt[:, :9]), np.ascontiguousarray(Rt[:, 9:]))

    def intrinsics(self):
        """(M, 2): focal length and radial parameter k1 of every camera."""
        fk = np.zeros((self.M, 2))
        lib().orc_get_intrinsics(self._h, fk)
        return fk

    def set_intrinsics(self, fk):
        lib().orc_set_intrinsics(self._h, _f64(fk, (self.M, 2)))

    def points(self):
        X, a = np.zeros((self.N, 3)), np.zeros(self.N, np.uint8)
        lib().orc_get_points(self._h, X, a)
        return X, a

    def set_points(self, X, active=None):
        a = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        lib().orc_set_points(self._h, _f64(X, (self.N, 3)),
                             None if a is None else a.ctypes.data_as(C.c_void_p))
        self._keep = a

    def instance_state(self):
        Xl, Wl = np.zeros((self.P, 3)), np.zeros((self.P, 6))
        lib().orc_get_instances(self._h, Xl, Wl)
        return Xl, Wl

    def set_instance_state(self, Xl, Wl):
        lib().orc_set_instances(self._h, _f64(Xl, (self.P, 3)), _f64(Wl, (self.P, 6)))

    def weights(self):
        w = np.zeros(self.K)
        lib().orc_get_weights(self._h, w)
        return w

    def set_weights(self, w):
        lib().orc_set_weights(self._h, _f64(w))

    # evaluations
    def residuals(self):
        v = np.zeros((self.K, 2))
        lib().orc_residuals(self._h, v)
        return v

    def jacobians(self):
        Jc, Jx = np.zeros((self.K, 2 * self.cd)), np.zeros((self.K, 6))
        lib().orc_jacobians(self._h, Jc, Jx)
        return Jc.reshape(self.K, 2, self.cd), Jx.reshape(self.K, 2, 3)

    def sigma0(self):
        return lib().orc_sigma0(self._h)

    def rms(self):
        return lib().orc_rms(self._h)

    def covariance(self, ids):
        ids = _i32(ids)
        out = np.zeros((ids.size, 9))
        lib().orc_covariance(self._h, ids, ids.size, out)
        return out.reshape(-1, 3, 3)

    def camera_scale(self):
        s = np.zeros(self.M)
        lib().orc_camera_scale(self._h, s)
        return s

    def robust_weights(self, t_v=4.0, downweight=1e-4):
        return lib().orc_robust_weights(self._h, t_v, downweight)

    def intersect(self, tp_only=False, **opts):
        o = default_options(**opts)
        return lib().orc_intersect(self._h, C.byref(o), int(tp_only))

    def intersect_points(self, ids, tp_only=False, **opts):
        """Eq. bars for the listed points only."""
        o = default_options(**opts)
        ids = _i32(ids)
        return lib().orc_intersect_points(self._h, C.byref(o), ids, ids.size, int(tp_only))

    def robust_weights_cams(self, cams, t_v=4.0, downweight=1e-4):
        """Robust weights of the observations of the listed cameras only."""
        cams = _i32(cams)
        return lib().orc_robust_weights_cams(self._h, cams, cams.size, t_v, downweight)

    def sub_cost(self, l):
        return lib().orc_sub_cost(self._h, l)

    def rcs(self, l, lam):
        n = self.cd * len(self.sub_cameras(l))
        S, y = np.zeros((n, n)), np.zeros(n)
        lib().orc_rcs(self._h, l, lam, S, y)
        return S, y

    def lm_step(self, l, lam):
        n = self.cd * len(self.sub_cameras(l))
        _, s = self.instances()
        nP = int((s == l).sum())
        dc, dx = np.zeros(max(n, 1)), np.zeros((max(nP, 1), 3))
        Fb, Ft = C.c_double(), C.c_double()
        r = lib().orc_lm_step(self._h, l, lam, C.byref(Fb), C.byref(Ft), dc, dx)
        return r, Fb.value, Ft.value, dc[:n], dx[:nP]

    def sub_lm(self, l, **opts):
        o = default_options(**opts)
        return lib().orc_sub_lm(self._h, l, C.byref(o))

    def sub_lm_trace(self, l, cap=64, **opts):
        """The LM loop of sub-block l with its trace: (iterations, lambda used,
        result of each step, F_l after each step)."""
        o = default_options(**opts)
        F, lam, acc = np.zeros(cap), np.zeros(cap), np.zeros(cap, np.int32)
        it = lib().orc_sub_lm_trace(self._h, l, C.byref(o), F, lam, acc, cap)
        n = min(it, cap)
        return it, lam[:n], acc[:n], F[:n]

    def run(self, **opts):
        o = default_options(**opts)
        r = Report()
        lib().orc_run(self._h, C.byref(o), C.byref(r))
        return {"sigma0": r.sigma0, "rms": r.rms, "sigma0_initial": r.sigma0_initial,
                "outer": r.outer, "inner_total": r.inner_total, "deleted_points": r.deleted_points,
                "active_points": r.active_points, "active_obs": r.active_obs,
                "robust_started_at": r.robust_started_at,
                "sigma0_hist": list(r.sigma0_hist[:min(r.outer, 128)])}
