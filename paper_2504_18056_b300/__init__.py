"""Thin Python binding of libgmcs.so, the C ABI declared in include/gmcs.h.

Argument marshalling only: every step of the per-frame particle update runs in
the library's CUDA kernels. Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA memory); they must be C-contiguous with the dtypes the
header names (float32 poses / points, float64 weights, int32 indices).

The library is loaded from this package's directory. If it is missing, import
fails loudly: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmcs.so")
DIAG_PATH = os.path.join(HERE, "libgmcs_diag.so")

OK = 0
E_INVALID, E_OOM, E_CUDA, E_CAPACITY, E_STATE, E_NONFINITE, E_BUDGET, E_IO = -1, -2, -3, -4, -5, -6, -7, -8
PENDING = 1
TABLE_F32, TABLE_BF16, TABLE_F16 = 0, 1, 2
LAYOUT_DENSE, LAYOUT_COLUMNS = 0, 1
RESAMPLE_ALWAYS, RESAMPLE_ESS_HALF, RESAMPLE_NEVER, RESAMPLE_PRUNE = 0, 1, 2, 3
MAX_NB = 8
MODEL_FIELD, MODEL_GICP = 0, 1
KNN_MAX = 32


class GmcsError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class Config(C.Structure):
    _fields_ = [("sigma", C.c_float), ("r_t", C.c_float), ("eps", C.c_float), ("lambda_", C.c_float),
                ("theta_max", C.c_float), ("t_max", C.c_float), ("w_min", C.c_float), ("k_nb", C.c_int),
                ("steps", C.c_int), ("table_dtype", C.c_int), ("resample", C.c_int), ("propagate", C.c_int),
                ("loop_recent", C.c_int), ("prune_w", C.c_float), ("prune_lr", C.c_float), ("model", C.c_int),
                ("knn", C.c_int), ("cov_eps", C.c_float), ("gicp_tau", C.c_float), ("kf_overlap", C.c_float),
                ("kf_voxel", C.c_float), ("kf_h", C.c_float), ("table_layout", C.c_int), ("seed", C.c_uint64)]


class Grid(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("h", C.c_double), ("n", C.c_int * 3)]


class StepOut(C.Structure):
    _fields_ = [("estimate", C.c_double * 12), ("ess", C.c_double), ("max_w", C.c_double),
                ("log_norm", C.c_double), ("argmax", C.c_int), ("resampled", C.c_int),
                ("frame", C.c_uint32), ("status", C.c_int), ("pruned", C.c_int), ("kf_inserted", C.c_int),
                ("overlap", C.c_double)]

    def as_dict(self):
        return {"estimate": np.array(list(self.estimate)), "ess": self.ess, "max_w": self.max_w,
                "log_norm": self.log_norm, "argmax": self.argmax, "resampled": bool(self.resampled),
                "frame": self.frame, "status": self.status, "pruned": self.pruned,
                "kf_inserted": bool(self.kf_inserted), "overlap": self.overlap}


class Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("frames", C.c_uint64), ("profiling", C.c_int), ("n_kinds", C.c_int),
                ("kind", C.c_char_p * 16), ("kind_launches", C.c_uint64 * 16), ("kind_ms", C.c_double * 16)]


class ServerStats(C.Structure):
    _fields_ = [("frames", C.c_uint64), ("ticks", C.c_uint64), ("sessions", C.c_int), ("pad", C.c_int),
                ("used_bytes", C.c_uint64), ("budget_bytes", C.c_uint64), ("evals", C.c_double), ("span_s", C.c_double),
                ("busy_s", C.c_double), ("mean_sessions_per_tick", C.c_double), ("latency_p50_s", C.c_double), ("latency_p99_s", C.c_double),
                ("latency_max_s", C.c_double), ("latency_mean_s", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


_LIB = None

_SIGS = {
    "gmcs_config_default": (None, [C.POINTER(Config)]),
    "gmcs_create": (C.c_int, [C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "gmcs_destroy": (C.c_int, [C.c_void_p]),
    "gmcs_init_particles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_add_keyframe": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Grid), C.c_void_p,
                                    C.POINTER(C.c_int)]),
    "gmcs_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_double), C.POINTER(StepOut)]),
    "gmcs_last_result": (C.c_int, [C.c_void_p, C.POINTER(StepOut)]),
    "gmcs_set_path": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "gmcs_predict": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p, C.c_uint32]),
    "gmcs_select": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gmcs_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gmcs_move": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "gmcs_loglik": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_loglik_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "gmcs_weigh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(StepOut)]),
    "gmcs_resample": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "gmcs_prune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                             C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "gmcs_get_particles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gmcs_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gmcs_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gmcs_checkpoint_info": (C.c_int, [C.c_char_p, C.POINTER(Config), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_uint32)]),
    "gmcs_get_kf_poses": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_get_table": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_get_records": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_void_p]),
    "gmcs_state_version": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "gmcs_point_covariances": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_overlap": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gmcs_set_kf_poses": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "gmcs_get_frame_diag": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gmcs_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_uint32)]),
    "gmcs_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "gmcs_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "gmcs_reset_stats": (C.c_int, [C.c_void_p]),
    "gmcs_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "gmcs_strerror": (C.c_char_p, [C.c_int]),
    "gmcs_resample_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "gmcs_server_create": (C.c_int, [C.POINTER(Config), C.c_uint64, C.c_int, C.POINTER(C.c_void_p)]),
    "gmcs_server_destroy": (C.c_int, [C.c_void_p]),
    "gmcs_server_start": (C.c_int, [C.c_void_p]),
    "gmcs_server_stop": (C.c_int, [C.c_void_p]),
    "gmcs_server_pump": (C.c_int, [C.c_void_p]),
    "gmcs_server_set_inflight": (C.c_int, [C.c_void_p, C.c_int]),
    "gmcs_server_set_tick_work": (C.c_int, [C.c_void_p, C.c_double]),
    "gmcs_server_open": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.POINTER(C.c_int)]),
    "gmcs_server_context": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "gmcs_server_ready": (C.c_int, [C.c_void_p, C.c_int]),
    "gmcs_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "gmcs_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(StepOut), C.POINTER(C.c_double)]),
    "gmcs_server_drain": (C.c_int, [C.c_void_p]),
    "gmcs_server_close": (C.c_int, [C.c_void_p, C.c_int]),
    "gmcs_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "gmcs_server_reset_stats": (C.c_int, [C.c_void_p]),
}
NOALLOC_MAX_P = 262144


def lib():
    """Load libgmcs.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2504_18056_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def strerror(code):
    return lib().gmcs_strerror(int(code)).decode()


def _check(rc, where):
    if rc != OK:
        raise GmcsError(rc, where)
    return rc


def _ptr(a, dtype=None):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    if dtype is not None and a.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {a.dtype}")
    return C.c_void_p(a.ctypes.data)


def _dbl(vals, n):
    arr = (C.c_double * n)(*[float(v) for v in np.asarray(vals, np.float64).reshape(-1)[:n]])
    return arr


def resample_noalloc(w, u, anc, stream=None):
    """Systematic resampling of device weights into device ancestors without any
    allocation (gmcs_resample_noalloc); enqueued on `stream` (default: torch's
    current stream), not synchronised."""
    st = _current_stream() if stream is None else C.c_void_p(int(stream))
    _check(lib().gmcs_resample_noalloc(_ptr(w), int(w.shape[0]), float(u), _ptr(anc), st), "gmcs_resample_noalloc")
    return anc


# diagnostics library (include/gmcs_diag.h): calibration, not the particle-update ABI
_DIAG_SIGS = {
    "gmcs_probe_gather": (C.c_int, [C.c_uint64, C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "gmcs_probe_ffma": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
}
_DIAG = None


def diag_lib():
    """Load libgmcs_diag.so (raises if it has not been built)."""
    global _DIAG
    if _DIAG is None:
        if not os.path.exists(DIAG_PATH):
            raise ImportError(f"{DIAG_PATH} is missing; build it with `python -m paper_2504_18056_b300.build`")
        L = C.CDLL(DIAG_PATH)
        for name, (res, args) in _DIAG_SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _DIAG = L
    return _DIAG


def probe_ffma(stream=None):
    """(FP32 FMA rate in TFLOP/s, multiprocessor count) of the current device (gmcs_probe_ffma)."""
    st = _current_stream() if stream is None else C.c_void_p(int(stream))
    r, n = C.c_double(), C.c_int()
    _check(diag_lib().gmcs_probe_ffma(st, C.byref(r), C.byref(n)), "gmcs_probe_ffma")
    return r.value, n.value


def probe_gather(buffer_bytes, rec_bytes=32, stream=None):
    """Random record-gather rate (GB/s) from a device buffer (gmcs_probe_gather, diagnostics library)."""
    st = _current_stream() if stream is None else C.c_void_p(int(stream))
    r = C.c_double()
    _check(diag_lib().gmcs_probe_gather(C.c_uint64(int(buffer_bytes)), int(rec_bytes), st, C.byref(r)),
           "gmcs_probe_gather")
    return r.value


def checkpoint_info(path):
    """Check a checkpoint file on the host (gmcs_checkpoint_info, no device needed);
    returns (config, P, K, frame) or raises GmcsError (E_IO for a bad file)."""
    cfg, P, K, fr = Config(), C.c_int(), C.c_int(), C.c_uint32()
    _check(lib().gmcs_checkpoint_info(os.fsencode(path), C.byref(cfg), C.byref(P), C.byref(K), C.byref(fr)),
           "gmcs_checkpoint_info")
    return cfg, P.value, K.value, fr.value


def default_config(**kw):
    cfg = Config()
    lib().gmcs_config_default(C.byref(cfg))
    for k, v in kw.items():
        k2 = "lambda_" if k == "lambda" else k
        if not hasattr(cfg, k2):
            raise KeyError(k)
        setattr(cfg, k2, v)
    return cfg


def make_grid(g):
    gr = Grid()
    for a in range(3):
        gr.origin[a] = float(g["origin"][a])
        gr.n[a] = int(g["dims"][a])
    gr.h = float(g["h"])
    return gr


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


class Filter:
    """One filter session: a gmcs_ctx with its particles, keyframe tables and scratch."""

    def __init__(self, max_particles, max_keyframes, max_points, stream=None, _ctx=None, **config):
        self.cfg = default_config(**config)
        if _ctx is not None:             # a view of a context owned elsewhere (a server session)
            self.ctx, self.owned = _ctx, False
            return
        self.ctx, self.owned = C.c_void_p(), True
        st = _current_stream() if stream is None else C.c_void_p(int(stream))
        _check(lib().gmcs_create(C.byref(self.cfg), int(max_particles), int(max_keyframes), int(max_points), st,
                                 C.byref(self.ctx)), "gmcs_create")

    def close(self):
        if self.ctx and self.owned:
            lib().gmcs_destroy(self.ctx)
        self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- state
    def init_particles(self, poses, logw=None):
        _check(lib().gmcs_init_particles(self.ctx, _ptr(poses), int(poses.shape[0]), _ptr(logw)), "gmcs_init_particles")

    def add_keyframe(self, points, grid, kf_poses=None):
        kid = C.c_int()
        gr = make_grid(grid) if isinstance(grid, dict) else grid
        _check(lib().gmcs_add_keyframe(self.ctx, _ptr(points), int(points.shape[0]), C.byref(gr), _ptr(kf_poses),
                                       C.byref(kid)), "gmcs_add_keyframe")
        return kid.value

    def set_path(self, now, kf_path=None):
        kp = None if kf_path is None else np.ascontiguousarray(kf_path, np.float64)
        _check(lib().gmcs_set_path(self.ctx, float(now), _ptr(kp)), "gmcs_set_path")

    def sizes(self):
        P, K, f = C.c_int(), C.c_int(), C.c_uint32()
        _check(lib().gmcs_get_sizes(self.ctx, C.byref(P), C.byref(K), C.byref(f)), "gmcs_get_sizes")
        return P.value, K.value, f.value

    # --- the frame
    def step(self, scan, delta_T, cov, u=None, sync=True):
        out = StepOut()
        uu = C.c_double(u) if u is not None else None
        _check(lib().gmcs_step(self.ctx, _ptr(scan), int(scan.shape[0]), _dbl(delta_T, 12), _dbl(cov, 36),
                               C.byref(uu) if uu is not None else None, C.byref(out) if sync else None), "gmcs_step")
        return out.as_dict() if sync else None

    def last_result(self):
        out = StepOut()
        _check(lib().gmcs_last_result(self.ctx, C.byref(out)), "gmcs_last_result")
        return out.as_dict()

    # --- stages
    def predict(self, delta_T, cov, z=None, frame=0):
        _check(lib().gmcs_predict(self.ctx, _dbl(delta_T, 12), _dbl(cov, 36), _ptr(z), int(frame)), "gmcs_predict")

    def select(self, nbr_out=None):
        _check(lib().gmcs_select(self.ctx, _ptr(nbr_out)), "gmcs_select")
        return nbr_out

    def eval(self, scan, ll=None, g=None, mom=None):
        _check(lib().gmcs_eval(self.ctx, _ptr(scan), int(scan.shape[0]), _ptr(ll), _ptr(g), _ptr(mom)), "gmcs_eval")

    def move(self, scan):
        _check(lib().gmcs_move(self.ctx, _ptr(scan), int(scan.shape[0])), "gmcs_move")

    def loglik(self, xi, scan, ll):
        _check(lib().gmcs_loglik(self.ctx, _ptr(xi), _ptr(scan), int(scan.shape[0]), _ptr(ll)), "gmcs_loglik")
        return ll

    def loglik_backward(self, xi, scan, grad_ll, grad_xi):
        _check(lib().gmcs_loglik_backward(self.ctx, _ptr(xi), _ptr(scan), int(scan.shape[0]), _ptr(grad_ll),
                                          _ptr(grad_xi)), "gmcs_loglik_backward")
        return grad_xi

    def weigh(self, ll, w_out=None):
        res = StepOut()
        _check(lib().gmcs_weigh(self.ctx, _ptr(ll), _ptr(w_out), C.byref(res)), "gmcs_weigh")
        return res.as_dict()

    def resample(self, w, u, anc):
        _check(lib().gmcs_resample(self.ctx, _ptr(w), int(w.shape[0]), float(u), _ptr(anc)), "gmcs_resample")
        return anc

    def prune(self, x, w, ll, argmax, u, anc, logw):
        """Dead-particle pruning of given weights (gmcs_prune); returns the dead count."""
        d = C.c_int()
        _check(lib().gmcs_prune(self.ctx, _ptr(x), _ptr(w), _ptr(ll), int(x.shape[0]), int(argmax), float(u),
                                _ptr(anc), _ptr(logw), C.byref(d)), "gmcs_prune")
        return d.value

    # --- checkpoint
    def save(self, path):
        _check(lib().gmcs_save(self.ctx, os.fsencode(path)), "gmcs_save")

    def load(self, path):
        _check(lib().gmcs_load(self.ctx, os.fsencode(path)), "gmcs_load")

    # --- readback
    def get_particles(self, poses=None, logw=None):
        _check(lib().gmcs_get_particles(self.ctx, _ptr(poses), _ptr(logw)), "gmcs_get_particles")

    def get_kf_poses(self, k, poses):
        _check(lib().gmcs_get_kf_poses(self.ctx, int(k), _ptr(poses)), "gmcs_get_kf_poses")

    def set_kf_poses(self, k, poses):
        _check(lib().gmcs_set_kf_poses(self.ctx, int(k), _ptr(poses)), "gmcs_set_kf_poses")

    def frame_diag(self, ll=None, w=None, anc=None, nbr=None):
        _check(lib().gmcs_get_frame_diag(self.ctx, _ptr(ll), _ptr(w), _ptr(anc), _ptr(nbr)), "gmcs_get_frame_diag")

    def overlap(self, scan, T_rel):
        """Overlap rate of a scan with the last keyframe (gmcs_overlap)."""
        r = C.c_double()
        _check(lib().gmcs_overlap(self.ctx, _ptr(scan), int(scan.shape[0]), _dbl(T_rel, 12), C.byref(r)),
               "gmcs_overlap")
        return r.value

    def point_covariances(self, pts, cov=None):
        """GICP point covariances of a cloud (gmcs_point_covariances): n x 6 doubles."""
        if cov is None:
            cov = np.zeros((pts.shape[0], 6))
        _check(lib().gmcs_point_covariances(self.ctx, _ptr(pts), int(pts.shape[0]), _ptr(cov)),
               "gmcs_point_covariances")
        return cov

    def get_table(self, k, vals):
        _check(lib().gmcs_get_table(self.ctx, int(k), _ptr(vals)), "gmcs_get_table")

    def state_version(self):
        """Counter bumped by every call that changes poses, neighbours or keyframes."""
        v = C.c_uint64()
        _check(lib().gmcs_state_version(self.ctx, C.byref(v)), "gmcs_state_version")
        return v.value

    def get_records(self, k, c0, n, coef):
        """Stored coefficients c0..c7 of cells [c0, c0 + n) of table k into coef (n x 8 float32)."""
        _check(lib().gmcs_get_records(self.ctx, int(k), int(c0), int(n), _ptr(coef)), "gmcs_get_records")

    def particles(self):
        P, _, _ = self.sizes()
        poses = np.zeros((P, 12), np.float32)
        logw = np.zeros(P, np.float64)
        self.get_particles(poses, logw)
        return poses, logw

    # --- instrumentation
    def set_profiling(self, on=True):
        _check(lib().gmcs_set_profiling(self.ctx, 1 if on else 0), "gmcs_set_profiling")

    def stats(self):
        s = Stats()
        _check(lib().gmcs_get_stats(self.ctx, C.byref(s)), "gmcs_get_stats")
        kinds = {s.kind[k].decode(): {"launches": int(s.kind_launches[k]), "ms": float(s.kind_ms[k])}
                 for k in range(s.n_kinds)}
        return {"launches": int(s.launches), "frames": int(s.frames), "kinds": kinds}

    def reset_stats(self):
        _check(lib().gmcs_reset_stats(self.ctx), "gmcs_reset_stats")

    def device_bytes(self):
        b = C.c_uint64()
        _check(lib().gmcs_device_bytes(self.ctx, C.byref(b)), "gmcs_device_bytes")
        return int(b.value)


class Server:
    """Continuous batching of frames from many sessions (gmcs_server_*)."""

    def __init__(self, budget_bytes, max_sessions=32, background=True, **config):
        self.cfg = default_config(**config)
        self.srv = C.c_void_p()
        _check(lib().gmcs_server_create(C.byref(self.cfg), int(budget_bytes), int(max_sessions), C.byref(self.srv)),
               "gmcs_server_create")
        if background:
            _check(lib().gmcs_server_start(self.srv), "gmcs_server_start")

    def close(self):
        if self.srv:
            lib().gmcs_server_destroy(self.srv)
            self.srv = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, max_particles, max_keyframes, max_points, table_bytes=0, seed=0):
        """Session id, or None when it does not fit the budget (GMCS_E_BUDGET)."""
        sid = C.c_int()
        rc = lib().gmcs_server_open(self.srv, int(max_particles), int(max_keyframes), int(max_points),
                                    C.c_uint64(int(table_bytes)), C.c_uint64(int(seed)), C.byref(sid))
        if rc == E_BUDGET:
            return None
        _check(rc, "gmcs_server_open")
        return sid.value

    def session(self, sid):
        """A Filter view of the session's context, for setup and readback."""
        ctx = C.c_void_p()
        _check(lib().gmcs_server_context(self.srv, int(sid), C.byref(ctx)), "gmcs_server_context")
        return Filter(0, 0, 0, _ctx=ctx)

    def ready(self, sid):
        _check(lib().gmcs_server_ready(self.srv, int(sid)), "gmcs_server_ready")

    def submit(self, sid, scan, delta_T, cov):
        t = C.c_uint64()
        _check(lib().gmcs_server_submit(self.srv, int(sid), _ptr(scan), int(scan.shape[0]), _dbl(delta_T, 12),
                                        _dbl(cov, 36), C.byref(t)), "gmcs_server_submit")
        return t.value

    def poll(self, ticket):
        """None while pending, else (result dict, latency seconds)."""
        out = StepOut()
        lat = C.c_double()
        rc = lib().gmcs_server_poll(self.srv, C.c_uint64(ticket), C.byref(out), C.byref(lat))
        if rc == PENDING:
            return None
        _check(rc, "gmcs_server_poll")
        return out.as_dict(), lat.value

    def pump(self):
        _check(lib().gmcs_server_pump(self.srv), "gmcs_server_pump")

    def set_inflight(self, ticks):
        _check(lib().gmcs_server_set_inflight(self.srv, int(ticks)), "gmcs_server_set_inflight")

    def set_tick_work(self, max_evals):
        """Cap (particles x points x steps) on the frames a tick gathers; 0 lifts it."""
        _check(lib().gmcs_server_set_tick_work(self.srv, float(max_evals)), "gmcs_server_set_tick_work")

    def drain(self):
        _check(lib().gmcs_server_drain(self.srv), "gmcs_server_drain")

    def close_session(self, sid):
        _check(lib().gmcs_server_close(self.srv, int(sid)), "gmcs_server_close")

    def stats(self):
        st = ServerStats()
        _check(lib().gmcs_server_get_stats(self.srv, C.byref(st)), "gmcs_server_get_stats")
        return st.as_dict()

    def reset_stats(self):
        _check(lib().gmcs_server_reset_stats(self.srv), "gmcs_server_reset_stats")
