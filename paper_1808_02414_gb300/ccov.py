"""Thin ctypes binding of the ccov C ABI (include/ccov.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libccov.so.  Host arrays are numpy arrays; device arrays are CUDA
torch tensors (their data pointers are passed with CCOV_MEM_DEVICE).  If the
library has not been built, importing works but the first call raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .synth import OBS_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccov.so")

CCOV_OK, CCOV_ERR_INVALID_ARG, CCOV_ERR_DEGENERATE, CCOV_ERR_NOT_CONVERGED = 0, 1, 2, 3
CCOV_ERR_TIMEOUT, CCOV_ERR_OOM, CCOV_ERR_CUDA = 4, 5, 6
CCOV_PREC_FP64, CCOV_PREC_MIXED = 0, 1
CCOV_MEM_HOST, CCOV_MEM_DEVICE = 0, 1
CCOV_NULL_PAPER, CCOV_NULL_CLOSED = 0, 1
CCOV_BATCH_AUTO, CCOV_BATCH_PER_SCENE, CCOV_BATCH_GROUPED, CCOV_BATCH_NO_TUNE = 0, 1, 2, 8
CCOV_GAUGE_NATURAL, CCOV_GAUGE_ZPINV, CCOV_GAUGE_FIXED3 = 0, 1, 2
CCOV_CAMERA_RT9, CCOV_CAMERA_CENTRE8 = 0, 1

EXPORTED = ["ccov_create", "ccov_load", "ccov_information", "ccov_schur", "ccov_nullspace",
            "ccov_covariance", "ccov_get_blocks", "ccov_get_schur", "ccov_get_schur_blocks", "ccov_get_stats",
            "ccov_destroy", "ccov_status_string", "ccov_last_error",
            "ccov_spd_inverse_blocks_noalloc", "ccov_batch_covariance", "ccov_batch_create",
            "ccov_batch_create_ex", "ccov_batch_get_info", "ccov_batch_run", "ccov_batch_destroy",
            "ccov_subrecon_plan", "ccov_subrecon_covariance", "ccov_update_observations"]


class CcovError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ccov status {status}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("mixed_slices", C.c_int), ("nullspace_route", C.c_int),
                ("input_memory", C.c_int), ("profile", C.c_int), ("est_cameras", C.c_int),
                ("gauge", C.c_int), ("fixed_points", C.c_int * 3), ("camera_model", C.c_int),
                ("reserved", C.c_int * 1)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("t", C.c_int64), ("N", C.c_int64),
                ("N_pad", C.c_int64), ("ms_information", C.c_double), ("ms_schur", C.c_double),
                ("ms_nullspace", C.c_double), ("ms_covariance", C.c_double),
                ("ms_factor", C.c_double), ("ms_inverse", C.c_double),
                ("bytes_device", C.c_int64), ("launches", C.c_int64), ("ms_gemm", C.c_double),
                ("gemm_flops", C.c_double), ("gemm_launches", C.c_int64), ("est_cameras", C.c_int64),
                ("est_index", C.c_int64 * 16), ("est_rel", C.c_double * 16), ("est_norm", C.c_double * 16),
                ("ms_update", C.c_double), ("update_launches", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        k = int(self.est_cameras)
        for name in ("est_index", "est_rel", "est_norm"):
            d[name] = list(d[name])[:k]
        return d


class SubreconOptions(C.Structure):
    _fields_ = [("cams_per_sub", C.c_int), ("decompositions", C.c_int), ("seed_order", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("form", C.c_int), ("gemm_ctas", C.c_int), ("gemm_stages", C.c_int), ("launches", C.c_int64),
                ("tune_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> C.CDLL:
    """Load libccov.so (built in-tree by paper_1808_02414_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1808_02414_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
    sig = {
        "ccov_create": ([P, I64, P, I64, P, I64, D, P, P, P, C.POINTER(C.c_void_p)], I),
        "ccov_load": ([P, P, P, P, P, I], I),
        "ccov_information": ([P], I),
        "ccov_schur": ([P], I),
        "ccov_nullspace": ([P, P], I),
        "ccov_covariance": ([P, P, I, P], I),
        "ccov_update_observations": ([P, P, I64, P, P, I], I),
        "ccov_get_blocks": ([P, P, P, P], I),
        "ccov_get_schur": ([P, P, P, P], I),
        "ccov_get_schur_blocks": ([P, P, I64, P], I),
        "ccov_get_stats": ([P, C.POINTER(Stats)], I),
        "ccov_destroy": ([P], None),
        "ccov_status_string": ([I], C.c_char_p),
        "ccov_last_error": ([P], C.c_char_p),
        "ccov_test_ozaki_gemm": ([I, I, I, I, P, P, P, P, I, I, I, P], I),
        "ccov_test_ozaki_gemm_wait": ([I, I, I, I, P, P, P, P, I, I, I, P, C.c_longlong, C.c_ulonglong], I),
        "ccov_spd_inverse_blocks_noalloc": ([P, I64, I64, P, P], I),
        "ccov_batch_covariance": ([P, I, P, I], I),
        "ccov_batch_create": ([P, I, P, C.POINTER(C.c_void_p)], I),
        "ccov_batch_create_ex": ([P, I, P, I, C.POINTER(C.c_void_p)], I),
        "ccov_batch_get_info": ([P, C.POINTER(BatchInfo)], I),
        "ccov_subrecon_plan": ([P, I64, I64, I64, C.POINTER(SubreconOptions), I64, I64, P, P,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)], I),
        "ccov_subrecon_covariance": ([P, I64, P, I64, P, I64, D, P, P, C.POINTER(SubreconOptions), P, P,
                                      C.POINTER(C.c_int64)], I),
        "ccov_batch_run": ([P, P], I),
        "ccov_batch_destroy": ([P], None),
        "ccov_surrogate_features": ([P, P, P], I),
        "ccov_surrogate_targets": ([I64, P, P, P, P], I),
        "ccov_surrogate_create": ([P, I64, P, C.POINTER(C.c_void_p)], I),
        "ccov_surrogate_fit_normalization": ([P, P, P, I64], I),
        "ccov_surrogate_set_normalization": ([P, P], I),
        "ccov_surrogate_get_normalization": ([P, P], I),
        "ccov_surrogate_set_params": ([P, P], I),
        "ccov_surrogate_get_params": ([P, P], I),
        "ccov_surrogate_backward": ([P, P, P, I64, P, I64, P], I),
        "ccov_surrogate_get_grads": ([P, P], I),
        "ccov_surrogate_adam": ([P, C.c_float], I),
        "ccov_surrogate_train": ([P, P, P, I64, P, I64, I, C.c_float, P], I),
        "ccov_surrogate_predict": ([P, P, P, I64, P], I),
        "ccov_surrogate_destroy": ([P], None),
        "ccov_surrogate_last_error": ([P], C.c_char_p),
        "ccov_surrogate_gauge_rows": ([P, P, P], I),
        "ccov_surrogate_set_gauge": ([P, P], I),
        "ccov_surrogate_get_gauge": ([P, P], I),
        "ccov_surrogate_fit_gauge": ([P, P, P, P, I64], I),
        "ccov_surrogate_apply_gauge": ([P, P, P, I64, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def obs_records(obs_cam, obs_pt, obs_u) -> np.ndarray:
    rec = np.zeros(len(obs_cam), dtype=OBS_DTYPE)
    rec["cam"] = obs_cam
    rec["pt"] = obs_pt
    rec["u"] = obs_u
    return rec


class Context:
    """One scene on the device (ccov_ctx).  Method names follow the C ABI."""

    def __init__(self, cameras, points, obs, sigma=1.0, obs_cov=None, precision=CCOV_PREC_FP64,
                 mixed_slices=0, nullspace_route=CCOV_NULL_PAPER, stream=None, profile=False, est_cameras=0,
                 gauge=CCOV_GAUGE_NATURAL, fixed_points=(-1, -1, -1), camera_model=CCOV_CAMERA_RT9):
        L = load()
        dev = _is_device(cameras)
        if not dev:
            cameras = np.ascontiguousarray(cameras, dtype=np.float64)
            points = np.ascontiguousarray(points, dtype=np.float64)
            if obs_cov is not None:
                obs_cov = np.ascontiguousarray(obs_cov, dtype=np.float64).reshape(-1, 4)
        n, m = int(cameras.shape[0]), int(points.shape[0])
        t = int(obs.shape[0]) if not dev else int(obs.numel() // 24)
        opt = Options(precision, mixed_slices, nullspace_route,
                      CCOV_MEM_DEVICE if dev else CCOV_MEM_HOST, 1 if profile else 0, est_cameras, gauge,
                      (C.c_int * 3)(*fixed_points), camera_model)
        h = C.c_void_p()
        s = L.ccov_create(_ptr(cameras), n, _ptr(points), m, _ptr(obs), t, float(sigma),
                          _ptr(obs_cov), C.byref(opt), stream, C.byref(h))
        self._h = h
        self.n, self.m, self.t = n, m, t
        self._check(s)

    def _check(self, s: int):
        if s != CCOV_OK:
            L = load()
            msg = L.ccov_last_error(self._h).decode() if self._h else ""
            raise CcovError(s, msg or L.ccov_status_string(s).decode())

    def ccov_load(self, cameras, points, obs, obs_cov=None):
        mem = CCOV_MEM_DEVICE if _is_device(cameras) else CCOV_MEM_HOST
        self._check(load().ccov_load(self._h, _ptr(cameras), _ptr(points), _ptr(obs),
                                     _ptr(obs_cov), mem))

    def ccov_information(self):
        self._check(load().ccov_information(self._h))

    def ccov_schur(self):
        self._check(load().ccov_schur(self._h))

    def ccov_nullspace(self, want_hp=False):
        hp = np.empty((self.n, 9, 7)) if want_hp else None
        self._check(load().ccov_nullspace(self._h, _ptr(hp)))
        return hp

    def ccov_covariance(self, out=None, want_err=False):
        """Returns (n, 9, 9) blocks on the host, or fills `out` (a CUDA tensor)."""
        err = np.empty(self.n) if want_err else None
        if out is None:
            host = np.empty((self.n, 9, 9))
            self._check(load().ccov_covariance(self._h, _ptr(host), CCOV_MEM_HOST, _ptr(err)))
            return (host, err) if want_err else host
        self._check(load().ccov_covariance(self._h, _ptr(out), CCOV_MEM_DEVICE, _ptr(err)))
        return (out, err) if want_err else out

    def ccov_update_observations(self, add, add_cov=None, out=None):
        """Covariance blocks (n, 9, 9) of the scene with the observations `add`
        (ccov_obs records, host) added, from the last ccov_covariance; the
        context keeps its scene.  `out`: a CUDA tensor to fill instead."""
        add = np.ascontiguousarray(add)
        if add_cov is not None:
            add_cov = np.ascontiguousarray(add_cov, dtype=np.float64).reshape(-1, 4)
        k = int(add.shape[0])
        if out is None:
            host = np.empty((self.n, 9, 9))
            self._check(load().ccov_update_observations(self._h, _ptr(add), k, _ptr(add_cov), _ptr(host),
                                                        CCOV_MEM_HOST))
            return host
        self._check(load().ccov_update_observations(self._h, _ptr(add), k, _ptr(add_cov), _ptr(out),
                                                    CCOV_MEM_DEVICE))
        return out

    def ccov_get_blocks(self):
        U = np.empty((self.n, 9, 9))
        A = np.empty((self.m, 3, 3))
        W = np.empty((self.t, 9, 3))
        self._check(load().ccov_get_blocks(self._h, _ptr(U), _ptr(A), _ptr(W)))
        return U, A, W

    def ccov_get_schur(self, want_z=True):
        N = 9 * self.n
        Z = np.empty((N, N)) if want_z else None
        G = np.empty((N, 7))
        W7 = np.empty((7, 7))
        self._check(load().ccov_get_schur(self._h, _ptr(Z), _ptr(G), _ptr(W7)))
        return Z, G, W7

    def ccov_get_stats(self) -> dict:
        st = Stats()
        self._check(load().ccov_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def ccov_get_schur_blocks(self, pairs):
        """Blocks Z_ij (k x 9 x 9) for pairs (i, j), 0 <= j <= i < n (of a
        diagonal block only the lower triangle is defined)."""
        ij = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        out = np.empty((ij.shape[0], 9, 9))
        self._check(load().ccov_get_schur_blocks(self._h, _ptr(ij), ij.shape[0], _ptr(out)))
        return out

    def run(self, out=None):
        """Steps (a)-(d) in order."""
        self.ccov_information()
        self.ccov_schur()
        self.ccov_nullspace()
        return self.ccov_covariance(out)

    def close(self):
        if self._h:
            load().ccov_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_scene(scene, **kw) -> Context:
    if getattr(scene, "model", "rt9") == "centre8":
        kw.setdefault("camera_model", CCOV_CAMERA_CENTRE8)
    return Context(scene.cams, scene.pts, scene.obs_records(), scene.sigma,
                   None if scene.obs_cov is None else scene.obs_cov.reshape(-1, 4), **kw)


def _handles(ctxs):
    return (C.c_void_p * len(ctxs))(*[c._h.value for c in ctxs])


def _first_error(ctxs, s: int):
    if s != CCOV_OK:
        L = load()
        msgs = [L.ccov_last_error(c._h).decode() for c in ctxs]
        raise CcovError(s, next((m for m in msgs if m), L.ccov_status_string(s).decode()))


def ccov_batch_covariance(ctxs, outs=None):
    """Steps (a)-(d) of every context in `ctxs`, all in flight at once.

    Returns a list of (n_i, 9, 9) host arrays, or fills `outs` (CUDA tensors)."""
    if outs is None:
        host = [np.empty((c.n, 9, 9)) for c in ctxs]
        ptrs = (C.c_void_p * len(ctxs))(*[_ptr(h) for h in host])
        _first_error(ctxs, load().ccov_batch_covariance(_handles(ctxs), len(ctxs), ptrs, CCOV_MEM_HOST))
        return host
    ptrs = (C.c_void_p * len(ctxs))(*[_ptr(o) for o in outs])
    _first_error(ctxs, load().ccov_batch_covariance(_handles(ctxs), len(ctxs), ptrs, CCOV_MEM_DEVICE))
    return outs


class Batch:
    """ccov_batch: a batch of contexts recorded once as a CUDA graph."""

    def __init__(self, ctxs, outs_device, form=CCOV_BATCH_AUTO):
        self._ctxs = list(ctxs)
        self._outs = list(outs_device)  # kept alive: the graph writes into them
        ptrs = (C.c_void_p * len(ctxs))(*[_ptr(o) for o in self._outs])
        h = C.c_void_p()
        s = load().ccov_batch_create_ex(_handles(self._ctxs), len(self._ctxs), ptrs, form, C.byref(h))
        self._h = h
        _first_error(self._ctxs, s)

    def info(self) -> dict:
        out = BatchInfo()
        s = load().ccov_batch_get_info(self._h, C.byref(out))
        if s != CCOV_OK:
            raise CcovError(s, "ccov_batch_get_info")
        return out.as_dict()

    def run(self, stream=None):
        _first_error(self._ctxs, load().ccov_batch_run(self._h, stream))
        return self._outs

    def close(self):
        if self._h:
            load().ccov_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def camera_covariances(scene, **kw) -> np.ndarray:
    """Per-camera 9x9 covariance blocks of a scene through the C ABI."""
    with from_scene(scene, **kw) as ctx:
        return ctx.run()


def _subrecon_opts(k: int, orders: np.ndarray):
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    return SubreconOptions(int(k), int(orders.shape[0]), orders.ctypes.data), orders


def subrecon_plan(scene, k: int, orders) -> list[list[int]]:
    """ccov_subrecon_plan: the camera sets of the sub-reconstructions (Sec. 5)."""
    L = load()
    so, keep = _subrecon_opts(k, orders)
    rec = scene.obs_records()
    nsub, total = C.c_int64(), C.c_int64()
    s = L.ccov_subrecon_plan(rec.ctypes.data, scene.t, scene.n, scene.m, C.byref(so), 0, 0, None, None,
                             C.byref(nsub), C.byref(total))
    if s not in (CCOV_OK, CCOV_ERR_INVALID_ARG) or nsub.value == 0:
        raise CcovError(s, "ccov_subrecon_plan")
    ptr = np.empty(nsub.value + 1, np.int32)
    cams = np.empty(max(total.value, 1), np.int32)
    s = L.ccov_subrecon_plan(rec.ctypes.data, scene.t, scene.n, scene.m, C.byref(so), nsub.value, total.value,
                             ptr.ctypes.data, cams.ctypes.data, C.byref(nsub), C.byref(total))
    if s != CCOV_OK:
        raise CcovError(s, "ccov_subrecon_plan")
    return [cams[ptr[q]:ptr[q + 1]].tolist() for q in range(nsub.value)]


def subrecon_covariances(scene, k: int, orders, precision=CCOV_PREC_MIXED, **kw):
    """ccov_subrecon_covariance: merged (n, 9, 9) blocks, cover counts and the
    number of sub-reconstructions solved."""
    L = load()
    so, keep = _subrecon_opts(k, orders)
    opt = Options(precision, kw.get("mixed_slices", 0), kw.get("nullspace_route", CCOV_NULL_PAPER), CCOV_MEM_HOST,
                  0, 0)
    rec = scene.obs_records()
    out = np.empty((scene.n, 9, 9))
    cover = np.empty(scene.n, np.int32)
    nsub = C.c_int64()
    cov = None if scene.obs_cov is None else np.ascontiguousarray(scene.obs_cov.reshape(-1, 4))
    s = L.ccov_subrecon_covariance(_ptr(np.ascontiguousarray(scene.cams)), scene.n,
                                   _ptr(np.ascontiguousarray(scene.pts)), scene.m, rec.ctypes.data, scene.t,
                                   float(scene.sigma), _ptr(cov), C.byref(opt), C.byref(so), out.ctypes.data,
                                   cover.ctypes.data, C.byref(nsub))
    if s != CCOV_OK:
        raise CcovError(s, "ccov_subrecon_covariance")
    return out, cover, nsub.value
