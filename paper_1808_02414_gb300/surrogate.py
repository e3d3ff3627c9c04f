"""Thin ctypes binding of include/ccov_surrogate.h (the learned covariance
surrogate).  Argument marshalling only: features, targets, training and
prediction all run in the CUDA kernels of libccov.so.  Device arrays are CUDA
torch tensors; parameters and normalisation travel as host float32 numpy
arrays."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import ccov

N_FEATURES, N_OUTPUTS, HIDDEN = 64, 45, 256
N_PARAMS = N_FEATURES * HIDDEN + HIDDEN + 2 * (HIDDEN * HIDDEN + HIDDEN) + N_OUTPUTS * HIDDEN + N_OUTPUTS
N_NORM = 2 * N_FEATURES + 2 * N_OUTPUTS

EXPORTED = ["ccov_surrogate_features", "ccov_surrogate_targets", "ccov_surrogate_create",
            "ccov_surrogate_fit_normalization", "ccov_surrogate_set_normalization",
            "ccov_surrogate_get_normalization", "ccov_surrogate_set_params", "ccov_surrogate_get_params",
            "ccov_surrogate_backward", "ccov_surrogate_get_grads", "ccov_surrogate_adam",
            "ccov_surrogate_train", "ccov_surrogate_predict", "ccov_surrogate_destroy",
            "ccov_surrogate_last_error", "ccov_surrogate_gauge_rows", "ccov_surrogate_set_gauge",
            "ccov_surrogate_get_gauge", "ccov_surrogate_fit_gauge", "ccov_surrogate_apply_gauge"]


def _dev(t, dtype_name: str):
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    return t.data_ptr()


def _rows(n: int, **arrays):
    """Each array holds n rows of the given width (the C calls read n rows)."""
    for name, (a, width) in arrays.items():
        if a.numel() != n * width:
            raise ValueError(f"{name} must hold {n} rows of {width} values")


def features(ctx: ccov.Context):
    """(features (n, 64) float32, L_z (n, 9, 9) float64) on the device, from
    a context that has run ccov_information."""
    import torch
    f = torch.empty((ctx.n, N_FEATURES), dtype=torch.float32, device="cuda")
    d = torch.empty((ctx.n, 9, 9), dtype=torch.float64, device="cuda")
    ctx._check(ccov.load().ccov_surrogate_features(ctx._h, _dev(f, "float32"), _dev(d, "float64")))
    return f, d


def gauge_rows(ctx: ccov.Context, scale):
    """Q_i = H_i L_c (n, 9, 7) float64 on the device, from a context that has
    run ccov_information and ccov_nullspace; scale: L_z from `features`."""
    import torch
    if tuple(scale.shape) != (ctx.n, 9, 9):
        raise ValueError("scale must be (n, 9, 9)")
    q = torch.empty((ctx.n, 9, 7), dtype=torch.float64, device="cuda")
    ctx._check(ccov.load().ccov_surrogate_gauge_rows(ctx._h, _dev(scale, "float64"), _dev(q, "float64")))
    return q


def targets(scale, sigma):
    """Cholesky-form training targets (n, 45) float32 from exact blocks."""
    import torch
    n = int(scale.shape[0])
    t = torch.empty((n, N_OUTPUTS), dtype=torch.float32, device="cuda")
    s = ccov.load().ccov_surrogate_targets(n, _dev(scale, "float64"), _dev(sigma.reshape(n, 81), "float64"),
                                           _dev(t, "float32"), None)
    if s != ccov.CCOV_OK:
        raise ccov.CcovError(s, "ccov_surrogate_targets")
    return t


class Surrogate:
    """ccov_surrogate: the model, its Adam state and its workspace."""

    def __init__(self, params: np.ndarray, max_batch: int = 4096, stream=None):
        L = ccov.load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (N_PARAMS,):
            raise ValueError(f"expected {N_PARAMS} parameters")
        h = C.c_void_p()
        s = L.ccov_surrogate_create(p.ctypes.data, int(max_batch), stream, C.byref(h))
        self._h = h
        self.max_batch = int(max_batch)
        self._check(s)

    def _check(self, s: int):
        if s != ccov.CCOV_OK:
            L = ccov.load()
            msg = L.ccov_surrogate_last_error(self._h).decode() if self._h else ""
            raise ccov.CcovError(s, msg or L.ccov_status_string(s).decode())

    def fit_normalization(self, feats, targs):
        self._check(ccov.load().ccov_surrogate_fit_normalization(
            self._h, _dev(feats, "float32"), _dev(targs, "float32"), int(feats.shape[0])))

    def set_normalization(self, norm: np.ndarray):
        a = np.ascontiguousarray(norm, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_set_normalization(self._h, a.ctypes.data))

    def normalization(self) -> np.ndarray:
        a = np.empty(N_NORM, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_get_normalization(self._h, a.ctypes.data))
        return a

    def set_gauge(self, M: np.ndarray):
        a = np.ascontiguousarray(M, dtype=np.float64).reshape(49)
        self._check(ccov.load().ccov_surrogate_set_gauge(self._h, a.ctypes.data))

    def gauge(self) -> np.ndarray:
        a = np.empty(49, dtype=np.float64)
        self._check(ccov.load().ccov_surrogate_get_gauge(self._h, a.ctypes.data))
        return a.reshape(7, 7)

    def fit_gauge(self, scale, q, sigma):
        """M by least squares over the cameras of (L_z, Q, exact blocks)."""
        n = int(scale.shape[0])
        _rows(n, scale=(scale, 81), q=(q, 63), sigma=(sigma, 81))
        self._check(ccov.load().ccov_surrogate_fit_gauge(
            self._h, _dev(scale, "float64"), _dev(q, "float64"), _dev(sigma.reshape(n, 81), "float64"), n))

    def apply_gauge(self, scale, q):
        """T_i = chol((Z_ii^-1 + Q_i M Q_i^T)^-1) (n, 9, 9) on the device."""
        import torch
        n = int(scale.shape[0])
        _rows(n, scale=(scale, 81), q=(q, 63))
        out = torch.empty((n, 9, 9), dtype=torch.float64, device="cuda")
        self._check(ccov.load().ccov_surrogate_apply_gauge(
            self._h, _dev(scale, "float64"), _dev(q, "float64"), n, _dev(out, "float64")))
        return out

    def set_params(self, params: np.ndarray):
        a = np.ascontiguousarray(params, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_set_params(self._h, a.ctypes.data))

    def params(self) -> np.ndarray:
        a = np.empty(N_PARAMS, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_get_params(self._h, a.ctypes.data))
        return a

    def grads(self) -> np.ndarray:
        a = np.empty(N_PARAMS, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_get_grads(self._h, a.ctypes.data))
        return a

    def backward(self, feats, targs, idx) -> float:
        loss = C.c_float()
        self._check(ccov.load().ccov_surrogate_backward(
            self._h, _dev(feats, "float32"), _dev(targs, "float32"), int(feats.shape[0]), _dev(idx, "int32"),
            int(idx.numel()), C.byref(loss)))
        return loss.value

    def adam(self, lr: float):
        self._check(ccov.load().ccov_surrogate_adam(self._h, float(lr)))

    def train(self, feats, targs, idx, lr: float) -> np.ndarray:
        """idx: (steps, batch) int32 CUDA tensor; returns the per-step losses."""
        steps, batch = int(idx.shape[0]), int(idx.shape[1])
        losses = np.empty(steps, dtype=np.float32)
        self._check(ccov.load().ccov_surrogate_train(
            self._h, _dev(feats, "float32"), _dev(targs, "float32"), int(feats.shape[0]), _dev(idx, "int32"),
            batch, steps, float(lr), losses.ctypes.data))
        return losses

    def predict(self, feats, scale):
        import torch
        n = int(feats.shape[0])
        out = torch.empty((n, 9, 9), dtype=torch.float64, device="cuda")
        self._check(ccov.load().ccov_surrogate_predict(
            self._h, _dev(feats, "float32"), _dev(scale, "float64"), n, _dev(out, "float64")))
        return out

    def close(self):
        if self._h:
            ccov.load().ccov_surrogate_destroy(self._h)
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
