"""Per-camera error measures between covariance blocks (oracle).

rel_fro   ||S_i - R_i||_F / ||R_i||_F per 9x9 block (R the reference).
norm_err  the same after the symmetric scaling D = diag(R_i)^-1/2, so that
          every parameter counts alike (k1, k2 variances dominate rel_fro).
pose_err  rel_fro of the 6x6 pose sub-block (r, t) alone: the entries that
          the gauge (the similarity nullspace, Sec. 4.1) acts on, which are
          about 1e-7 of a block's Frobenius norm and so invisible in rel_fro.
intr_err  rel_fro of the 3x3 intrinsic sub-block (f, k1, k2) alone.
paper_err the paper's err (Sec. 6, Eq. relative-error): the mean over the
          block's entries of sqrt(|S_lm - R_lm|) / O_lm with
          O = sqrt(E|P| E|P|^T), E|P| the mean absolute parameter value over
          the cameras.  Reading: the garbled parenthesisation is taken as
          elementwise sqrt of the absolute difference divided elementwise by O,
          averaged over the 81 entries of the 9-parameter block.
"""
from __future__ import annotations

import numpy as np


def rel_fro(S: np.ndarray, R: np.ndarray) -> np.ndarray:
    return np.linalg.norm(S - R, axis=(-2, -1)) / np.linalg.norm(R, axis=(-2, -1))


def norm_err(S: np.ndarray, R: np.ndarray) -> np.ndarray:
    d = 1.0 / np.sqrt(np.abs(np.einsum("...ii->...i", R)))
    Dd = d[..., :, None] * d[..., None, :]
    return np.linalg.norm((S - R) * Dd, axis=(-2, -1)) / np.linalg.norm(R * Dd, axis=(-2, -1))


POSE = slice(0, 6)
INTR = slice(6, 9)


def pose_err(S: np.ndarray, R: np.ndarray) -> np.ndarray:
    return rel_fro(S[..., POSE, POSE], R[..., POSE, POSE])


def intr_err(S: np.ndarray, R: np.ndarray) -> np.ndarray:
    return rel_fro(S[..., INTR, INTR], R[..., INTR, INTR])


def all_errors(S: np.ndarray, R: np.ndarray) -> dict:
    """Every per-block measure above, keyed by name (arrays over the blocks)."""
    return {"rel_fro": rel_fro(S, R), "norm_err": norm_err(S, R), "pose_err": pose_err(S, R),
            "intr_err": intr_err(S, R)}


def paper_err(S: np.ndarray, R: np.ndarray, cams: np.ndarray) -> np.ndarray:
    e = np.abs(cams).mean(axis=0)
    O = np.sqrt(np.outer(e, e))
    return (np.sqrt(np.abs(S - R)) / O).mean(axis=(-2, -1))
