"""Per-camera error measures between covariance blocks (oracle).

rel_fro   ||S_i - R_i||_F / ||R_i||_F per 9x9 block (R the reference).
norm_err  the same after the symmetric scaling D = diag(R_i)^-1/2, so that
          every parameter counts alike (k1, k2 variances dominate rel_fro).
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


def paper_err(S: np.ndarray, R: np.ndarray, cams: np.ndarray) -> np.ndarray:
    e = np.abs(cams).mean(axis=0)
    O = np.sqrt(np.outer(e, e))
    return (np.sqrt(np.abs(S - R)) / O).mean(axis=(-2, -1))
