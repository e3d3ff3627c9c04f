"""Blocks of the Fisher information matrix M = J^T Sigma_u^-1 J (oracle).

Sec. 3 (normal equation system): M = J^T Sigma_u^-1 J with Sigma_u block
diagonal in 2x2 blocks, one per observation (i, j) in S.  With the parameter
order theta = {P_1..P_n, X_1..X_m} (Sec. 4.1), M has the camera blocks
U_i = sum_j J_c^T Sigma^-1 J_c (9x9), the point blocks A_j (3x3) and the
off-diagonal blocks W_ij = J_c^T Sigma^-1 J_p (9x3) of each observation.
"""
from __future__ import annotations

import numpy as np

from . import camera


def obs_information(scene) -> np.ndarray:
    """Sigma_u^-1 per observation, (t, 2, 2)."""
    if scene.obs_cov is None:
        return np.broadcast_to(np.eye(2) / scene.sigma ** 2, (scene.t, 2, 2))
    return np.linalg.inv(scene.obs_cov)


def model(scene) -> str:
    return getattr(scene, "model", "rt9")


def blocks(scene, Jc=None, Jp=None):
    """Returns U (n,nc,nc), A (m,3,3), W (t,nc,3) and the Jacobians (nc = 9, or
    8 for the centre camera)."""
    if Jc is None:
        Jc, Jp = camera.jacobians(scene.cams, scene.pts, scene.obs_cam, scene.obs_pt, model(scene))
    nc = Jc.shape[2]
    Wu = obs_information(scene)
    JcW = np.einsum("tab,tbc->tac", Jc.transpose(0, 2, 1), Wu)   # (t, nc, 2)
    JpW = np.einsum("tab,tbc->tac", Jp.transpose(0, 2, 1), Wu)   # (t, 3, 2)
    U = np.zeros((scene.n, nc, nc))
    np.add.at(U, scene.obs_cam, np.einsum("tab,tbc->tac", JcW, Jc))
    A = np.zeros((scene.m, 3, 3))
    np.add.at(A, scene.obs_pt, np.einsum("tab,tbc->tac", JpW, Jp))
    W = np.einsum("tab,tbc->tac", JcW, Jp)
    return U, A, W, Jc, Jp


def dense_jacobian(scene, Jc=None, Jp=None) -> np.ndarray:
    """J as a dense (2t) x (nc n + 3m) matrix, cameras first (tiny scenes only)."""
    if Jc is None:
        Jc, Jp = camera.jacobians(scene.cams, scene.pts, scene.obs_cam, scene.obs_pt, model(scene))
    n, m, t = scene.n, scene.m, scene.t
    nc = Jc.shape[2]
    J = np.zeros((2 * t, nc * n + 3 * m))
    for o in range(t):
        i, j = scene.obs_cam[o], scene.obs_pt[o]
        J[2 * o:2 * o + 2, nc * i:nc * i + nc] = Jc[o]
        J[2 * o:2 * o + 2, nc * n + 3 * j:nc * n + 3 * j + 3] = Jp[o]
    return J


def dense_obs_information(scene) -> np.ndarray:
    """Sigma_u^-1 as a dense (2t) x (2t) block-diagonal matrix (tiny scenes)."""
    Wu = obs_information(scene)
    out = np.zeros((2 * scene.t, 2 * scene.t))
    for o in range(scene.t):
        out[2 * o:2 * o + 2, 2 * o:2 * o + 2] = Wu[o]
    return out


def dense_information(scene) -> np.ndarray:
    """M = J^T Sigma_u^-1 J, dense (tiny scenes only)."""
    J = dense_jacobian(scene)
    return J.T @ dense_obs_information(scene) @ J
