"""Similarity-gauge nullspace H of the Jacobian (oracle), Sec. 4.1.

A similarity q = [T, s, mu] of the scene leaves every projection unchanged
(Eq. transformation-conditions), so H = d(theta^s)/dq spans the nullspace of J
(Eq. jacobian-nullspace-condition).  Columns are ordered [T (3), omega (3),
mu (1)], omega being the infinitesimal rotation of R(s).  Reading of the signs
(the paper's Delta = theta - theta^s and its +I, +[X]_x entries disagree in
sign, and any per-column sign spans the same space): H is the derivative of
the transformed parameters,
    X' = X + omega x X + dmu X + dT           ->  H_X = [I, -[X]_x, X]
    t' = (1 + dmu) t - R dT                   ->  H_t = [-R, 0, t]
    f, k1, k2 unchanged                       ->  zero rows.
For the paper's centre camera (model "centre8", Sec. 4.1):
    C' = C + omega x C + dmu C + dT           ->  H_C = [I, -[C]_x, C]
(the paper's [I, [C]_x, C] up to the sign of the omega columns), c and k
unchanged -> zero rows.
The rotation rows H_r are not linear in s; as in Eq. rotation-nullspace-
equation they are obtained from J H = 0: for camera i, J_r H_r = B with J_r
the columns of J for r_i on the rows of camera i's observations and B minus
the product of the other non-zero blocks of J and H on those rows.  Which rows
make up the square "red" blocks is lost with Fig. 1; this oracle solves the
system in the least-squares sense over all of the camera's rows, which is
exact because the system is consistent.
"""
from __future__ import annotations

import numpy as np

from . import camera


def skew(v: np.ndarray) -> np.ndarray:
    """[v]_x for v of shape (..., 3)."""
    z = np.zeros(v.shape[:-1])
    return np.stack([np.stack([z, -v[..., 2], v[..., 1]], -1),
                     np.stack([v[..., 2], z, -v[..., 0]], -1),
                     np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def point_rows(pts: np.ndarray) -> np.ndarray:
    """H_X (m, 3, 7) = [I, -[X]_x, X]."""
    m = pts.shape[0]
    H = np.zeros((m, 3, 7))
    H[:, :, 0:3] = np.eye(3)
    H[:, :, 3:6] = -skew(pts)
    H[:, :, 6] = pts
    return H


def _position_rows(scene, i: int) -> np.ndarray:
    """Rows of H for the position values of camera i (3, 7)."""
    if getattr(scene, "model", "rt9") == "centre8":
        C = scene.cams[i, 3:6]
        return np.concatenate([np.eye(3), -skew(C), C[:, None]], 1)
    R = camera.rotation_matrix(scene.cams[i, 0:3])
    return np.concatenate([-R, np.zeros((3, 3)), scene.cams[i, 3:6, None]], 1)


def camera_rows(scene, Jc: np.ndarray, Jp: np.ndarray) -> np.ndarray:
    """H_P (n, nc, 7): position rows in closed form, rotation rows from the
    per-camera system J_r H_r = B (least squares over the camera's rows)."""
    n = scene.n
    nc = Jc.shape[2]
    HX = point_rows(scene.pts)
    H = np.zeros((n, nc, 7))
    for i in range(n):
        H[i, 3:6] = _position_rows(scene, i)
    obs = np.argsort(scene.obs_cam, kind="stable")
    starts = np.searchsorted(scene.obs_cam[obs], np.arange(n + 1))
    for i in range(n):
        rows = obs[starts[i]:starts[i + 1]]
        Jr = Jc[rows][:, :, 0:3].reshape(-1, 3)                     # (2 t_i, 3)
        other = (np.einsum("tab,bc->tac", Jc[rows][:, :, 3:nc], H[i, 3:nc])
                 + np.einsum("tab,tbc->tac", Jp[rows], HX[scene.obs_pt[rows]]))
        B = -other.reshape(-1, 7)
        H[i, 0:3], *_ = np.linalg.lstsq(Jr, B, rcond=None)
    return H


def right_jacobian_inverse(phi: np.ndarray) -> np.ndarray:
    """Inverse right Jacobian of SO(3) (Barfoot, State Estimation for Robotics):
    J_r^-1 = I + 1/2 [phi]_x + (1/theta^2 - (1 + cos theta)/(2 theta sin theta)) [phi]_x^2."""
    th = np.linalg.norm(phi)
    K = skew(phi)
    if th < 1e-5:
        c = 1.0 / 12.0 + th * th / 720.0
    else:
        c = 1.0 / th ** 2 - (1.0 + np.cos(th)) / (2.0 * th * np.sin(th))
    return np.eye(3) + 0.5 * K + c * (K @ K)


def camera_rows_closed_form(scene) -> np.ndarray:
    """H_P with the rotation rows -J_r^-1(r_i) in the omega columns: the exact
    solution of J_r H_r = B for the angle-axis parametrisation (a cross-check
    of the per-camera solve, not used by the oracle's covariance)."""
    n = scene.n
    nc = camera.N_CAM_OF[getattr(scene, "model", "rt9")]
    H = np.zeros((n, nc, 7))
    for i in range(n):
        H[i, 0:3, 3:6] = -right_jacobian_inverse(scene.cams[i, 0:3])
        H[i, 3:6] = _position_rows(scene, i)
    return H


def dense_nullspace(scene, HP: np.ndarray) -> np.ndarray:
    """H as a dense (nc n + 3m) x 7 matrix, cameras first."""
    return np.concatenate([HP.reshape(-1, 7), point_rows(scene.pts).reshape(-1, 7)], 0)
