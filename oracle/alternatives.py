"""The comparison algorithms of Sec. 6, Table 2 (oracle): Alg. 4 and Alg. 5.

Test infrastructure: a plain CPU restatement that only tests, smoke() and
bench.py's baseline legs may use.

Alg. 4 (Lhuillier and Perriollat, as Sec. 2 describes it): the Moore-Penrose
inverse of the Schur complement Z of the point block (the reduced camera
matrix, Eq. schur-complement-inversion without the border), projected onto
the space orthogonal to the similarity transformation.  Reading: Z H_P = 0
and rank Z = 9n - 7, so Z+ already lies in that space and the projection
leaves it unchanged; the result is Z+ itself.  It differs from the natural
covariance [M+]_PP wherever the gauge acts (the pose entries); the gauge-
invariant intrinsic blocks agree.  Computed here as Z+ = P (Z + H_P H_P^T)^-1 P
with P = I - H_P (H_P^T H_P)^-1 H_P^T, the inverse taken on the Jacobi-scaled
matrix.

Alg. 5 (Polic et al., "three points fixed"): the gauge is fixed by taking
the coordinates of three points that are far from each other out of the
parameters (they are known, their observations still constrain the
cameras).  Reading: the Schur complement of the remaining point blocks,
Z_F = blockdiag(U) - sum over the free points of W A^-1 W^T, is then of full
rank, and Sigma = Z_F^-1 (computed exactly; the reference's TE approximation
of this inverse is not reproduced).  The three points: the point farthest
from the centroid of all points, the point farthest from it, then the point
farthest from the line through those two (ties: the smaller index).
"""
from __future__ import annotations

import numpy as np

from . import covariance, information, nullspace


def _blocks(M: np.ndarray, n: int) -> np.ndarray:
    return np.stack([M[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(n)])


def _spd_inverse(A: np.ndarray) -> np.ndarray:
    d = 1.0 / np.sqrt(np.diag(A))
    return d[:, None] * np.linalg.inv(d[:, None] * A * d[None, :]) * d[None, :]


def zpinv_covariance(scene, full=False):
    """Alg. 4: Z+ of the reduced camera matrix (n, 9, 9 blocks, or 9n x 9n)."""
    Z, G, W7 = covariance.schur_blocks_unscaled(scene)
    U, A, W, Jc, Jp = information.blocks(scene)
    H = nullspace.camera_rows(scene, Jc, Jp).reshape(-1, 7)
    Zr = Z + H @ H.T
    P = np.eye(Z.shape[0]) - H @ np.linalg.solve(H.T @ H, H.T)
    Zp = P @ _spd_inverse(0.5 * (Zr + Zr.T)) @ P
    return Zp if full else _blocks(Zp, scene.n)


def three_far_points(pts: np.ndarray) -> list[int]:
    """The three fixed points of Alg. 5 (see the module docstring)."""
    c = pts.mean(axis=0)
    d0 = np.linalg.norm(pts - c, axis=1)
    p1 = int(np.argmax(d0))                      # argmax returns the first (smallest) index
    d1 = np.linalg.norm(pts - pts[p1], axis=1)
    p2 = int(np.argmax(d1))
    u = (pts[p2] - pts[p1]) / np.linalg.norm(pts[p2] - pts[p1])
    v = pts - pts[p1]
    d2 = np.linalg.norm(v - np.outer(v @ u, u), axis=1)
    p3 = int(np.argmax(d2))
    return [p1, p2, p3]


def fixed_points_covariance(scene, fixed=None, full=False):
    """Alg. 5: Z_F^-1 with the points `fixed` (default: three_far_points)."""
    if fixed is None:
        fixed = three_far_points(scene.pts)
    U, A, W, Jc, Jp = information.blocks(scene)
    n = scene.n
    Z = np.zeros((9 * n, 9 * n))
    for i in range(n):
        Z[9 * i:9 * i + 9, 9 * i:9 * i + 9] += U[i]
    Ainv = np.linalg.inv(A)
    free = np.ones(scene.m, dtype=bool)
    free[list(fixed)] = False
    for j in np.flatnonzero(free):
        obs = np.flatnonzero(scene.obs_pt == j)
        for a in obs:
            for b in obs:
                i, k = scene.obs_cam[a], scene.obs_cam[b]
                Z[9 * i:9 * i + 9, 9 * k:9 * k + 9] -= W[a] @ Ainv[j] @ W[b].T
    S = _spd_inverse(0.5 * (Z + Z.T))
    return S if full else _blocks(S, n)
