"""Camera covariances by the paper's route (oracle), Sec. 3 and Sec. 4.2.

The natural covariance is the top-left block of the inverse of the bordered
matrix [M H; H^T 0] (Eq. inversion-of-extended-information-matrix).  Sec. 4.2
conditions it with diagonal S = diag(S_a, S_b) (S Q^-1 S), permutes the point
parameters first, Q_p = [A_p B_p; B_p^T D_p], and inverts Q_p by block matrix
inversion (Eq. block-inversion-Qp): the camera part is the top-left block of
Z_p^-1, Z_p = D_p - B_p^T A_p^-1 B_p (Eq. schur-complement-inversion), and
Sigma_P = S_P Z_s S_P.

Readings (the paper leaves S_a, S_b unspecified): S_a = diag(M)^-1/2 (Jacobi
scaling of the columns of J) and S_b makes each column of S_a H unit-norm.
The result does not depend on S.  Z_p is symmetric indefinite; it is
inverted by LU with partial pivoting (LAPACK getrf/getrs via scipy).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import camera, information, nullspace


def _scales(U, A, HP, HX, mode):
    n, m = U.shape[0], A.shape[0]
    if mode == "none":
        sP, sX, sb = np.ones((n, U.shape[1])), np.ones((m, 3)), np.ones(7)
    elif mode == "jacobi":
        sP = 1.0 / np.sqrt(np.einsum("nii->ni", U))
        sX = 1.0 / np.sqrt(np.einsum("mii->mi", A))
        col = np.sqrt(((sP[:, :, None] * HP) ** 2).sum((0, 1))
                      + ((sX[:, :, None] * HX) ** 2).sum((0, 1)))
        sb = 1.0 / col
    else:
        raise ValueError(mode)
    return sP, sX, sb


def schur_system(scene, scaling="jacobi"):
    """Z_p = D_p - B_p^T A_p^-1 B_p of the (conditioned) permuted bordered
    matrix, dense (9n+7)^2, plus the scale vector of its rows/columns."""
    U, A, W, Jc, Jp = information.blocks(scene)
    HP = nullspace.camera_rows(scene, Jc, Jp)
    HX = nullspace.point_rows(scene.pts)
    return _schur_from_blocks(scene, U, A, W, HP, HX, scaling)


def _schur_from_blocks(scene, U, A, W, HP, HX, scaling):
    n, m, t = scene.n, scene.m, scene.t
    nc = U.shape[1]
    N = nc * n
    sP, sX, sb = _scales(U, A, HP, HX, scaling)
    # conditioned blocks: S_a M S_a and S_a H S_b
    Us = sP[:, :, None] * U * sP[:, None, :]
    As = sX[:, :, None] * A * sX[:, None, :]
    Ws = sP[scene.obs_cam][:, :, None] * W * sX[scene.obs_pt][:, None, :]
    HPs = sP[:, :, None] * HP * sb
    HXs = sX[:, :, None] * HX * sb
    # A_p^-1: block diagonal with the inverted 3x3 point blocks
    Ainv = np.linalg.inv(As)
    ii = (3 * np.arange(m)[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
    jj = (3 * np.arange(m)[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
    Ap_inv = sp.csr_matrix((Ainv.ravel(), (ii.ravel(), jj.ravel())), shape=(3 * m, 3 * m))
    # B_p = [M_XP, H_X]: rows of points, columns of cameras then the 7 of H
    r = (3 * scene.obs_pt[:, None, None] + np.arange(3)[None, :, None]).repeat(nc, 2)
    c = (nc * scene.obs_cam[:, None, None] + np.arange(nc)[None, None, :]).repeat(3, 1)
    rh = (np.arange(3 * m)[:, None]).repeat(7, 1)
    ch = (N + np.arange(7)[None, :]).repeat(3 * m, 0)
    Bp = sp.csr_matrix((np.concatenate([Ws.transpose(0, 2, 1).ravel(), HXs.reshape(-1, 7).ravel()]),
                        (np.concatenate([r.ravel(), rh.ravel()]),
                         np.concatenate([c.ravel(), ch.ravel()]))),
                       shape=(3 * m, N + 7))
    # D_p = [M_PP, H_P; H_P^T, 0]
    Dp = np.zeros((N + 7, N + 7))
    for i in range(n):
        Dp[nc * i:nc * i + nc, nc * i:nc * i + nc] = Us[i]
    Dp[:N, N:] = HPs.reshape(N, 7)
    Dp[N:, :N] = HPs.reshape(N, 7).T
    Zp = Dp - (Bp.T @ (Ap_inv @ Bp)).toarray()
    scale = np.concatenate([sP.ravel(), sb])
    return Zp, scale


def schur_blocks_unscaled(scene):
    """Z (9n x 9n), G (9n x 7) and W7 (7 x 7) with Z_p = [Z, G; G^T, -W7]
    for the unconditioned system: Z = M_PP - M_PX A^-1 M_XP,
    G = H_P - M_PX A^-1 H_X, W7 = H_X^T A^-1 H_X."""
    Zp, _ = schur_system(scene, scaling="none")
    N = Zp.shape[0] - 7
    return Zp[:N, :N], Zp[:N, N:], -Zp[N:, N:]


class _SubScene:
    """The part of a scene that the oracle reads: cameras, points and
    observations (with their information weights)."""

    def __init__(self, cams, pts, obs_cam, obs_pt, sigma, obs_cov):
        self.cams, self.pts, self.obs_cam, self.obs_pt = cams, pts, obs_cam, obs_pt
        self.sigma, self.obs_cov = sigma, obs_cov
        self.n, self.m, self.t = cams.shape[0], pts.shape[0], obs_cam.shape[0]


def schur_rows_unscaled(scene, cams):
    """Block rows Z[i, :] (9 x 9n) of the unconditioned reduced camera matrix
    Z = M_PP - M_PX A^-1 M_XP (Eq. schur-complement-inversion) for the cameras
    i in `cams`, for scenes too large for the dense route.  The definition
    written out per block: Z_ij = [i = j] M_PP,ii - sum over the points p that
    i and j both observe of W_ip A_p^-1 W_jp^T, with W_ip the camera-point
    block of M summed over the observations of p by i.  Only the points that
    camera i observes enter, each with A_p from all of its observations, so
    the information blocks come from the sub-scene of those points.
    Returns {i: array (9, 9n)}."""
    cams = np.unique(np.asarray(cams, dtype=np.int64))
    pts_sel = np.unique(scene.obs_pt[np.isin(scene.obs_cam, cams)])
    keep = np.isin(scene.obs_pt, pts_sel)
    cam_sel = np.unique(scene.obs_cam[keep])
    cam_of = np.full(scene.n, -1, dtype=np.int64)
    cam_of[cam_sel] = np.arange(cam_sel.size)
    pt_of = np.full(scene.m, -1, dtype=np.int64)
    pt_of[pts_sel] = np.arange(pts_sel.size)
    sub = _SubScene(scene.cams[cam_sel], scene.pts[pts_sel], cam_of[scene.obs_cam[keep]],
                    pt_of[scene.obs_pt[keep]], scene.sigma,
                    None if scene.obs_cov is None else scene.obs_cov[keep])
    U, A, W, _, _ = information.blocks(sub)
    Ainv = np.linalg.inv(A)
    # observations of each point of the sub-scene
    order = np.argsort(sub.obs_pt, kind="stable")
    start = np.searchsorted(sub.obs_pt[order], np.arange(sub.m + 1))
    rows = {}
    for i in cams:
        a = cam_of[i]
        row = np.zeros((9, 9 * scene.n))
        row[:, 9 * i:9 * i + 9] = U[a]
        for o in np.nonzero(sub.obs_cam == a)[0]:
            p = sub.obs_pt[o]
            K = W[o] @ Ainv[p]                       # W_ip A_p^-1 (9 x 3)
            for o2 in order[start[p]:start[p + 1]]:
                j = cam_sel[sub.obs_cam[o2]]
                row[:, 9 * j:9 * j + 9] -= K @ W[o2].T
        rows[int(i)] = row
    return rows


def camera_covariance(scene, scaling="jacobi", full=False):
    """Sigma_P = S_P Z_s S_P, Z_s the top-left nc n x nc n block of Z_p^-1
    (nc = 9, or 8 for the centre camera).  Returns the diagonal blocks
    (n, nc, nc), or the whole nc n x nc n matrix."""
    Zp, scale = schur_system(scene, scaling)
    N = Zp.shape[0] - 7
    nc = N // scene.n
    lu = sla.lu_factor(Zp, check_finite=True)
    E = np.zeros((N + 7, N))
    E[np.arange(N), np.arange(N)] = 1.0
    Zinv_cols = sla.lu_solve(lu, E)
    Zs = Zinv_cols[:N, :N]
    sP = scale[:N]
    Sigma = sP[:, None] * Zs * sP[None, :]
    if full:
        return Sigma
    n = scene.n
    return np.stack([Sigma[nc * i:nc * i + nc, nc * i:nc * i + nc] for i in range(n)])
