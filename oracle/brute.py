"""Extended-precision ground truth for tiny scenes (oracle), Sec. 6.

The paper's ground truth (Table 2, Alg. 1, and the accuracy paragraph of
Sec. 6) decomposes the dense information matrix M by SVD, sets exactly the
last seven singular values to zero, inverts the rest, and works with 100
significant digits because double precision "sometimes produces completely
wrong results" (caption of Fig. 3).  This module does the same with mpmath at
a chosen number of digits (default 40).  Its Jacobian is also independent of
the double-precision oracle: it is taken by the complex-step method on a
projection whose rotation is the matrix exponential exp([r]_x), evaluated in
mpmath complex arithmetic with a step of 1e-30.

Everything here is O(N^3) in pure Python: only for N = 9n + 3m below ~100.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np


def _skew(v):
    return mp.matrix([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def _project_mp(cam, X):
    """u_hat with R = expm([r]_x); cam and X are lists of mp numbers."""
    R = mp.expm(_skew(cam[0:3]))
    Xc = [R[k, 0] * X[0] + R[k, 1] * X[1] + R[k, 2] * X[2] + cam[3 + k] for k in range(3)]
    x, y = Xc[0] / Xc[2], Xc[1] / Xc[2]
    rho2 = x * x + y * y
    g = 1 + cam[7] * rho2 + cam[8] * rho2 * rho2
    return [cam[6] * g * x, cam[6] * g * y]


def jacobian_complex_step(cam: np.ndarray, X: np.ndarray, dps=40, h=mp.mpf("1e-30")):
    """(2, 12) Jacobian of one observation w.r.t. [P (9), X (3)]."""
    with mp.workdps(dps):
        base = [mp.mpf(float(v)) for v in list(cam) + list(X)]
        J = mp.matrix(2, 12)
        for k in range(12):
            z = [mp.mpc(v) for v in base]
            z[k] = mp.mpc(base[k], h)
            u = _project_mp(z[:9], z[9:])
            J[0, k] = mp.im(u[0]) / h
            J[1, k] = mp.im(u[1]) / h
        return J


def information_mp(scene, dps=40):
    """Dense M = J^T Sigma_u^-1 J in mpmath, cameras first then points."""
    n, m, t = scene.n, scene.m, scene.t
    Ntot = 9 * n + 3 * m
    with mp.workdps(dps):
        J = mp.zeros(2 * t, Ntot)
        for o in range(t):
            i, j = int(scene.obs_cam[o]), int(scene.obs_pt[o])
            Jo = jacobian_complex_step(scene.cams[i], scene.pts[j], dps)
            for a in range(2):
                for k in range(9):
                    J[2 * o + a, 9 * i + k] = Jo[a, k]
                for k in range(3):
                    J[2 * o + a, 9 * n + 3 * j + k] = Jo[a, 9 + k]
        Winv = mp.zeros(2 * t, 2 * t)
        for o in range(t):
            if scene.obs_cov is None:
                C = mp.matrix([[scene.sigma ** 2, 0], [0, scene.sigma ** 2]])
            else:
                C = mp.matrix([[float(scene.obs_cov[o, a, b]) for b in range(2)] for a in range(2)])
            Ci = mp.inverse(C)
            for a in range(2):
                for b in range(2):
                    Winv[2 * o + a, 2 * o + b] = Ci[a, b]
        return J.T * Winv * J


def pinv_svd_mp(M, gauge_dim=7, dps=40):
    """M^+ from the SVD of M with exactly the last `gauge_dim` singular values
    set to zero; also returns the singular values and the right singular
    vectors of the zeroed ones (a basis of the nullspace)."""
    with mp.workdps(dps):
        U, S, V = mp.svd_r(M)
        N = M.rows
        order = sorted(range(N), key=lambda k: -S[k])
        keep = order[:N - gauge_dim]
        P = mp.zeros(N, N)
        for k in keep:
            s_inv = 1 / S[k]
            for a in range(N):
                va = V[k, a] * s_inv
                if va == 0:
                    continue
                for b in range(N):
                    P[a, b] += va * U[b, k]
        null = mp.matrix(N, gauge_dim)
        for c, k in enumerate(order[N - gauge_dim:]):
            for a in range(N):
                null[a, c] = V[k, a]
        return P, [S[k] for k in order], null


def bordered_inverse_mp(M, H, dps=40):
    """Top-left block of [M H; H^T 0]^-1 (Eq. inversion-of-extended-
    information-matrix) in mpmath."""
    with mp.workdps(dps):
        N, g = M.rows, H.cols
        Q = mp.zeros(N + g, N + g)
        for a in range(N):
            for b in range(N):
                Q[a, b] = M[a, b]
            for c in range(g):
                Q[a, N + c] = H[a, c]
                Q[N + c, a] = H[a, c]
        Qi = mp.inverse(Q)
        out = mp.zeros(N, N)
        for a in range(N):
            for b in range(N):
                out[a, b] = Qi[a, b]
        return out


def to_numpy(A) -> np.ndarray:
    return np.array([[float(A[i, j]) for j in range(A.cols)] for i in range(A.rows)])


def camera_blocks(Sigma_full: np.ndarray, n: int) -> np.ndarray:
    return np.stack([Sigma_full[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(n)])
