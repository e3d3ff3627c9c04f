"""Projection model and its Jacobian by forward-mode dual numbers (oracle).

Sec. 4.1 writes the projection as p(X_j, P_i) = Phi_i(c_i R(r_i)(X_j - C_i)),
where Phi_i divides by the third coordinate and then applies radial
distortion.  The cameras here carry 9 values {r (angle-axis), t, f, k1, k2}
with X_c = R(r) X + t (the translation form of the same model), and
    u_hat = f * (1 + k1 rho^2 + k2 rho^4) * (X_c[0], X_c[1]) / X_c[2],
    rho^2 = (X_c[0]^2 + X_c[1]^2) / X_c[2]^2.
Sec. 4 assumes the Jacobian J is "provided numerically"; this module obtains it
by propagating dual numbers (value + 12 partial derivatives) through the
projection, a derivation that does not use any hand-written derivative.

The paper's own camera (Sec. 3, Sec. 4.1), model "centre8": 8 values
{r (angle-axis), C (centre), c (focal length), k (radial)},
    X_c = R(r) (X - C),  u_hat = c * (1 + k rho^2) * (X_c[0], X_c[1]) / X_c[2]
(reading of Phi: divide by the third coordinate, then distort; multiplying by
c before the division would cancel it).  The default model "rt9" is the one
above.
"""
from __future__ import annotations

import numpy as np

N_CAM = 9
N_PT = 3
N_CAM_OF = {"rt9": 9, "centre8": 8}


class Dual:
    """Vectorised first-order dual numbers: value v (...,) and gradient d (..., k)."""

    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=float)
        self.d = np.asarray(d, dtype=float)

    @staticmethod
    def _lift(x, like):
        if isinstance(x, Dual):
            return x
        x = np.asarray(x, dtype=float)
        return Dual(np.broadcast_to(x, like.v.shape), np.zeros(like.d.shape))

    def __add__(self, o):
        o = Dual._lift(o, self)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        o = Dual._lift(o, self)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return Dual._lift(o, self) - self

    def __mul__(self, o):
        o = Dual._lift(o, self)
        return Dual(self.v * o.v, self.d * o.v[..., None] + o.d * self.v[..., None])

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual._lift(o, self)
        q = self.v / o.v
        return Dual(q, (self.d - o.d * q[..., None]) / o.v[..., None])

    def __rtruediv__(self, o):
        return Dual._lift(o, self) / self


def dsqrt(x: Dual) -> Dual:
    r = np.sqrt(x.v)
    return Dual(r, x.d / (2.0 * r)[..., None])


def dsin(x: Dual) -> Dual:
    return Dual(np.sin(x.v), x.d * np.cos(x.v)[..., None])


def dcos(x: Dual) -> Dual:
    return Dual(np.cos(x.v), -x.d * np.sin(x.v)[..., None])


def dwhere(mask, a: Dual, b: Dual) -> Dual:
    return Dual(np.where(mask, a.v, b.v), np.where(mask[..., None], a.d, b.d))


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0]]


def rotate(r, X):
    """R(r) X by Rodrigues' formula X + a (r x X) + b r x (r x X),
    a = sin(theta)/theta, b = (1 - cos theta)/theta^2, theta = |r|.
    Below theta^2 = 1e-8 the Taylor series of a and b in theta^2 is used."""
    th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2]
    small = th2.v < 1e-8
    safe = dwhere(small, Dual._lift(1.0, th2), th2)
    th = dsqrt(safe)
    a_big = dsin(th) / th
    b_big = (1.0 - dcos(th)) / safe
    a_small = 1.0 - th2 * (1.0 / 6.0) + th2 * th2 * (1.0 / 120.0)
    b_small = 0.5 - th2 * (1.0 / 24.0) + th2 * th2 * (1.0 / 720.0)
    a = dwhere(small, a_small, a_big)
    b = dwhere(small, b_small, b_big)
    rx = _cross(r, X)
    rrx = _cross(r, rx)
    return [X[k] + a * rx[k] + b * rrx[k] for k in range(3)]


def project(cam, X):
    """u_hat(P, X) on lists of Dual (or plain arrays lifted to Dual)."""
    r, t, f, k1, k2 = cam[0:3], cam[3:6], cam[6], cam[7], cam[8]
    RX = rotate(r, X)
    Xc = [RX[k] + t[k] for k in range(3)]
    x = Xc[0] / Xc[2]
    y = Xc[1] / Xc[2]
    rho2 = x * x + y * y
    g = 1.0 + k1 * rho2 + k2 * rho2 * rho2
    return [f * g * x, f * g * y]


def project_centre(cam, X):
    """u_hat of the 8-value centre camera on lists of Dual."""
    r, C, c, k = cam[0:3], cam[3:6], cam[6], cam[7]
    Xc = rotate(r, [X[q] - C[q] for q in range(3)])
    x = Xc[0] / Xc[2]
    y = Xc[1] / Xc[2]
    g = 1.0 + k * (x * x + y * y)
    return [c * g * x, c * g * y]


def project_values(cams_t: np.ndarray, pts_t: np.ndarray) -> np.ndarray:
    """u_hat for paired rows of cameras (t, 9) and points (t, 3)."""
    t = cams_t.shape[0]
    z = np.zeros((t, 0))
    cam = [Dual(cams_t[:, k], z) for k in range(N_CAM)]
    X = [Dual(pts_t[:, k], z) for k in range(N_PT)]
    u = project(cam, X)
    return np.stack([u[0].v, u[1].v], axis=1)


def jacobians(cams: np.ndarray, pts: np.ndarray, obs_cam: np.ndarray,
              obs_pt: np.ndarray, model: str = "rt9"):
    """Per observation (i, j) in S: J_c = d u_hat / d P_i (t, 2, nc) and
    J_p = d u_hat / d X_j (t, 2, 3), by seeding nc + 3 dual directions
    (nc = 9 for "rt9", 8 for "centre8")."""
    nc = N_CAM_OF[model]
    cams_t = cams[obs_cam]
    pts_t = pts[obs_pt]
    t = cams_t.shape[0]
    k = nc + N_PT
    eye = np.eye(k)
    cam = [Dual(cams_t[:, c], np.broadcast_to(eye[c], (t, k))) for c in range(nc)]
    X = [Dual(pts_t[:, c], np.broadcast_to(eye[nc + c], (t, k))) for c in range(N_PT)]
    u = (project_centre if model == "centre8" else project)(cam, X)
    J = np.stack([u[0].d, u[1].d], axis=1)          # (t, 2, nc + 3)
    return J[:, :, :nc].copy(), J[:, :, nc:].copy()


def rotation_matrix(r: np.ndarray) -> np.ndarray:
    """R(r) for one angle-axis vector, by rotating the three unit vectors."""
    z = np.zeros((3, 0))
    rr = [Dual(np.full(3, r[k]), z) for k in range(3)]
    E = np.eye(3)
    cols = rotate(rr, [Dual(E[k], z) for k in range(3)])
    return np.stack([c.v for c in cols], axis=0)  # row k = component k of R e_col
