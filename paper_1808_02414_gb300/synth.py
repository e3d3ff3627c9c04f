"""Seeded synthetic SfM scenes (inputs only).

This module draws cameras, points, tracks and noisy image observations with
the shapes of the paper's datasets (Table 1: mean track length N_u/N_X of
about 3-8).  It is the one module that both the CUDA path and the CPU oracle
are fed from; it holds none of the covariance method's arithmetic.  Camera
rotations are built as look-at matrices and handed out as angle-axis vectors;
the observed image points u are synthetic measurements (a look-at projection
plus Gaussian noise) and never enter the covariance, which depends only on
the parameters, the index set S and Sigma_u (Sec. 3, Eq. for M).

Camera vector (9 values): r (angle-axis, 3), t (3), f, k1, k2, with the camera
frame X_c = R(r) X + t, +z forward, and u = f (1 + k1 rho^2 + k2 rho^4) x for
x = X_c[:2] / X_c[2].
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = ["Scene", "ring_scene", "shell_scene", "batch_scenes", "tiny_scene",
           "subscene", "weak_camera_scene", "local_scene", "decomposition_orders", "centre_scene",
           "added_observations", "WORKLOADS", "workload", "surrogate_init", "minibatch_indices",
           "training_scene_specs", "training_scene"]


@dataclass
class Scene:
    cams: np.ndarray          # (n, 9) float64
    pts: np.ndarray           # (m, 3) float64
    obs_cam: np.ndarray       # (t,) int32, observations sorted by point
    obs_pt: np.ndarray        # (t,) int32
    obs_u: np.ndarray         # (t, 2) float64
    sigma: float = 1.0
    obs_cov: np.ndarray | None = None   # (t, 2, 2) float64 or None (sigma^2 I)
    meta: dict = field(default_factory=dict)
    model: str = "rt9"        # "rt9": (r, t, f, k1, k2); "centre8": (r, C, c, k), cams (n, 8)

    @property
    def n(self) -> int:
        return self.cams.shape[0]

    @property
    def m(self) -> int:
        return self.pts.shape[0]

    @property
    def t(self) -> int:
        return self.obs_cam.shape[0]

    def obs_records(self) -> np.ndarray:
        """Observations as the packed 24-byte record array of the C ABI."""
        rec = np.zeros(self.t, dtype=OBS_DTYPE)
        rec["cam"] = self.obs_cam
        rec["pt"] = self.obs_pt
        rec["u"] = self.obs_u
        return rec


OBS_DTYPE = np.dtype([("cam", "<i4"), ("pt", "<i4"), ("u", "<f8", (2,))])


def _look_at(center: np.ndarray, up: np.ndarray) -> np.ndarray:
    """World-to-camera rotation whose third row points from center to origin."""
    z = -center / np.linalg.norm(center)
    if abs(float(z @ up)) > 0.95:
        up = np.array([1.0, 0.0, 0.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z])


def _roll(gamma: float) -> np.ndarray:
    c, s = np.cos(gamma), np.sin(gamma)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _angle_axis(R: np.ndarray) -> np.ndarray:
    """Rotation vector of a proper rotation with angle below pi - 0.1."""
    cos_t = np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)
    theta = np.arccos(cos_t)
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2.0
    if theta < 1e-7:
        return w
    return w * (theta / np.sin(theta))


def _make_cameras(rng, centers: np.ndarray, f_range=(950.0, 1050.0), k_std=1e-3):
    """Look-at cameras with a random roll; the roll is redrawn until the
    rotation angle lies in (0.05, pi - 0.1), where the angle-axis vector read
    off the matrix is well defined and accurate."""
    n = centers.shape[0]
    cams = np.zeros((n, 9))
    Rs = np.zeros((n, 3, 3))
    up = np.array([0.0, 0.0, 1.0])
    for i in range(n):
        R = None
        for _ in range(64):
            base = _look_at(centers[i], up)
            for _ in range(64):
                cand = _roll(rng.uniform(0.0, 2.0 * np.pi)) @ base
                theta = np.arccos(np.clip((np.trace(cand) - 1.0) / 2.0, -1.0, 1.0))
                if 0.05 < theta < np.pi - 0.1:
                    R = cand
                    break
            if R is not None:
                break
            # a camera looking almost straight down -z has a rotation angle
            # near pi for every roll: redraw its direction on the same sphere
            d = rng.normal(size=3)
            centers[i] = np.linalg.norm(centers[i]) * d / np.linalg.norm(d)
        if R is None:
            raise RuntimeError("could not place a camera")
        Rs[i] = R
        cams[i, 0:3] = _angle_axis(R)
        cams[i, 3:6] = -R @ centers[i]
    cams[:, 6] = rng.uniform(f_range[0], f_range[1], n)
    cams[:, 7] = rng.normal(0.0, k_std, n)
    cams[:, 8] = rng.normal(0.0, k_std, n)
    return cams, Rs


def _distinct_tracks(rng, n: int, lengths: np.ndarray) -> list[np.ndarray]:
    """For each point, `lengths[j]` distinct camera indices drawn uniformly."""
    m = lengths.shape[0]
    out: list[np.ndarray | None] = [None] * m
    for L in np.unique(lengths):
        idx = np.nonzero(lengths == L)[0]
        if L * (L - 1) > n:
            # rejection would rarely succeed: take the first L of a random
            # permutation (argsort of uniform keys), a few rows at a time
            for c0 in range(0, idx.size, 4096):
                blk = idx[c0:c0 + 4096]
                rows = np.argsort(rng.random((blk.size, n)), axis=1)[:, :L]
                for k, j in enumerate(blk):
                    out[j] = rows[k]
            continue
        rows = rng.integers(0, n, size=(idx.size, L))
        while True:
            srt = np.sort(rows, axis=1)
            bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0] if L > 1 else np.array([], int)
            if bad.size == 0:
                break
            rows[bad] = rng.integers(0, n, size=(bad.size, L))
        for k, j in enumerate(idx):
            out[j] = rows[k]
    return out  # type: ignore[return-value]


def _observe(rng, cams, Rs, pts, tracks, noise_px=1.0):
    cam_idx = np.concatenate(tracks).astype(np.int32)
    pt_idx = np.repeat(np.arange(len(tracks), dtype=np.int32),
                       [len(tr) for tr in tracks])
    # sort by (point, camera) for a deterministic layout
    order = np.lexsort((cam_idx, pt_idx))
    cam_idx, pt_idx = cam_idx[order], pt_idx[order]
    Xc = np.einsum("tij,tj->ti", Rs[cam_idx], pts[pt_idx]) + cams[cam_idx, 3:6]
    if np.any(Xc[:, 2] <= 0.0):
        raise RuntimeError("synthetic point behind a camera")
    x = Xc[:, :2] / Xc[:, 2:3]
    rho2 = (x * x).sum(1)
    g = 1.0 + cams[cam_idx, 7] * rho2 + cams[cam_idx, 8] * rho2 * rho2
    u = cams[cam_idx, 6:7] * g[:, None] * x + rng.normal(0.0, noise_px, size=x.shape)
    return cam_idx, pt_idx, u


def _ensure_min_obs(rng, n, tracks, min_obs=5):
    counts = np.bincount(np.concatenate(tracks), minlength=n)
    for c in np.nonzero(counts < min_obs)[0]:
        need = min_obs - counts[c]
        cand = [j for j in rng.permutation(len(tracks)) if c not in tracks[j]]
        for j in cand[:need]:
            tracks[j] = np.append(tracks[j], c)
    return tracks


def ring_scene(n=20, m=500, track_len=5, radius=10.0, seed=0, noise_px=1.0,
               sigma=1.0) -> Scene:
    """n cameras on a ring of `radius` in the z=0 plane at angles 2*pi*i/n,
    looking at the origin; m points uniform in [-1/2, 1/2]^3; every point seen
    by exactly `track_len` distinct random cameras."""
    rng = np.random.default_rng(seed)
    ang = 2.0 * np.pi * np.arange(n) / n
    centers = np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n)], 1)
    cams, Rs = _make_cameras(rng, centers)
    pts = rng.uniform(-0.5, 0.5, size=(m, 3))
    tracks = _distinct_tracks(rng, n, np.full(m, min(track_len, n)))
    tracks = _ensure_min_obs(rng, n, tracks)
    ci, pi, u = _observe(rng, cams, Rs, pts, tracks, noise_px)
    return Scene(cams, pts, ci, pi, u, sigma, None,
                 {"kind": "ring", "seed": seed, "n": n, "m": m})


def shell_scene(n=1000, m=100_000, p_geom=1.0 / 7.0, radius=10.0, seed=1,
                noise_px=1.0, sigma=1.0, min_obs=5) -> Scene:
    """n cameras with directions uniform on the sphere at `radius`, looking at
    the origin; m points uniform in the unit cube [-1/2, 1/2]^3; track length
    L = 1 + Geometric(p) (min 2, mean 1/p + 1), capped at n, distinct cameras."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centers = radius * d
    cams, Rs = _make_cameras(rng, centers)
    pts = rng.uniform(-0.5, 0.5, size=(m, 3))
    lengths = np.minimum(1 + rng.geometric(p_geom, size=m), n)
    tracks = _distinct_tracks(rng, n, lengths)
    tracks = _ensure_min_obs(rng, n, tracks, min_obs)
    ci, pi, u = _observe(rng, cams, Rs, pts, tracks, noise_px)
    return Scene(cams, pts, ci, pi, u, sigma, None,
                 {"kind": "shell", "seed": seed, "n": n, "m": m})


def local_scene(n=200, m=20_000, p_geom=1.0 / 7.0, radius=10.0, seed=3, noise_px=1.0, sigma=1.0,
                min_obs=5) -> Scene:
    """A shell scene with visibility locality (as in real reconstructions,
    where a point is seen from nearby viewpoints): n cameras with directions
    uniform on the sphere at `radius`, looking at the origin; m points uniform
    in the unit cube; each point's track is an anchor camera drawn uniformly
    and the L - 1 cameras whose directions are closest to the anchor's,
    L = 1 + Geometric(p) (min 2, mean 1/p + 1), capped at n."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centers = radius * d
    cams, Rs = _make_cameras(rng, centers)
    dirs = centers / np.linalg.norm(centers, axis=1, keepdims=True)
    near = np.argsort(-(dirs @ dirs.T), axis=1, kind="stable")     # row i: cameras by closeness to i
    pts = rng.uniform(-0.5, 0.5, size=(m, 3))
    lengths = np.minimum(1 + rng.geometric(p_geom, size=m), n)
    anchors = rng.integers(0, n, size=m)
    tracks = [near[a, :L].copy() for a, L in zip(anchors, lengths)]
    tracks = _ensure_min_obs(rng, n, tracks, min_obs)
    ci, pi, u = _observe(rng, cams, Rs, pts, tracks, noise_px)
    return Scene(cams, pts, ci, pi, u, sigma, None,
                 {"kind": "local", "seed": seed, "n": n, "m": m})


def centre_scene(sc: Scene) -> Scene:
    """The same cameras and points in the paper's 8-value parametrisation
    {r, C, c, k} (Sec. 3): C = -R^T t, c = f, k = k1 (k2 dropped).  The
    observations are kept: they do not enter the covariance."""
    cams = np.zeros((sc.n, 8))
    for i in range(sc.n):
        th = np.linalg.norm(sc.cams[i, 0:3])
        K = np.array([[0.0, -sc.cams[i, 2], sc.cams[i, 1]], [sc.cams[i, 2], 0.0, -sc.cams[i, 0]],
                      [-sc.cams[i, 1], sc.cams[i, 0], 0.0]])
        R = np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / th ** 2 * K @ K
        cams[i, 0:3] = sc.cams[i, 0:3]
        cams[i, 3:6] = -R.T @ sc.cams[i, 3:6]
        cams[i, 6] = sc.cams[i, 6]
        cams[i, 7] = sc.cams[i, 7]
    return Scene(cams, sc.pts, sc.obs_cam, sc.obs_pt, sc.obs_u, sc.sigma, sc.obs_cov,
                 dict(sc.meta, model="centre8"), "centre8")


def added_observations(sc: Scene, k: int, cams=None, seed=11):
    """k new observations (camera, point) of existing points by existing
    cameras, none already in S: from the cameras `cams` (default: any),
    points drawn uniformly; u = projection + N(0, 1 px^2).  A scene with
    per-observation covariances gives the added ones random SPD 2x2
    covariances (axes uniform in [0.5, 2] px^2, random orientation).  Returns
    (the scene with them merged, sorted by point; the added records, sorted
    by point)."""
    rng = np.random.default_rng(seed)
    have = set(zip(sc.obs_cam.tolist(), sc.obs_pt.tolist()))
    pool = np.arange(sc.n) if cams is None else np.asarray(cams)
    add = set()
    while len(add) < k:
        c, j = int(rng.choice(pool)), int(rng.integers(0, sc.m))
        if (c, j) not in have and (c, j) not in add:
            add.add((c, j))
    add = sorted(add, key=lambda cj: (cj[1], cj[0]))
    ac = np.array([c for c, _ in add], np.int32)
    ap = np.array([j for _, j in add], np.int32)
    Rs = np.stack([_rotation(sc.cams[c, 0:3]) for c in ac])
    if sc.model == "centre8":   # (r, C, c, k): R (X - C), one distortion value
        Xc = np.einsum("tij,tj->ti", Rs, sc.pts[ap] - sc.cams[ac, 3:6])
    else:
        Xc = np.einsum("tij,tj->ti", Rs, sc.pts[ap]) + sc.cams[ac, 3:6]
    x = Xc[:, :2] / Xc[:, 2:3]
    rho2 = (x * x).sum(1)
    g = 1.0 + sc.cams[ac, 7] * rho2
    if sc.model != "centre8":
        g = g + sc.cams[ac, 8] * rho2 * rho2
    au = sc.cams[ac, 6:7] * g[:, None] * x + rng.normal(0.0, 1.0, size=x.shape)
    acov = None
    if sc.obs_cov is not None:
        a = rng.uniform(0.5, 2.0, size=(k, 2))
        th = rng.uniform(0, np.pi, size=k)
        c, s = np.cos(th), np.sin(th)
        Rr = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)
        acov = np.einsum("tij,tj,tkj->tik", Rr, a, Rr)
        acov = 0.5 * (acov + acov.transpose(0, 2, 1))   # exactly symmetric
    cam = np.concatenate([sc.obs_cam, ac])
    pt = np.concatenate([sc.obs_pt, ap])
    u = np.concatenate([sc.obs_u, au])
    order = np.lexsort((cam, pt))
    cov = None if acov is None else np.concatenate([sc.obs_cov, acov])[order]
    merged = Scene(sc.cams, sc.pts, cam[order].astype(np.int32), pt[order].astype(np.int32), u[order],
                   sc.sigma, cov, dict(sc.meta, added=k))
    merged.model = sc.model
    added = Scene(sc.cams, sc.pts, ac, ap, au, sc.sigma, acov, {"kind": "added"})
    added.model = sc.model
    return merged, added


def _rotation(r: np.ndarray) -> np.ndarray:
    th = np.linalg.norm(r)
    K = np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / th ** 2 * K @ K


def decomposition_orders(n: int, decompositions: int, seed=7) -> np.ndarray:
    """Per decomposition of a scene into sub-reconstructions, the order in
    which cameras are tried as seeds: `decompositions` seeded random
    permutations of 0..n-1, (decompositions, n) int32."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(n) for _ in range(decompositions)]).astype(np.int32)


def tiny_scene(n=4, m=14, track_len=3, seed=0, anisotropic=False) -> Scene:
    """A very small ring scene for brute-force checks.  With `anisotropic`,
    each observation gets its own random SPD 2x2 covariance."""
    sc = ring_scene(n=n, m=m, track_len=track_len, seed=seed)
    if anisotropic:
        rng = np.random.default_rng(1000 + seed)
        a = rng.uniform(0.5, 2.0, size=(sc.t, 2))
        th = rng.uniform(0, np.pi, size=sc.t)
        c, s = np.cos(th), np.sin(th)
        Rr = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)
        sc.obs_cov = np.einsum("tij,tj,tkj->tik", Rr, a, Rr)
    return sc


def subscene(sc: Scene, cam_ids: np.ndarray, min_track=2) -> Scene:
    """The sub-reconstruction spanned by `cam_ids`: their observations of points
    still seen by at least `min_track` of them (Sec. 5, sub-reconstructions)."""
    cam_ids = np.asarray(cam_ids)
    remap = -np.ones(sc.n, dtype=np.int64)
    remap[cam_ids] = np.arange(cam_ids.size)
    keep = remap[sc.obs_cam] >= 0
    cnt = np.bincount(sc.obs_pt[keep], minlength=sc.m)
    keep &= cnt[sc.obs_pt] >= min_track
    pts_used = np.unique(sc.obs_pt[keep])
    premap = -np.ones(sc.m, dtype=np.int64)
    premap[pts_used] = np.arange(pts_used.size)
    ci = remap[sc.obs_cam[keep]].astype(np.int32)
    pi = premap[sc.obs_pt[keep]].astype(np.int32)
    order = np.lexsort((ci, pi))
    cov = None if sc.obs_cov is None else sc.obs_cov[keep][order]
    return Scene(sc.cams[cam_ids].copy(), sc.pts[pts_used].copy(), ci[order], pi[order],
                 sc.obs_u[keep][order], sc.sigma, cov,
                 {"kind": "sub", "parent": sc.meta, "n": int(cam_ids.size)})


def weak_camera_scene(n=30, m=3000, keep=6, spread=1e-4, seed=8) -> Scene:
    """A shell scene in which camera 0 keeps only `keep` of its observations,
    of points moved onto a short line segment (plus `spread` of noise): its
    parameters are nearly undetermined, which makes the reduced camera matrix
    badly conditioned (condition number of the scaled matrix about 2e8 at
    spread 1e-4, against 2e4 for the plain shell).  Points left with fewer
    than two observations are removed."""
    sc = shell_scene(n=n, m=m, seed=seed)
    rng = np.random.default_rng(seed)
    mine = np.nonzero(sc.obs_cam == 0)[0]
    pts0 = sc.obs_pt[mine]
    cnt = np.bincount(sc.obs_pt, minlength=sc.m)
    sel = pts0[cnt[pts0] >= 3][:keep]
    keepmask = ~(np.isin(sc.obs_pt, np.setdiff1d(pts0, sel)) & (sc.obs_cam == 0))
    pts = sc.pts.copy()
    s = np.linspace(-0.4, 0.4, sel.size)
    pts[sel] = np.stack([s, 0.1 * s, np.full(sel.size, 0.05)], 1) + spread * rng.standard_normal((sel.size, 3))
    oc, op, ou = sc.obs_cam[keepmask], sc.obs_pt[keepmask], sc.obs_u[keepmask]
    live = np.bincount(op, minlength=sc.m) >= 2
    k2 = live[op]
    newid = np.cumsum(live) - 1
    return Scene(cams=sc.cams, pts=pts[live], obs_cam=oc[k2].astype(np.int32),
                 obs_pt=newid[op[k2]].astype(np.int32), obs_u=ou[k2], sigma=sc.sigma,
                 meta={"kind": "weak_camera", "spread": spread})


def batch_scenes(k=256, n_lo=10, n_hi=300, pts_per_cam=100, p_geom=0.2, seed=4):
    """k independent sub-reconstructions, n_b ~ U{n_lo..n_hi}, m_b = 100 n_b,
    track length 1 + Geometric(p) (mean 6 for p = 0.2)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=k)
    return [shell_scene(n=int(nb), m=int(pts_per_cam * nb), p_geom=p_geom,
                        seed=int(seed * 100003 + b)) for b, nb in enumerate(ns)]


# Named workloads: the camera counts, point counts and track statistics of the
# small ring case, the 1000-camera and the 4000-camera shell scenes.
WORKLOADS = {
    "ring20": dict(fn="ring", n=20, m=500, track_len=5, seed=0),
    "shell1k": dict(fn="shell", n=1000, m=100_000, p_geom=1.0 / 7.0, seed=1),
    "shell4k": dict(fn="shell", n=4000, m=400_000, p_geom=1.0 / 7.0, seed=2),
}


def workload(name: str, **over) -> Scene:
    spec = dict(WORKLOADS[name])
    spec.update(over)
    fn = spec.pop("fn")
    return ring_scene(**spec) if fn == "ring" else shell_scene(**spec)


# ---------------------------------------------------------------------------
# Random draws of the learned surrogate (initial weights, mini-batch order).
# Layer widths 64 -> 256 -> 256 -> 256 -> 45; weights packed W1, b1, ..., W4, b4
# with W of shape (out, in), row-major.
SURROGATE_DIMS = (64, 256, 256, 256, 45)


def surrogate_init(seed=0) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(SURROGATE_DIMS[:-1], SURROGATE_DIMS[1:]):
        bound = np.sqrt(6.0 / a)
        parts.append(rng.uniform(-bound, bound, size=(b, a)).ravel())
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def minibatch_indices(n: int, batch: int, steps: int, seed=0) -> np.ndarray:
    """steps x batch sample indices: consecutive shuffled epochs over range(n)."""
    rng = np.random.default_rng(seed)
    need = steps * batch
    out = np.concatenate([rng.permutation(n) for _ in range(-(-need // n))])[:need]
    return out.astype(np.int32).reshape(steps, batch)


def training_scene_specs(k=2000, n_lo=50, n_hi=500, seed=5):
    """(n, seed) of k training scenes for the surrogate: n ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=k)
    return [(int(nb), int(seed * 100003 + b)) for b, nb in enumerate(ns)]


def training_scene(spec) -> Scene:
    """Shell scene with 100 points per camera and track length 1 + Geometric(1/7) (mean 8)."""
    n, s = spec
    return shell_scene(n=n, m=100 * n, p_geom=1.0 / 7.0, seed=s)
