"""Uncertainty from sub-reconstructions (oracle), Sec. 5.

Test infrastructure: a plain CPU restatement that only tests, smoke() and
bench.py's baseline legs may use.

Sec. 5: the uncertainty of a camera can be evaluated from a sub-reconstruction
of cameras and points in its vicinity; each evaluation gives an upper bound
of the camera's uncertainty, the reconstruction is decomposed several times
and, per camera, the covariance with the smallest trace is kept.  Sec. 6 uses
a camera's neighbours in the view graph (100 of them, or k = 5..320).

Readings (the paper gives no algorithm for the neighbourhoods):
- view graph: cameras i, k are adjacent with weight w_ik = the number of
  points both observe;
- neighbourhood of a seed camera: grown one camera at a time, always adding
  the camera with the largest total weight to the cameras already chosen
  (ties: the smaller index), until it holds k cameras or no camera is
  adjacent;
- decomposition: cameras are tried as seeds in a given order (a random
  permutation, an input); a camera already in a neighbourhood of this
  decomposition is skipped, so every decomposition covers every camera;
- sub-reconstruction of a neighbourhood: its cameras, the points that at least
  two of them observe and those observations; then cameras with fewer than
  two observations and points with fewer than two are dropped, repeatedly,
  until none is left to drop;
- merge: per camera, among the sub-reconstructions that contain it, the 9x9
  block with the smallest trace.
"""
from __future__ import annotations

import numpy as np

from . import covariance


def view_graph(n: int, obs_cam: np.ndarray, obs_pt: np.ndarray) -> list[dict[int, int]]:
    """Adjacency with weights: adj[i][k] = number of points seen by i and k."""
    adj: list[dict[int, int]] = [dict() for _ in range(n)]
    order = np.argsort(obs_pt, kind="stable")
    pts = obs_pt[order]
    cams = obs_cam[order]
    bounds = np.flatnonzero(np.diff(pts)) + 1
    for track in np.split(cams, bounds):
        for a in track:
            for b in track:
                if a != b:
                    adj[int(a)][int(b)] = adj[int(a)].get(int(b), 0) + 1
    return adj


def grow(seed: int, k: int, adj: list[dict[int, int]]) -> list[int]:
    """The neighbourhood of `seed`: best-first by total weight to the chosen set."""
    chosen = {seed}
    score: dict[int, int] = {}
    for nb, w in adj[seed].items():
        score[nb] = score.get(nb, 0) + w
    while len(chosen) < k:
        best, best_s = -1, 0
        for c, sc in score.items():
            if c in chosen:
                continue
            if sc > best_s or (sc == best_s and sc > 0 and c < best):
                best, best_s = c, sc
        if best < 0:
            break
        chosen.add(best)
        for nb, w in adj[best].items():
            if nb not in chosen:
                score[nb] = score.get(nb, 0) + w
    return sorted(chosen)


def plan(scene, k: int, orders: np.ndarray) -> list[list[int]]:
    """Camera sets of the sub-reconstructions of every decomposition, in order."""
    adj = view_graph(scene.n, scene.obs_cam, scene.obs_pt)
    subs = []
    for order in orders:
        covered = np.zeros(scene.n, dtype=bool)
        for c in order:
            if covered[c]:
                continue
            S = grow(int(c), k, adj)
            covered[S] = True
            subs.append(S)
    return subs


class SubScene:
    """A scene made of a subset of another's cameras, points and observations."""

    def __init__(self, cams, pts, obs_cam, obs_pt, obs_u, sigma, obs_cov):
        self.cams, self.pts, self.obs_cam, self.obs_pt, self.obs_u = cams, pts, obs_cam, obs_pt, obs_u
        self.sigma, self.obs_cov = sigma, obs_cov
        self.n, self.m, self.t = cams.shape[0], pts.shape[0], obs_cam.shape[0]


def extract(scene, cams: list[int]):
    """The sub-reconstruction of a camera set: (SubScene, its global camera ids)."""
    cam_keep = np.zeros(scene.n, dtype=bool)
    cam_keep[cams] = True
    obs_keep = cam_keep[scene.obs_cam]
    while True:
        cnt_pt = np.bincount(scene.obs_pt[obs_keep], minlength=scene.m)
        obs_keep &= cnt_pt[scene.obs_pt] >= 2
        cnt_cam = np.bincount(scene.obs_cam[obs_keep], minlength=scene.n)
        drop = obs_keep & (cnt_cam[scene.obs_cam] < 2)
        if not drop.any():
            break
        obs_keep &= ~drop
    used_cams = np.unique(scene.obs_cam[obs_keep])
    used_pts = np.unique(scene.obs_pt[obs_keep])
    cam_of = np.full(scene.n, -1)
    cam_of[used_cams] = np.arange(used_cams.size)
    pt_of = np.full(scene.m, -1)
    pt_of[used_pts] = np.arange(used_pts.size)
    idx = np.flatnonzero(obs_keep)                     # still sorted by point
    sub = SubScene(scene.cams[used_cams], scene.pts[used_pts], cam_of[scene.obs_cam[idx]].astype(np.int32),
                   pt_of[scene.obs_pt[idx]].astype(np.int32), scene.obs_u[idx], scene.sigma,
                   None if scene.obs_cov is None else scene.obs_cov[idx])
    return sub, used_cams


def merge(n: int, results) -> tuple[np.ndarray, np.ndarray]:
    """Per camera the block of smallest trace over (global ids, blocks) results;
    NaN blocks for cameras no sub-reconstruction holds.  Returns (blocks, cover)."""
    out = np.full((n, 9, 9), np.nan)
    best = np.full(n, np.inf)
    cover = np.zeros(n, dtype=np.int32)
    for ids, blocks in results:
        tr = np.trace(blocks, axis1=1, axis2=2)
        for c, b, t in zip(ids, blocks, tr):
            cover[c] += 1
            if t < best[c]:
                best[c] = t
                out[c] = b
    return out, cover


def camera_covariance(scene, k: int, orders: np.ndarray):
    """Sec. 5 pipeline: plan, the natural covariance of every sub-reconstruction
    (oracle route), minimum-trace merge.  Returns (blocks, cover, subs)."""
    subs = plan(scene, k, orders)
    results = []
    for S in subs:
        sub, ids = extract(scene, S)
        if sub.n < 2:
            continue
        results.append((ids, covariance.camera_covariance(sub)))
    out, cover = merge(scene.n, results)
    return out, cover, subs
