"""Pins of the oracle's camera covariance (Sec. 3, Sec. 4.2, Sec. 6)."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
from oracle import brute, camera, covariance, information, metrics, nullspace  # noqa: E402
from paper_1808_02414_gb300 import synth  # noqa: E402

from _scenes import golden_entries  # noqa: E402


def _dense_bordered(sc):
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt)
    HP = nullspace.camera_rows(sc, Jc, Jp)
    M = information.dense_information(sc)
    H = nullspace.dense_nullspace(sc, HP)
    return M, H


@pytest.mark.parametrize("name,sc,gt", golden_entries(), ids=lambda x: x if isinstance(x, str) else "")
def test_matches_extended_precision_svd_ground_truth(name, sc, gt):
    """Paper's ground truth (40 digits, fixture written by oracle.brute)."""
    S = covariance.camera_covariance(sc)
    assert metrics.rel_fro(S, gt).max() < 1e-9
    assert metrics.norm_err(S, gt).max() < 1e-8


def test_matches_extended_precision_bordered_inverse_live():
    """Second route: [M H; H^T 0]^-1 in 40-digit arithmetic, M from complex-step J."""
    sc = synth.tiny_scene(n=3, m=12, track_len=3, seed=21)
    M = brute.information_mp(sc)
    _, H = _dense_bordered(sc)
    B = brute.bordered_inverse_mp(M, mp.matrix(H.tolist()))
    want = brute.camera_blocks(brute.to_numpy(B), sc.n)
    got = covariance.camera_covariance(sc)
    assert metrics.rel_fro(got, want).max() < 1e-9


def test_sparse_schur_equals_dense_schur():
    """Z_p assembled sparsely per point equals D - B^T A^-1 B of the explicit
    dense bordered matrix with the point block inverted densely."""
    sc = synth.ring_scene(n=5, m=40, track_len=3, seed=4)
    M, H = _dense_bordered(sc)
    N, m = 9 * sc.n, sc.m
    Q = np.block([[M, H], [H.T, np.zeros((7, 7))]])
    pts = np.arange(N, N + 3 * m)
    rest = np.concatenate([np.arange(N), np.arange(N + 3 * m, N + 3 * m + 7)])
    A = Q[np.ix_(pts, pts)]
    B = Q[np.ix_(pts, rest)]
    D = Q[np.ix_(rest, rest)]
    want = D - B.T @ np.linalg.inv(A) @ B
    Zp, _ = covariance.schur_system(sc, scaling="none")
    np.testing.assert_allclose(Zp, want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_sampled_schur_rows_equal_rows_of_the_whole_schur_complement():
    """The block rows that schur_rows_unscaled builds from the sub-scene of a
    camera's points equal the rows of Z over the whole scene (pinned above
    against the dense bordered matrix), on a scene whose sub-scenes drop
    points, and on one whose tracks leave camera pairs without shared points."""
    for sc in (synth.shell_scene(n=40, m=600, seed=8), synth.ring_scene(n=12, m=60, track_len=2, seed=3)):
        _check_sampled_rows(sc, [0, 7, sc.n - 1])


def _check_sampled_rows(sc, picks):
    Z, _, _ = covariance.schur_blocks_unscaled(sc)
    rows = covariance.schur_rows_unscaled(sc, picks)
    assert sorted(rows) == picks
    for i in picks:
        np.testing.assert_allclose(rows[i], Z[9 * i:9 * i + 9], rtol=0, atol=1e-12 * np.abs(Z).max())


def test_planted_mistake_in_sampled_schur_rows_is_caught(monkeypatch):
    """Drop one observation's camera-point block from the sampled rows (as a
    wrong track lookup would): the comparison with the whole Schur complement
    fails."""
    sc = synth.shell_scene(n=20, m=300, seed=8)
    Z, _, _ = covariance.schur_blocks_unscaled(sc)
    orig = covariance.information.blocks

    def broken(scene, *a, **k):
        U, A, W, Jc, Jp = orig(scene, *a, **k)
        W = W.copy()
        W[0] = 0.0
        return U, A, W, Jc, Jp

    monkeypatch.setattr(covariance.information, "blocks", broken)
    rows = covariance.schur_rows_unscaled(sc, [int(sc.obs_cam[0])])
    i = int(sc.obs_cam[0])
    assert np.abs(rows[i] - Z[9 * i:9 * i + 9]).max() > 1e-6 * np.abs(Z).max()


def test_invariants_of_natural_covariance():
    sc = synth.workload("ring20")
    Sigma = covariance.camera_covariance(sc, full=True)
    Z, G, W7 = covariance.schur_blocks_unscaled(sc)
    nS = np.linalg.norm(Sigma)
    # symmetric and positive definite
    assert np.linalg.norm(Sigma - Sigma.T) / nS < 1e-10
    d = 1.0 / np.sqrt(np.diag(Sigma))
    ev = np.linalg.eigvalsh(d[:, None] * Sigma * d[None, :])
    assert ev.min() > 0.0
    # Sigma_P is a reflexive generalised inverse of Z: Z S Z = Z, S Z S = S
    assert np.linalg.norm(Z @ Sigma @ Z - Z) / np.linalg.norm(Z) < 1e-7
    assert np.linalg.norm(Sigma @ Z @ Sigma - Sigma) / nS < 1e-7
    # Z H_P = 0 and Sigma_P G = 0
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt)
    HP = nullspace.camera_rows(sc, Jc, Jp).reshape(-1, 7)
    assert np.linalg.norm(Z @ HP) / (np.linalg.norm(Z) * np.linalg.norm(HP)) < 1e-13
    assert np.linalg.norm(Sigma @ G) / (nS * np.linalg.norm(G)) < 1e-9


def test_independent_of_conditioning():
    sc = synth.ring_scene(n=6, m=60, track_len=4, seed=8)
    a = covariance.camera_covariance(sc, scaling="jacobi")
    b = covariance.camera_covariance(sc, scaling="none")
    assert metrics.rel_fro(a, b).max() < 1e-6


def test_relabelling_permutes_blocks():
    sc = synth.ring_scene(n=6, m=50, track_len=3, seed=12)
    rng = np.random.default_rng(0)
    pc = rng.permutation(sc.n)
    pp = rng.permutation(sc.m)
    inv_c = np.argsort(pc)
    inv_p = np.argsort(pp)
    ci = inv_c[sc.obs_cam].astype(np.int32)
    pi = inv_p[sc.obs_pt].astype(np.int32)
    order = np.lexsort((ci, pi))
    sc2 = synth.Scene(sc.cams[pc], sc.pts[pp], ci[order], pi[order], sc.obs_u[order], sc.sigma)
    a = covariance.camera_covariance(sc)
    b = covariance.camera_covariance(sc2)
    assert metrics.rel_fro(b, a[pc]).max() < 1e-9


def _fixed_gauge_full(sc, M):
    """SLAM-style gauge: fix r, t of camera 0 and t_x of camera 1, invert the
    remaining full-rank M by Cholesky, pad the fixed rows with zeros."""
    fixed = np.array([0, 1, 2, 3, 4, 5, 9 + 3])
    free = np.setdiff1d(np.arange(M.shape[0]), fixed)
    Mf = M[np.ix_(free, free)]
    L = np.linalg.cholesky(Mf)
    Li = np.linalg.inv(L)
    full = np.zeros_like(M)
    full[np.ix_(free, free)] = Li.T @ Li
    return full


def test_intrinsics_are_gauge_invariant():
    """(f, k1, k2) rows of H vanish, so their covariance is the same under any
    gauge: compare with a fixed-gauge inverse (Sec. 2, SLAM-style fixation)."""
    sc = synth.ring_scene(n=5, m=40, track_len=4, seed=3)
    M, _ = _dense_bordered(sc)
    fixed = _fixed_gauge_full(sc, M)
    S = covariance.camera_covariance(sc, full=True)
    intr = np.concatenate([9 * i + np.arange(6, 9) for i in range(sc.n)])
    a = S[np.ix_(intr, intr)]
    b = fixed[np.ix_(intr, intr)]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8


def test_s_transformation_of_fixed_gauge_gives_natural_covariance():
    """Projecting any gauge's covariance with P = I - H (H^T H)^-1 H^T gives the
    M-P inverse (inner constraints H^T dtheta = 0)."""
    sc = synth.ring_scene(n=5, m=40, track_len=4, seed=3)
    M, H = _dense_bordered(sc)
    fixed = _fixed_gauge_full(sc, M)
    P = np.eye(M.shape[0]) - H @ np.linalg.solve(H.T @ H, H.T)
    inner = P @ fixed @ P.T
    want = np.stack([inner[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(sc.n)])
    got = covariance.camera_covariance(sc)
    assert metrics.rel_fro(got, want).max() < 1e-8


def test_planted_sign_error_in_nullspace_is_caught(monkeypatch):
    """Flip the sign of the mu column of H_X in the oracle: the ground-truth pin fails."""
    orig = nullspace.point_rows

    def broken(pts):
        H = orig(pts)
        H[:, :, 6] *= -1.0
        return H

    monkeypatch.setattr(nullspace, "point_rows", broken)
    name, sc, gt = golden_entries()[0]
    S = covariance.camera_covariance(sc)
    # rel_fro is dominated by the gauge-invariant k2 variance; the scaled
    # measure sees the wrong pose blocks
    assert metrics.norm_err(S, gt).max() > 1e-3
