"""Pins of the comparison algorithms' oracle (Sec. 6, Table 2, Alg. 4 and 5):
the Moore-Penrose conditions and a 40-digit SVD pseudo-inverse for Alg. 4,
the dense information matrix without the fixed points for Alg. 5, the
gauge-invariant intrinsic blocks, the three-point rule on a hand-made set,
and the paper's accuracy ordering against the 40-digit ground truth."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
from oracle import alternatives, brute, camera, covariance, information, metrics, nullspace  # noqa: E402
from paper_1808_02414_gb300 import synth  # noqa: E402

from _scenes import golden_entries  # noqa: E402


def _H(sc):
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt)
    return nullspace.camera_rows(sc, Jc, Jp).reshape(-1, 7)


def test_zpinv_satisfies_the_moore_penrose_conditions():
    sc = synth.shell_scene(n=12, m=600, seed=3)
    Z, _, _ = covariance.schur_blocks_unscaled(sc)
    Zp = alternatives.zpinv_covariance(sc, full=True)
    H = _H(sc)
    # Z Z+ Z = Z and Z+ Z Z+ = Z+, Jacobi-scaled (d = diag(Z)^-1/2)
    d = 1.0 / np.sqrt(np.diag(Z))
    Zs = d[:, None] * Z * d[None, :]
    Ps = Zp / d[:, None] / d[None, :]
    assert np.abs(Zs @ Ps @ Zs - Zs).max() < 1e-8 * np.abs(Zs).max()
    assert np.abs(Ps @ Zs @ Ps - Ps).max() < 1e-8 * np.abs(Ps).max()
    # Z Z+ and Z+ Z symmetric: both equal the orthogonal projector onto
    # range Z = span(H_P)^perp (compared in the same scaling)
    P = np.eye(Z.shape[0]) - H @ np.linalg.solve(H.T @ H, H.T)
    for got, want in ((d[:, None] * (Z @ Zp) / d[None, :], d[:, None] * P / d[None, :]),
                      ((Zp @ Z) / d[:, None] * d[None, :], P / d[:, None] * d[None, :])):
        assert np.abs(got - want).max() < 1e-7 * np.abs(want).max()
    np.testing.assert_allclose(Zp, Zp.T, rtol=0, atol=1e-12 * np.abs(Zp).max())
    assert np.abs(Zp @ H).max() < 1e-10 * np.abs(Zp).max() * np.abs(H).max()


def test_zpinv_matches_the_svd_pseudo_inverse_at_40_digits():
    """Z formed at 40 digits (Schur complement of the point block of the
    40-digit M from complex-step Jacobians), then its SVD pseudo-inverse with
    exactly seven zero singular values."""
    sc = synth.tiny_scene(n=3, m=12, track_len=3, seed=21)
    with mp.workdps(40):
        M = brute.information_mp(sc)
        N = 9 * sc.n
        Mpp = M[0:N, 0:N]
        Mpx = M[0:N, N:M.rows]
        Mxx = M[N:M.rows, N:M.rows]
        Z = Mpp - Mpx * mp.inverse(Mxx) * Mpx.T
    P, s, _ = brute.pinv_svd_mp(Z, gauge_dim=7)
    want = brute.camera_blocks(brute.to_numpy(P), sc.n)
    got = alternatives.zpinv_covariance(sc)
    assert metrics.rel_fro(got, want).max() < 1e-8


def test_zpinv_keeps_the_gauge_invariant_intrinsics_only():
    sc = synth.workload("ring20")
    nat = covariance.camera_covariance(sc)
    z = alternatives.zpinv_covariance(sc)
    assert metrics.intr_err(z, nat).max() < 1e-9
    assert metrics.pose_err(z, nat).max() > 1e-6          # another gauge: the pose entries move


def test_three_far_points_rule():
    pts = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0], [2.0, 0.5, 0.0], [2.0, 3.0, 0.0], [1.0, 0.0, 0.1]])
    # centroid (1.8, 0.7, 0.02): farthest is point 1 (2.3); farthest from it is
    # point 0 (4.0) before point 3 (3.6); farthest from the x axis is point 3
    assert alternatives.three_far_points(pts) == [1, 0, 3]


def test_fixed_points_equal_the_dense_information_without_those_points():
    sc = synth.tiny_scene(n=4, m=14, track_len=3, seed=2)
    fixed = alternatives.three_far_points(sc.pts)
    M = information.dense_information(sc)
    N = 9 * sc.n
    drop = [N + 3 * j + c for j in fixed for c in range(3)]
    keep = np.setdiff1d(np.arange(M.shape[0]), drop)
    MF = M[np.ix_(keep, keep)]
    d = 1.0 / np.sqrt(np.diag(MF))
    S = d[:, None] * np.linalg.inv(d[:, None] * MF * d[None, :]) * d[None, :]
    want = brute.camera_blocks(S[:N, :N], sc.n)
    got = alternatives.fixed_points_covariance(sc, fixed)
    assert metrics.rel_fro(got, want).max() < 1e-9


def test_fixed_points_bound_the_intrinsics_from_below():
    # nine fixed coordinates remove the seven gauge freedoms and two more:
    # more information, smaller marginal covariance of the intrinsics
    sc = synth.workload("ring20")
    nat = covariance.camera_covariance(sc)
    fx = alternatives.fixed_points_covariance(sc)
    for a, b in zip(nat, fx):
        dd = a[6:9, 6:9] - b[6:9, 6:9]
        assert np.linalg.eigvalsh(0.5 * (dd + dd.T)).min() > -1e-9 * np.abs(a[6:9, 6:9]).max()


@pytest.mark.parametrize("name,sc,gt", golden_entries(), ids=lambda x: x if isinstance(x, str) else "")
def test_accuracy_ordering_against_the_ground_truth(name, sc, gt):
    """Fig. 3: the method (NBUP) is the most accurate; Alg. 4 and 5 fix the
    gauge differently and miss the natural covariance by far more."""
    e6 = metrics.paper_err(covariance.camera_covariance(sc), gt, sc.cams).mean()
    e4 = metrics.paper_err(alternatives.zpinv_covariance(sc), gt, sc.cams).mean()
    e5 = metrics.paper_err(alternatives.fixed_points_covariance(sc), gt, sc.cams).mean()
    assert e6 < 1e-3 * min(e4, e5)
