"""Pins of the oracle's gauge nullspace (Sec. 4.1)."""
import numpy as np

from oracle import camera, information, nullspace
from paper_1808_02414_gb300 import synth


def _setup(sc):
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt)
    HP = nullspace.camera_rows(sc, Jc, Jp)
    return Jc, Jp, HP


def test_jacobian_times_nullspace_vanishes():
    sc = synth.ring_scene(n=6, m=40, track_len=3, seed=2)
    Jc, Jp, HP = _setup(sc)
    J = information.dense_jacobian(sc, Jc, Jp)
    H = nullspace.dense_nullspace(sc, HP)
    # Eq. jacobian-nullspace-condition: J H = 0, relative to |J| |H|
    rel = np.abs(J @ H).max() / (np.abs(J).max() * np.abs(H).max())
    assert rel < 1e-14
    assert np.linalg.matrix_rank(H) == 7


def test_per_camera_solve_matches_closed_form():
    sc = synth.ring_scene(n=10, m=200, track_len=4, seed=5)
    _, _, HP = _setup(sc)
    np.testing.assert_allclose(HP, nullspace.camera_rows_closed_form(sc), rtol=0, atol=1e-12)


def test_nullspace_is_orthogonal_to_dense_information():
    sc = synth.ring_scene(n=5, m=30, track_len=3, seed=9)
    _, _, HP = _setup(sc)
    H = nullspace.dense_nullspace(sc, HP)
    M = information.dense_information(sc)
    assert np.abs(M @ H).max() / (np.abs(M).max() * np.abs(H).max()) < 1e-14


def test_translation_and_scale_columns_by_finite_motion():
    """Moving the scene by a finite similarity (exact translation, scale) leaves
    the projections unchanged; the T and mu columns are its derivative."""
    sc = synth.ring_scene(n=4, m=10, track_len=3, seed=1)
    u0 = camera.project_values(sc.cams[sc.obs_cam], sc.pts[sc.obs_pt])
    T = np.array([0.3, -0.2, 0.1])
    mu = 1.7
    cams = sc.cams.copy()
    for i in range(sc.n):
        R = camera.rotation_matrix(cams[i, :3])
        cams[i, 3:6] = mu * cams[i, 3:6] - R @ T
    pts = mu * sc.pts + T
    u1 = camera.project_values(cams[sc.obs_cam], pts[sc.obs_pt])
    np.testing.assert_allclose(u1, u0, rtol=1e-12)
