"""Pins of the error measures (closed-form cases)."""
import numpy as np

from oracle import metrics


def test_rel_fro_and_norm_err_closed_forms():
    R = np.diag([4.0, 1.0, 9.0])[None]
    S = R * 1.01
    np.testing.assert_allclose(metrics.rel_fro(S, R), [0.01])
    np.testing.assert_allclose(metrics.norm_err(S, R), [0.01])


def test_paper_err_closed_form():
    R = np.zeros((1, 9, 9))
    S = np.zeros((1, 9, 9))
    S[0, 0, 0] = 4.0                      # sqrt(|4|) = 2
    cams = np.ones((3, 9)) * 2.0           # E|P| = 2, O = 2
    np.testing.assert_allclose(metrics.paper_err(S, R, cams), [2.0 / 2.0 / 81.0])


def _block(seed=0):
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((30, 9)) * np.array([1e3, 1e3, 1e3, 10, 10, 10, 1e-2, 1e-4, 1e-4])
    return np.linalg.inv(J.T @ J)[None]      # variances spread over ten orders, like a camera block


def test_pose_and_intrinsic_sub_block_errors_see_what_rel_fro_does_not():
    R = _block()
    S = R.copy()
    S[0, 0:6, 0:6] *= 2.0                    # pose sub-block entirely wrong
    assert metrics.rel_fro(S, R)[0] < 1e-6   # invisible in the whole-block measure
    np.testing.assert_allclose(metrics.pose_err(S, R), [1.0])
    assert metrics.norm_err(S, R)[0] > 0.1
    assert metrics.intr_err(S, R)[0] == 0.0
    S = R.copy()
    S[0, 6:9, 6:9] *= 1.5
    np.testing.assert_allclose(metrics.intr_err(S, R), [0.5])
    assert metrics.pose_err(S, R)[0] == 0.0


def test_all_errors_keys_and_zero_on_identity():
    R = _block(1)
    e = metrics.all_errors(R, R)
    assert set(e) == {"rel_fro", "norm_err", "pose_err", "intr_err"}
    assert all(v.max() == 0.0 for v in e.values())
