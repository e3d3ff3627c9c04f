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
