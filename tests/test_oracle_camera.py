"""Pins of the oracle's projection and Jacobian (Sec. 4.1 projection model)."""
import numpy as np
import pytest
import scipy.linalg as sla

pytest.importorskip("mpmath")
from oracle import brute, camera, nullspace  # noqa: E402


def test_projection_closed_form_identity_rotation():
    # r = 0, t = (0, 0, d): u = f (1 + k1 rho^2 + k2 rho^4) (X + t)_xy / (X + t)_z
    cams = np.array([[0, 0, 0, 0.1, -0.2, 9.0, 1000.0, 0.01, -0.003]])
    X = np.array([[0.3, -0.4, 0.5]])
    Xc = X[0] + cams[0, 3:6]
    x = Xc[:2] / Xc[2]
    rho2 = x @ x
    want = 1000.0 * (1 + 0.01 * rho2 - 0.003 * rho2 ** 2) * x
    got = camera.project_values(cams, X)[0]
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)


@pytest.mark.parametrize("theta", [0.0, 1e-9, 1e-5, 0.3, 2.0, np.pi - 0.05])
def test_rotation_matches_matrix_exponential(theta):
    rng = np.random.default_rng(7)
    axis = rng.normal(size=3)
    r = theta * axis / np.linalg.norm(axis)
    R = camera.rotation_matrix(r)
    want = sla.expm(nullspace.skew(r))
    np.testing.assert_allclose(R, want, rtol=0, atol=2e-15)


def _random_obs(rng, theta):
    axis = rng.normal(size=3)
    r = theta * axis / np.linalg.norm(axis)
    cam = np.concatenate([r, rng.normal(size=2) * 0.3, [8.0 + rng.random()],
                          [rng.uniform(900, 1100)], rng.normal(size=2) * 0.01])
    X = rng.uniform(-0.5, 0.5, size=3)
    return cam, X


@pytest.mark.parametrize("theta", [1e-9, 1e-6, 0.7, 3.0])
def test_jacobian_matches_complex_step_of_expm_projection(theta):
    rng = np.random.default_rng(11)
    for _ in range(3):
        cam, X = _random_obs(rng, theta)
        Jc, Jp = camera.jacobians(cam[None], X[None], np.array([0]), np.array([0]))
        got = np.concatenate([Jc[0], Jp[0]], axis=1)
        want = brute.to_numpy(brute.jacobian_complex_step(cam, X))
        scale = np.abs(want).max(axis=1, keepdims=True)
        assert np.abs(got - want).max() / scale.max() < 1e-13


def test_jacobian_pin_catches_dropped_k2_term(monkeypatch):
    """Plant a mistake in the oracle (drop the k2 rho^4 term): the pin fails."""
    orig = camera.project

    def broken(cam, X):
        cam = list(cam)
        cam[8] = cam[8] * 0.0
        return orig(cam, X)

    monkeypatch.setattr(camera, "project", broken)
    rng = np.random.default_rng(3)
    cam, X = _random_obs(rng, 0.5)
    Jc, Jp = camera.jacobians(cam[None], X[None], np.array([0]), np.array([0]))
    want = brute.to_numpy(brute.jacobian_complex_step(cam, X))
    got = np.concatenate([Jc[0], Jp[0]], axis=1)
    assert np.abs(got - want).max() > 1e-6 * np.abs(want).max()
