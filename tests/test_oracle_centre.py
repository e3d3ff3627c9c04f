"""Pins of the oracle for the paper's 8-value centre camera {r, C, c, k}
(Sec. 3, Sec. 4.1): the dual-number Jacobian against the complex-step
derivative of an independent mpmath projection (R = expm([r]_x)); J H = 0 and
M H = 0 with the position rows [I, -[C]_x, C]; the per-camera nullspace solve
against the closed form; the covariance against the bordered inverse at 40
digits built from complex-step Jacobians."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
from oracle import brute, camera, covariance, information, metrics, nullspace  # noqa: E402
from paper_1808_02414_gb300 import synth  # noqa: E402


def _project_mp(cam, X):
    K = mp.matrix([[0, -cam[2], cam[1]], [cam[2], 0, -cam[0]], [-cam[1], cam[0], 0]])
    R = mp.expm(K)
    d = mp.matrix([X[q] - cam[3 + q] for q in range(3)])
    Xc = R * d
    x, y = Xc[0] / Xc[2], Xc[1] / Xc[2]
    g = 1 + cam[7] * (x * x + y * y)
    return [cam[6] * g * x, cam[6] * g * y]


def _jac_complex_step(cam, X, dps=40):
    h = mp.mpf("1e-30")
    with mp.workdps(dps):
        base = [mp.mpf(float(v)) for v in list(cam) + list(X)]
        J = np.zeros((2, 11))
        for k in range(11):
            z = [mp.mpc(v) for v in base]
            z[k] = mp.mpc(base[k], h)
            u = _project_mp(z[:8], z[8:])
            J[0, k] = float(mp.im(u[0]) / h)
            J[1, k] = float(mp.im(u[1]) / h)
    return J


def _scene(n=5, m=30, seed=3):
    return synth.centre_scene(synth.ring_scene(n=n, m=m, track_len=3, seed=seed))


def test_jacobian_against_complex_step():
    sc = _scene()
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt, "centre8")
    assert Jc.shape == (sc.t, 2, 8)
    for o in (0, 7, 19, sc.t - 1):
        want = _jac_complex_step(sc.cams[sc.obs_cam[o]], sc.pts[sc.obs_pt[o]])
        got = np.concatenate([Jc[o], Jp[o]], 1)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def test_nullspace_of_the_centre_model():
    sc = _scene(n=6, m=40, seed=5)
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt, "centre8")
    HP = nullspace.camera_rows(sc, Jc, Jp)
    assert HP.shape == (sc.n, 8, 7)
    np.testing.assert_allclose(HP, nullspace.camera_rows_closed_form(sc), rtol=0, atol=1e-12)
    J = information.dense_jacobian(sc, Jc, Jp)
    H = nullspace.dense_nullspace(sc, HP)
    assert np.abs(J @ H).max() < 1e-12 * np.abs(J).max() * np.abs(H).max()
    M = information.dense_information(sc)
    assert np.abs(M @ H).max() < 1e-12 * np.abs(M).max() * np.abs(H).max()
    assert np.linalg.matrix_rank(J, tol=1e-9 * np.abs(J).max()) == J.shape[1] - 7


def test_covariance_against_the_bordered_inverse_at_40_digits():
    sc = _scene(n=3, m=14, seed=7)
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt, "centre8")
    H = nullspace.dense_nullspace(sc, nullspace.camera_rows(sc, Jc, Jp))
    with mp.workdps(40):
        N = 8 * sc.n + 3 * sc.m
        J = mp.zeros(2 * sc.t, N)
        for o in range(sc.t):
            jj = _jac_complex_step(sc.cams[sc.obs_cam[o]], sc.pts[sc.obs_pt[o]])
            i, j = sc.obs_cam[o], sc.obs_pt[o]
            for a in range(2):
                for b in range(8):
                    J[2 * o + a, 8 * i + b] = jj[a, b] / sc.sigma
                for b in range(3):
                    J[2 * o + a, 8 * sc.n + 3 * j + b] = jj[a, 8 + b] / sc.sigma
        M = J.T * J
        B = brute.bordered_inverse_mp(M, mp.matrix(H.tolist()))
    full = brute.to_numpy(B)[:8 * sc.n, :8 * sc.n]
    want = np.stack([full[8 * i:8 * i + 8, 8 * i:8 * i + 8] for i in range(sc.n)])
    got = covariance.camera_covariance(sc)
    assert got.shape == (sc.n, 8, 8)
    assert metrics.rel_fro(got, want).max() < 1e-8
