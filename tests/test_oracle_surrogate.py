"""Pins of the surrogate oracle against things other than itself: torch's
bf16 conversion, torch autograd and torch.optim.Adam in float64, central
finite differences, the dense Schur complement of the covariance oracle,
brute-force counting, closed forms and round trips."""
import numpy as np
import pytest

from oracle import covariance, surrogate as S
from paper_1808_02414_gb300 import synth


def _params(seed=0, scale=1.0):
    p = S.unpack(synth.surrogate_init(seed).astype(np.float64))
    rng = np.random.default_rng(seed + 100)
    # non-zero biases so that their gradients are exercised
    return [a if a.ndim == 2 else scale * rng.normal(0, 0.1, a.shape) for a in p]


def _batch(B=7, seed=1):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, S.F_IN)), rng.normal(size=(B, S.F_OUT))


def test_shapes_and_packing():
    assert S.n_params() == 64 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 45 + 45
    flat = synth.surrogate_init(3)
    assert flat.shape == (S.n_params(),)
    np.testing.assert_array_equal(S.pack(S.unpack(flat)), flat.astype(np.float64))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3e38, -7e-39]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16(x), want)


def test_exact_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    p = _params()
    x, t = _batch()
    loss, g = S.loss_and_grads(p, x, t, quantize=False)
    tp = [torch.tensor(a, requires_grad=True) for a in p]
    h = torch.tensor(x)
    for layer in range(4):
        h = h @ tp[2 * layer].T + tp[2 * layer + 1]
        if layer < 3:
            h = torch.relu(h)
    tl = ((h - torch.tensor(t)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12 * abs(loss)
    for a, b in zip(g, tp):
        np.testing.assert_allclose(a, b.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_exact_gradients_match_finite_differences():
    p = _params(seed=2)
    x, t = _batch(B=5, seed=3)
    _, g = S.loss_and_grads(p, x, t, quantize=False)
    rng = np.random.default_rng(4)
    h = 1e-6
    for k in range(8):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            pp = [a.copy() for a in p]
            pp[k][idx] += h
            lp, _ = S.loss_and_grads(pp, x, t, quantize=False)
            pp[k][idx] -= 2 * h
            lm, _ = S.loss_and_grads(pp, x, t, quantize=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1e-3, abs(fd)), (k, idx, fd, g[k][idx])


def test_planted_mistake_in_backward_is_caught():
    """A backward that forgets the ReLU mask disagrees with finite differences."""
    p = _params(seed=5)
    x, t = _batch(B=4, seed=6)
    _, g = S.loss_and_grads(p, x, t, quantize=False)
    y, acts = S.forward(p, x, quantize=False)
    gout = 2.0 * (y - t) / (4 * S.F_OUT)
    wrong = (gout @ p[6]).T @ acts[2]              # no mask on layer 3
    assert np.abs(wrong - g[4]).max() > 1e-6 * np.abs(g[4]).max()


def test_quantized_forward_is_within_bf16_error_of_exact():
    p = _params(seed=7)
    x, _ = _batch(B=64, seed=8)
    yq, acts = S.forward(p, x, quantize=True)
    ye, _ = S.forward(p, x, quantize=False)
    rel = np.abs(yq - ye).max() / np.abs(ye).max()
    assert 1e-4 < rel < 5e-2          # rounded, but only at bf16 precision
    for a in acts:
        np.testing.assert_array_equal(S.bf16(a), a)   # activations are bf16 values


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    p = [rng.normal(size=(3, 4)), rng.normal(size=5)]
    m = [np.zeros_like(a) for a in p]
    v = [np.zeros_like(a) for a in p]
    tp = [torch.tensor(a, requires_grad=True) for a in p]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(S.BETA1, S.BETA2), eps=S.EPS)
    for step in range(1, 4):
        g = [rng.normal(size=a.shape) for a in p]
        p, m, v = S.adam(p, g, m, v, step, 1e-2)
        for a, b in zip(tp, g):
            a.grad = torch.tensor(b)
        opt.step()
        for a, b in zip(p, tp):
            np.testing.assert_allclose(a, b.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_diagonal_blocks_match_dense_schur_complement():
    sc = synth.shell_scene(n=12, m=300, seed=3)
    Zd = S.diagonal_blocks(sc)
    Z, _, _ = covariance.schur_blocks_unscaled(sc)
    for i in range(sc.n):
        blk = Z[9 * i:9 * i + 9, 9 * i:9 * i + 9]
        np.testing.assert_allclose(Zd[i], blk, rtol=0, atol=1e-10 * np.abs(blk).max())


def test_degree_stats_by_counting():
    sc = synth.shell_scene(n=10, m=200, seed=4)
    track = {}
    for j in sc.obs_pt:
        track[int(j)] = track.get(int(j), 0) + 1
    got = S.degree_stats(sc)
    for i in range(sc.n):
        lens = [track[int(j)] for c, j in zip(sc.obs_cam, sc.obs_pt) if c == i]
        assert got[i, 0] == pytest.approx(np.log(len(lens)), rel=1e-14)
        assert got[i, 1] == pytest.approx(sum(np.log(v) for v in lens) / len(lens), rel=1e-14)
        assert got[i, 2] == pytest.approx(sum(v == 2 for v in lens) / len(lens), rel=1e-14)


def test_centre_distance_on_a_ring_is_one():
    sc = synth.workload("ring20")   # centres on a circle about the origin
    np.testing.assert_allclose(S.centre_distance(sc), 1.0, rtol=1e-12)


def test_features_layout():
    sc = synth.shell_scene(n=8, m=150, seed=5)
    f, Lz = S.features(sc)
    Z = S.diagonal_blocks(sc)
    d = np.sqrt(np.einsum("ikk->ik", Z))
    assert f.shape == (8, 64) and Lz.shape == (8, 9, 9)
    np.testing.assert_allclose(Lz @ Lz.transpose(0, 2, 1), Z, rtol=1e-12, atol=1e-12 * np.abs(Z).max())
    assert np.all(np.triu(Lz[2], 1) == 0) and np.all(np.einsum("ikk->ik", Lz) > 0)
    assert f[3, 0] == pytest.approx(Z[3, 0, 1] / (d[3, 0] * d[3, 1]), rel=1e-14)   # C_01
    assert f[3, 35] == pytest.approx(Z[3, 7, 8] / (d[3, 7] * d[3, 8]), rel=1e-14)  # C_78
    np.testing.assert_allclose(f[:, 36:45], np.log(d), rtol=1e-14)
    np.testing.assert_allclose(f[:, 48], 10.0 / np.sqrt(8.0), rtol=1e-15)
    assert np.all(f[:, 50:] == 0)
    assert np.all(np.abs(f[:, :36]) < 1)   # off-diagonal correlations of an SPD block


def test_targets_round_trip_and_closed_form():
    sc = synth.shell_scene(n=10, m=300, seed=6)
    sig = covariance.camera_covariance(sc)
    _, Lz = S.features(sc)
    t = S.targets(sig, Lz)
    np.testing.assert_allclose(S.covariance_from_output(t, Lz), sig, rtol=1e-10,
                               atol=1e-12 * np.abs(sig).max())
    # the covariance with every other camera fixed, Z_ii^-1, whitens to I
    local = np.linalg.inv(S.diagonal_blocks(sc))
    np.testing.assert_allclose(S.targets(local, Lz), 0.0, atol=1e-9)
    # a whitened block 4 I: log L_kk = log 2, no off-diagonal part
    Li = np.linalg.inv(Lz)
    four = 4.0 * Li.transpose(0, 2, 1) @ Li
    tt = S.targets(four, Lz)
    np.testing.assert_allclose(tt[:, :9], np.log(2.0), atol=1e-9)
    np.testing.assert_allclose(tt[:, 9:], 0.0, atol=1e-9)


def test_gaussian_kl_closed_form():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(4, 9, 9))
    Q = A @ A.transpose(0, 2, 1) + 9 * np.eye(9)
    np.testing.assert_allclose(S.gaussian_kl(Q, Q), 0.0, atol=1e-12)
    # pred = c true: KL = 9/2 (1/c - 1 + log c)
    c = 2.5
    np.testing.assert_allclose(S.gaussian_kl(c * Q, Q), 4.5 * (1 / c - 1 + np.log(c)), rtol=1e-12)


def test_normalization():
    rng = np.random.default_rng(0)
    x = rng.normal(3.0, 2.0, size=(500, 4))
    x[:, 2] = 5.0
    mu, sd = S.normalization(x)
    z = (x - mu) / sd
    np.testing.assert_allclose(z.mean(axis=0), 0, atol=1e-12)
    np.testing.assert_allclose(z[:, [0, 1, 3]].std(axis=0), 1, rtol=1e-12)
    assert sd[2] == 1.0 and np.all(z[:, 2] == 0)


# ---------------------------------------------------------------------------
# Gauge term of the base covariance
def _gauge_inputs(n=14, m=600, seed=21):
    from oracle import nullspace
    sc = synth.shell_scene(n=n, m=m, seed=seed)
    _, Lz = S.features(sc)
    H = nullspace.camera_rows_closed_form(sc).reshape(n, 9, 7)
    return sc, Lz, H


def _spd(k, seed):
    A = np.random.default_rng(seed).normal(size=(k, k))
    return A @ A.T + k * np.eye(k)


def test_gauge_rows_are_normalised_and_span_the_nullspace_rows():
    sc, Lz, H = _gauge_inputs()
    Q = S.gauge_rows(Lz, H)
    Z = S.diagonal_blocks(sc)                 # from the information blocks, not from Lz
    np.testing.assert_allclose(np.einsum("iak,iab,ibl->kl", Q, Z, Q), np.eye(7), atol=1e-10)
    # Q_i = H_i C for one 7 x 7 C shared by every camera
    C = np.linalg.lstsq(H.reshape(-1, 7), Q.reshape(-1, 7), rcond=None)[0]
    np.testing.assert_allclose(H @ C, Q, rtol=1e-10, atol=1e-12 * np.abs(Q).max())


def test_base_factor_against_the_push_through_form():
    sc, Lz, H = _gauge_inputs()
    Q = S.gauge_rows(Lz, H)
    np.testing.assert_allclose(S.base_factor(Lz, Q, np.zeros((7, 7))), Lz, rtol=1e-9,
                               atol=1e-12 * np.abs(Lz).max())
    M = 0.05 * _spd(7, 3)
    T = S.base_factor(Lz, Q, M)
    assert np.all(np.triu(T, 1) == 0) and np.all(np.einsum("ikk->ik", T) > 0)
    # (Z^-1 + Q M Q^T)^-1 = Z - Z Q M (I + Q^T Z Q M)^-1 Q^T Z
    Z = Lz @ Lz.transpose(0, 2, 1)
    ZQ = Z @ Q
    inner = np.linalg.inv(np.eye(7) + Q.transpose(0, 2, 1) @ ZQ @ M)
    want = Z - ZQ @ M @ inner @ ZQ.transpose(0, 2, 1)
    got = T @ T.transpose(0, 2, 1)
    err = np.linalg.norm(got - want, axis=(1, 2)) / np.linalg.norm(want, axis=(1, 2))
    assert err.max() < 1e-9


def test_fit_gauge_recovers_a_planted_matrix():
    parts = []
    for seed, n in ((21, 14), (22, 20)):
        sc, Lz, H = _gauge_inputs(n=n, m=40 * n, seed=seed)
        parts.append((Lz, S.gauge_rows(Lz, H)))
    Mstar = _spd(7, 5) / 7.0
    Lz = np.concatenate([p[0] for p in parts])
    Q = np.concatenate([p[1] for p in parts])
    sig = np.linalg.inv(Lz @ Lz.transpose(0, 2, 1)) + Q @ Mstar @ Q.transpose(0, 2, 1)
    M = S.fit_gauge(Lz, Q, sig)
    np.testing.assert_allclose(M, M.T, atol=0)
    np.testing.assert_allclose(M, Mstar, rtol=1e-8, atol=1e-9 * np.abs(Mstar).max())


def test_fit_gauge_meets_the_least_squares_optimality_condition():
    sc, Lz, H = _gauge_inputs(n=16, m=900, seed=23)
    sig = covariance.camera_covariance(sc)
    Q = S.gauge_rows(Lz, H)
    M = S.fit_gauge(Lz, Q, sig)
    # residual orthogonal to every basis image, by explicit sums per camera
    grad = np.zeros(28)
    for i in range(sc.n):
        Qt = Lz[i].T @ Q[i]
        R = Lz[i].T @ sig[i] @ Lz[i] - np.eye(9) - Qt @ M @ Qt.T
        for p, Eb in enumerate(S.sym_basis()):
            grad[p] += np.sum(R * (Qt @ Eb @ Qt.T))
    scale = np.abs(Lz.transpose(0, 2, 1) @ sig @ Lz).max()
    assert np.abs(grad).max() < 1e-9 * scale * sc.n


def test_gauge_term_explains_the_exact_blocks():
    """The premise of the base: on exact blocks, Sigma_i - Z_ii^-1 lies almost
    entirely in the span of H_i (measured: 4.5-6% of its whitened Frobenius
    norm outside it on 60- and 200-camera shells, so over 99% of the squared
    norm inside), and one M per scene takes the Gaussian KL far below that of
    Z_ii^-1."""
    sc, Lz, H = _gauge_inputs(n=60, m=6000, seed=24)
    sig = covariance.camera_covariance(sc)
    Zinv = np.linalg.inv(Lz @ Lz.transpose(0, 2, 1))
    Ew = Lz.transpose(0, 2, 1) @ (sig - Zinv) @ Lz
    Hw = Lz.transpose(0, 2, 1) @ H
    for i in range(sc.n):
        U, s, _ = np.linalg.svd(Hw[i], full_matrices=False)
        U = U[:, s > 1e-12 * s[0]]
        P = U @ U.T
        assert np.linalg.norm(Ew[i] - P @ Ew[i] @ P) <= 0.1 * np.linalg.norm(Ew[i])
    Q = S.gauge_rows(Lz, H)
    T = S.base_factor(Lz, Q, S.fit_gauge(Lz, Q, sig))
    Ti = np.linalg.inv(T)
    kl_base = S.gaussian_kl(Ti.transpose(0, 2, 1) @ Ti, sig)
    kl_local = S.gaussian_kl(Zinv, sig)
    assert np.median(kl_base) < 0.02 * np.median(kl_local)


def test_predict_head_scale_closed_form():
    """Output weights zero: y = 0, so t = s mu_t.  With mu_t = log 2 on the
    diagonal entries and zero elsewhere, L = 2^s I and Sigma_hat =
    4^s (T T^T)^-1 for each camera's own s (1 where feature 48 is not
    positive)."""
    rng = np.random.default_rng(4)
    n = 6
    p = _params(2)
    p[6] = np.zeros_like(p[6])
    p[7] = np.zeros_like(p[7])
    f = rng.normal(size=(n, 64))
    f[:, 48] = [0.2, 0.7, 1.3, -1.0, 0.0, 2.0]
    A = rng.normal(size=(n, 9, 9))
    T = np.linalg.cholesky(A @ A.transpose(0, 2, 1) + 9 * np.eye(9))
    mu_t = np.concatenate([np.full(9, np.log(2.0)), np.zeros(36)])
    norm = (np.zeros(64), np.ones(64), mu_t, np.ones(45))
    got = S.predict(p, f, T, norm)
    s = np.array([0.2, 0.7, 1.3, 1.0, 1.0, 2.0])
    base = np.linalg.inv(T @ T.transpose(0, 2, 1))
    want = (4.0 ** s)[:, None, None] * base
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
