"""Learned surrogate on the GPU against the surrogate oracle, through the C ABI.

Tolerances.  Features and targets are fp32 values of fp64 computations:
1e-6 absolute/relative.  The network multiplies bf16 operands (rounded at the
same points as the oracle's `quantize` mode) with fp32 accumulation; the
oracle accumulates in fp64.  A numpy model of exactly that difference (fp32
against fp64 sums, same rounding points) gives gradient errors up to 1.3e-4
(relative Frobenius per tensor) and output errors up to 8e-4 (an occasional
bf16 rounding that flips between the two); the tests allow 2e-3 and 1e-2.
Adam runs in fp32 against the oracle's fp64: 1e-5 relative."""
import numpy as np
import pytest

from oracle import covariance, metrics, surrogate as S
from paper_1808_02414_gb300 import ccov, surrogate, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scene_data(sc):
    """GPU features, L_z and exact FP64 covariance blocks of one scene."""
    with ccov.from_scene(sc) as ctx:
        ctx.ccov_information()
        ctx.ccov_schur()
        f, lz = surrogate.features(ctx)
        ctx.ccov_nullspace()
        sig = torch.empty((sc.n, 9, 9), dtype=torch.float64, device="cuda")
        ctx.ccov_covariance(out=sig)
    return f, lz, sig


def _params(seed):
    p = synth.surrogate_init(seed)
    rng = np.random.default_rng(seed + 7)
    q = S.unpack(p.astype(np.float64))
    q = [a if a.ndim == 2 else rng.normal(0, 0.1, a.shape) for a in q]
    return S.pack(q).astype(np.float32)


def _random_norm(rng):
    return np.concatenate([rng.normal(0, 0.3, 64), rng.uniform(0.5, 2.0, 64),
                           rng.normal(0, 0.3, 45), rng.uniform(0.5, 2.0, 45)]).astype(np.float32)


def test_features_and_targets_match_oracle():
    sc = synth.shell_scene(n=40, m=2000, seed=31)
    f, lz, sig = _scene_data(sc)
    fo, lzo = S.features(sc)
    np.testing.assert_allclose(lz.cpu().numpy(), lzo, rtol=1e-9, atol=1e-9 * np.abs(lzo).max())
    np.testing.assert_allclose(f.cpu().numpy(), fo, rtol=1e-6, atol=1e-6)
    t = surrogate.targets(lz, sig)
    to = S.targets(covariance.camera_covariance(sc), lzo)
    np.testing.assert_allclose(t.cpu().numpy(), to, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("B", [1, 300, 1024])
def test_loss_and_gradients_match_oracle(B):
    rng = np.random.default_rng(B)
    n = 1500
    F = rng.normal(size=(n, 64)).astype(np.float32)
    F[:, 50:] = 0
    T = rng.normal(size=(n, 45)).astype(np.float32)
    params = _params(3)
    norm = _random_norm(rng)
    idx = rng.choice(n, size=B, replace=False).astype(np.int32)
    with surrogate.Surrogate(params, max_batch=1024) as sm:
        sm.set_normalization(norm)
        loss = sm.backward(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(idx).cuda())
        g = sm.grads()
    mu_f, sd_f, mu_t, sd_t = norm[:64], norm[64:128], norm[128:173], norm[173:]
    x = (F[idx].astype(np.float64) - mu_f) / sd_f
    t = (T[idx].astype(np.float64) - mu_t) / sd_t
    lo, go = S.loss_and_grads(S.unpack(params.astype(np.float64)), x, t, quantize=True)
    assert abs(loss - lo) <= 1e-4 * lo
    for a, b in zip(S.unpack(g.astype(np.float64)), go):
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b)


def test_adam_steps_match_oracle():
    rng = np.random.default_rng(5)
    n, B, lr = 800, 256, 1e-3
    F = rng.normal(size=(n, 64)).astype(np.float32)
    T = rng.normal(size=(n, 45)).astype(np.float32)
    params = _params(4)
    dF, dT = torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda()
    with surrogate.Surrogate(params, max_batch=B) as sm:
        p = S.unpack(params.astype(np.float64))
        m = [np.zeros_like(a) for a in p]
        v = [np.zeros_like(a) for a in p]
        for step in (1, 2):
            idx = torch.from_numpy(rng.choice(n, B, replace=False).astype(np.int32)).cuda()
            sm.backward(dF, dT, idx)
            g = S.unpack(sm.grads().astype(np.float64))
            p, m, v = S.adam(p, g, m, v, step, lr)
            sm.adam(lr)
            got = S.unpack(sm.params().astype(np.float64))
            for a, b in zip(got, p):
                np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-3 * lr)


def test_graph_training_equals_step_by_step():
    rng = np.random.default_rng(6)
    n, B, steps, lr = 700, 200, 4, 2e-3
    F = torch.from_numpy(rng.normal(size=(n, 64)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(n, 45)).astype(np.float32)).cuda()
    idx = torch.from_numpy(synth.minibatch_indices(n, B, steps, seed=3)).cuda()
    params = _params(5)
    with surrogate.Surrogate(params, max_batch=B) as a, surrogate.Surrogate(params, max_batch=B) as b:
        losses = a.train(F, T, idx, lr)
        ref = []
        for k in range(steps):
            ref.append(b.backward(F, T, idx[k].contiguous()))
            b.adam(lr)
        np.testing.assert_allclose(losses, ref, rtol=1e-4)
        np.testing.assert_allclose(a.params(), b.params(), rtol=1e-4, atol=1e-6)


def test_features_and_training_repeat_bit_for_bit():
    """Every sum of the features and of a training step runs in a fixed order
    (partial sums reduced in order, no atomics), so the same inputs give the
    same bits: features twice, and two trainings from the same start."""
    sc = synth.shell_scene(n=60, m=3000, seed=21)
    f1, _, _ = _scene_data(sc)
    f2, _, _ = _scene_data(sc)
    assert torch.equal(f1, f2)
    rng = np.random.default_rng(7)
    n, B, steps, lr = 900, 256, 6, 2e-3
    F = torch.from_numpy(rng.normal(size=(n, 64)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(n, 45)).astype(np.float32)).cuda()
    idx = torch.from_numpy(synth.minibatch_indices(n, B, steps, seed=4)).cuda()
    params = _params(8)
    runs = []
    for _ in range(2):
        with surrogate.Surrogate(params, max_batch=B) as sm:
            losses = np.array(sm.train(F, T, idx, lr))
            runs.append((losses, sm.params().copy()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])


def test_prediction_matches_oracle():
    sc = synth.shell_scene(n=50, m=2500, seed=32)
    f, lz, _ = _scene_data(sc)
    rng = np.random.default_rng(8)
    params = _params(6)
    norm = _random_norm(rng)
    with surrogate.Surrogate(params, max_batch=32) as sm:   # several ragged chunks
        sm.set_normalization(norm)
        got = sm.predict(f, lz).cpu().numpy()
    want = S.predict(S.unpack(params.astype(np.float64)), f.cpu().numpy().astype(np.float64),
                     lz.cpu().numpy(), (norm[:64], norm[64:128], norm[128:173], norm[173:]))
    e = metrics.rel_fro(got, want)
    assert np.median(e) < 2e-3 and e.max() < 1e-2


def test_normalization_fit_matches_oracle():
    rng = np.random.default_rng(9)
    F = rng.normal(2.0, 3.0, size=(3000, 64)).astype(np.float32)
    F[:, 60:] = 0.0
    T = rng.normal(-1.0, 0.5, size=(3000, 45)).astype(np.float32)
    with surrogate.Surrogate(synth.surrogate_init(0), max_batch=128) as sm:
        sm.fit_normalization(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda())
        got = sm.normalization()
    mf, sf = S.normalization(F.astype(np.float64))
    mt, st = S.normalization(T.astype(np.float64))
    np.testing.assert_allclose(got, np.concatenate([mf, sf, mt, st]), rtol=1e-5, atol=1e-6)


def test_trained_surrogate_gains_over_the_local_block():
    """Trained on exact blocks of small scenes, the network predicts held-out
    scenes' blocks far better than Z_ii^-1 (the covariance with every other
    camera fixed, which costs the same) and better than a constant learned
    correction, in the unit-free Gaussian KL measure."""
    train = synth.batch_scenes(k=24, n_lo=30, n_hi=120, pts_per_cam=60, seed=41)
    test = synth.batch_scenes(k=4, n_lo=60, n_hi=120, pts_per_cam=60, seed=42)
    F, LZ, TG = [], [], []
    for sc in train:
        f, lz, sig = _scene_data(sc)
        F.append(f)
        TG.append(surrogate.targets(lz, sig))
    F, TG = torch.cat(F), torch.cat(TG)
    idx = torch.from_numpy(synth.minibatch_indices(F.shape[0], 512, 600, seed=1)).cuda()
    with surrogate.Surrogate(synth.surrogate_init(0), max_batch=512) as sm:
        sm.fit_normalization(F, TG)
        losses = sm.train(F, TG, idx, 1e-3)
        assert losses[-50:].mean() < 0.2 * losses[:10].mean()
        kl_sur, kl_loc, kl_mean = [], [], []
        mu_t = sm.normalization()[128:173].astype(np.float64)
        for sc in test:
            f, lz, sig = _scene_data(sc)
            pred = sm.predict(f, lz).cpu().numpy()
            truth, L = sig.cpu().numpy(), lz.cpu().numpy()
            kl_sur.append(S.gaussian_kl(pred, truth))
            kl_loc.append(S.gaussian_kl(S.covariance_from_output(np.zeros((sc.n, 45)), L), truth))
            kl_mean.append(S.gaussian_kl(S.covariance_from_output(np.tile(mu_t, (sc.n, 1)), L), truth))
    kl_sur, kl_loc, kl_mean = (np.median(np.concatenate(k)) for k in (kl_sur, kl_loc, kl_mean))
    assert kl_sur < 0.01 * kl_loc
    assert kl_sur < 0.6 * kl_mean


def test_sample_index_outside_the_training_set_is_rejected():
    F = torch.zeros((100, 64), dtype=torch.float32, device="cuda")
    T = torch.zeros((100, 45), dtype=torch.float32, device="cuda")
    idx = torch.tensor([3, 100, 5], dtype=torch.int32, device="cuda")
    with surrogate.Surrogate(synth.surrogate_init(0), max_batch=8) as sm:
        with pytest.raises(ccov.CcovError) as e:
            sm.backward(F, T, idx)
        assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
        sm.backward(F, T, torch.tensor([0, 99], dtype=torch.int32, device="cuda"))  # usable afterwards
