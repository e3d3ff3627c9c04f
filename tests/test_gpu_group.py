"""The batched form as grouped launches (Sec. 5, sub-reconstructions): every
step of every scene in one launch per step.

Every sum of the grouped form runs in the same order as in a scene's own
launches (the same pair lists, the same W7 partial sums per scene, the same
sub-panel groups, integer tensor-core products that commute exactly), so the
grouped batch must
equal the per-scene batch and the single-scene path bit for bit; against the
oracle it is held to the mixed form's bar (four measures, 1e-6)."""
import numpy as np
import pytest

from _checks import MIXED_TOL, assert_blocks_close
from oracle import covariance
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu


def _scenes(k, seed, n_hi=80):
    # up to 80 cameras: N up to 720, six 128-column blocks, three sub-panel pairs
    return synth.batch_scenes(k=k, n_lo=10, n_hi=n_hi, pts_per_cam=60, seed=seed)


def test_grouped_equals_per_scene_and_single_scene_bit_for_bit():
    torch = pytest.importorskip("torch")
    scenes = _scenes(7, 41)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    og = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    op = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with ccov.Batch(ctxs, og, form=ccov.CCOV_BATCH_GROUPED) as bg, \
                ccov.Batch(ctxs, op, form=ccov.CCOV_BATCH_PER_SCENE) as bp:
            info = bg.info()
            assert info["form"] == ccov.CCOV_BATCH_GROUPED
            assert bp.info()["form"] == ccov.CCOV_BATCH_PER_SCENE
            assert info["launches"] < bp.info()["launches"]
            for _ in range(2):
                for o in og:
                    o.zero_()
                torch.cuda.synchronize()
                bg.run()
                bp.run()
                for a, b in zip(og, op):
                    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    finally:
        for c in ctxs:
            c.close()
    for sc, a in zip(scenes, og):
        assert np.array_equal(a.cpu().numpy(), ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED))
    for i in (0, int(np.argmax([sc.n for sc in scenes]))):
        assert_blocks_close(og[i].cpu().numpy(), covariance.camera_covariance(scenes[i]), MIXED_TOL)


def test_grouped_with_groups_of_four_and_pairs_equals_single_scene_bit_for_bit():
    """A 950-camera scene (72 sub-panels: groups of four, K = 512 trailing
    updates) in one grouped batch with small scenes (pairs, K = 256): every
    scene's blocks are those of its own single-scene step, bit for bit."""
    torch = pytest.importorskip("torch")
    scenes = [synth.shell_scene(n=950, m=95_000, seed=44)] + _scenes(3, 45, n_hi=120)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with ccov.Batch(ctxs, outs, form=ccov.CCOV_BATCH_GROUPED) as b:
            assert b.info()["form"] == ccov.CCOV_BATCH_GROUPED
            b.run()
    finally:
        for c in ctxs:
            c.close()
    for sc, o in zip(scenes, outs):
        assert np.array_equal(o.cpu().numpy(), ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED))


def test_grouped_replay_reads_reloaded_inputs():
    torch = pytest.importorskip("torch")
    scenes = _scenes(4, 42, n_hi=40)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with ccov.Batch(ctxs, outs, form=ccov.CCOV_BATCH_GROUPED) as b:
            moved = []
            for ctx, sc in zip(ctxs, scenes):
                cams = sc.cams.copy()
                cams[:, 3:6] *= 1.02
                pts = sc.pts * 1.02
                ctx.ccov_load(cams, pts, sc.obs_records())
                moved.append(synth.Scene(cams=cams, pts=pts, obs_cam=sc.obs_cam, obs_pt=sc.obs_pt,
                                         obs_u=sc.obs_u, sigma=sc.sigma))
            b.run()
            got = [o.cpu().numpy() for o in outs]
    finally:
        for c in ctxs:
            c.close()
    for mv, g in zip(moved, got):
        assert np.array_equal(g, ccov.camera_covariances(mv, precision=ccov.CCOV_PREC_MIXED))


def test_form_selection():
    torch = pytest.importorskip("torch")
    scenes = _scenes(3, 43, n_hi=30)
    ctxs = [ccov.from_scene(scenes[0], precision=ccov.CCOV_PREC_MIXED),
            ccov.from_scene(scenes[1]),                                   # FP64: not groupable
            ccov.from_scene(scenes[2], precision=ccov.CCOV_PREC_MIXED)]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with pytest.raises(ccov.CcovError) as e:
            ccov.Batch(ctxs, outs, form=ccov.CCOV_BATCH_GROUPED)
        assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
        with ccov.Batch(ctxs, outs) as b:
            assert b.info()["form"] == ccov.CCOV_BATCH_PER_SCENE
            b.run()
            assert np.array_equal(outs[1].cpu().numpy(), ccov.camera_covariances(scenes[1]))
    finally:
        for c in ctxs:
            c.close()
