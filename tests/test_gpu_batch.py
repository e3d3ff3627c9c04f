"""Batched form (Sec. 5, sub-reconstructions): many independent scenes in one
call and in one replayed CUDA graph, checked against the single-scene path and
the oracle.  Same tolerances as the single-scene tests: 1e-9 relative
Frobenius per block for FP64 against the oracle, 1e-6 for the mixed path;
batch against single-scene results bit for bit (every sum of the path runs
in a fixed order)."""
import numpy as np
import pytest

from _checks import assert_blocks_close
from oracle import camera, covariance, metrics
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu


def _scenes(k=5, seed=21):
    # sub-reconstructions of the sizes the batched workload draws, scaled down
    return synth.batch_scenes(k=k, n_lo=10, n_hi=45, pts_per_cam=60, seed=seed)


def test_batch_matches_single_scene_and_oracle():
    scenes = _scenes()
    ctxs = [ccov.from_scene(sc) for sc in scenes]
    try:
        got = ccov.ccov_batch_covariance(ctxs)
        again = ccov.ccov_batch_covariance(ctxs)          # contexts are reusable
    finally:
        for c in ctxs:
            c.close()
    for sc, g, a in zip(scenes, got, again):
        single = ccov.camera_covariances(sc)
        assert np.array_equal(g, single)
        assert np.array_equal(a, single)
        assert_blocks_close(g, covariance.camera_covariance(sc), 1e-9)


def test_batch_graph_replay_and_reload():
    torch = pytest.importorskip("torch")
    scenes = _scenes(k=4, seed=22)
    ctxs = [ccov.from_scene(sc) for sc in scenes]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with ccov.Batch(ctxs, outs) as b:
            for o in outs:
                o.zero_()
            torch.cuda.synchronize()
            b.run()
            first = [o.cpu().numpy() for o in outs]
            b.run()
            second = [o.cpu().numpy() for o in outs]
            # new inputs, same index set: the next replay picks them up
            moved = []
            for ctx, sc in zip(ctxs, scenes):
                cams = sc.cams.copy()
                cams[:, 3:6] *= 1.01
                pts = sc.pts * 1.01
                ctx.ccov_load(cams, pts, sc.obs_records())
                moved.append(synth.Scene(cams=cams, pts=pts, obs_cam=sc.obs_cam, obs_pt=sc.obs_pt,
                                         obs_u=sc.obs_u, sigma=sc.sigma, obs_cov=sc.obs_cov))
            b.run()
            third = [o.cpu().numpy() for o in outs]
    finally:
        for c in ctxs:
            c.close()
    for sc, mv, f, s, t in zip(scenes, moved, first, second, third):
        want = covariance.camera_covariance(sc)
        assert_blocks_close(f, want, 1e-9)
        assert np.array_equal(s, f)
        assert_blocks_close(t, covariance.camera_covariance(mv), 1e-9)
        assert metrics.rel_fro(t, f).max() > 1e-6               # the reload took effect


def test_batch_mixed_precision():
    scenes = _scenes(k=3, seed=23)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    try:
        got = ccov.ccov_batch_covariance(ctxs)
    finally:
        for c in ctxs:
            c.close()
    for sc, g in zip(scenes, got):
        assert_blocks_close(g, covariance.camera_covariance(sc), 1e-6)


def test_batch_reports_a_degenerate_member():
    scenes = _scenes(k=3, seed=24)
    bad = scenes[1]
    pts = bad.pts.copy()
    i = bad.obs_cam[0]
    center = -camera.rotation_matrix(bad.cams[i, :3]).T @ bad.cams[i, 3:6]
    pts[bad.obs_pt[0]] = 2.0 * center                 # behind the camera that observes it
    ctxs = [ccov.from_scene(sc) for sc in scenes]
    try:
        ctxs[1].ccov_load(bad.cams, pts, bad.obs_records())
        with pytest.raises(ccov.CcovError) as e:
            ccov.ccov_batch_covariance(ctxs)
        assert e.value.status == ccov.CCOV_ERR_DEGENERATE
        # the healthy members still compute
        ok = ccov.ccov_batch_covariance([ctxs[0], ctxs[2]])
    finally:
        for c in ctxs:
            c.close()
    assert_blocks_close(ok[0], covariance.camera_covariance(scenes[0]), 1e-9)
    assert_blocks_close(ok[1], covariance.camera_covariance(scenes[2]), 1e-9)


def test_mixed_batch_graph_replays_match_direct_calls():
    torch = pytest.importorskip("torch")
    scenes = _scenes(k=3, seed=25)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        direct = ccov.ccov_batch_covariance(ctxs)
        with ccov.Batch(ctxs, outs) as b:
            for _ in range(3):
                for o in outs:
                    o.zero_()
                torch.cuda.synchronize()
                b.run()
                for o, d in zip(outs, direct):
                    assert np.array_equal(o.cpu().numpy(), d)
    finally:
        for c in ctxs:
            c.close()
