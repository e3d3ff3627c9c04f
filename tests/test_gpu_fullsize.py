"""Parity at the full sizes of the workloads, in the launch configuration
that bench.py times (one context per scene with default options; the batched
form as one replayed graph).

- 1000 cameras, 100 000 points: every camera block of the FP64 path against
  the oracle (1e-9 relative Frobenius) and of the mixed path (1e-6).
- 4000 cameras, 400 000 points (N = 36 000): the oracle cannot invert Z in a
  test, so steps (a)-(c) are checked on outputs the oracle computes one by
  one (block rows of Z for sampled cameras, 1e-11 of max |Z| as for the small
  scenes; the nullspace rows of every camera against their closed form), and
  step (d) of the mixed path against the FP64 GPU path (1e-6) together with
  properties that hold at any size (symmetric, positive semi-definite
  blocks).
- the same scene with 200 observations added by the Woodbury update (mixed)
  against the FP64 GPU path on the merged scene (1e-6).
- 256 sub-reconstructions of 10-300 cameras, mixed, grouped launches replayed
  as one graph: the smallest and the largest scenes against the oracle (1e-6),
  and a few hundred kernels per replay."""
import numpy as np
import pytest

from _checks import assert_blocks_close
from oracle import covariance, metrics, nullspace
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu


def _psd_symmetric(S):
    scale = np.abs(S).max()
    assert np.isfinite(S).all()
    np.testing.assert_allclose(S, np.transpose(S, (0, 2, 1)), rtol=0, atol=1e-12 * scale)
    ev = np.linalg.eigvalsh(0.5 * (S + np.transpose(S, (0, 2, 1))))
    assert ev.min() > -1e-9 * scale


def test_1000_cameras_fp64_and_mixed_against_oracle():
    sc = synth.workload("shell1k")
    want = covariance.camera_covariance(sc)
    fp64 = ccov.camera_covariances(sc)
    mixed = ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED)
    assert_blocks_close(fp64, want, 1e-9)
    assert_blocks_close(mixed, want, 1e-6)


def test_4000_cameras_sampled_steps_and_mixed_against_fp64():
    sc = synth.workload("shell4k")
    picks = [0, 1337, 2500, sc.n - 1]
    rows = covariance.schur_rows_unscaled(sc, picks)
    with ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) as ctx:
        ctx.ccov_information()
        ctx.ccov_schur()
        zmax = 0.0
        for i in picks:
            pairs = [(max(i, j), min(i, j)) for j in range(sc.n)]
            blk = ctx.ccov_get_schur_blocks(pairs)
            # Z_ij; a diagonal block is stored by its lower triangle
            got = np.stack([np.tril(b) + np.tril(b, -1).T if i == j else (b if i > j else b.T)
                            for b, j in zip(blk, range(sc.n))])
            want = rows[i].reshape(9, sc.n, 9).transpose(1, 0, 2)
            zmax = max(zmax, np.abs(want).max())
            assert np.abs(got - want).max() < 1e-11 * max(zmax, np.abs(got).max())
        hp = ctx.ccov_nullspace(want_hp=True)
        closed = nullspace.camera_rows_closed_form(sc)
        assert np.abs(hp - closed).max() < 1e-8 * np.abs(closed).max()
        mixed = ctx.ccov_covariance()
        with pytest.raises(ccov.CcovError):
            ctx.ccov_get_schur_blocks([(0, 0)])          # Z was consumed by step (d)
    fp64 = ccov.camera_covariances(sc)
    _psd_symmetric(mixed)
    _psd_symmetric(fp64)
    assert_blocks_close(mixed, fp64, 1e-6)


def test_4000_cameras_update_against_fp64_of_the_merged_scene():
    """The Woodbury update (Sec. 5) at the bench's size: 200 observations
    added to the mixed factorisation of the 4000-camera scene, against the
    FP64 GPU form of the merged scene computed from scratch (1e-6)."""
    sc = synth.workload("shell4k")
    merged, added = synth.added_observations(sc, 200, cams=np.arange(0, sc.n, sc.n // 10)[:10], seed=21)
    with ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) as ctx:
        ctx.run()
        upd = ctx.ccov_update_observations(added.obs_records())
    want = ccov.camera_covariances(merged)
    _psd_symmetric(upd)
    assert_blocks_close(upd, want, 1e-6)


def test_256_subreconstructions_graph_against_oracle():
    torch = pytest.importorskip("torch")
    scenes = synth.batch_scenes(k=256, n_lo=10, n_hi=300, pts_per_cam=100, p_geom=0.2)
    ctxs = [ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) for sc in scenes]
    outs = [torch.zeros((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        with ccov.Batch(ctxs, outs) as b:
            info = b.info()
            b.run()
            b.run()
            got = [o.cpu().numpy() for o in outs]
        # the grouped form: one launch per step for all 256 scenes
        assert info["form"] == ccov.CCOV_BATCH_GROUPED
        assert info["launches"] < 1000
    finally:
        for c in ctxs:
            c.close()
    for g in got:
        _psd_symmetric(g)
    sizes = [sc.n for sc in scenes]
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        want = covariance.camera_covariance(scenes[k])
        assert_blocks_close(got[k], want, 1e-6)
