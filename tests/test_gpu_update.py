"""Covariance after added observations (Sec. 5: M_{i+1} = M_i + M_Delta and
the Woodbury identity) through the C ABI, against the oracle's covariance of
the scene with the observations added, computed from scratch.

The update is exact up to rounding, so the bars are those of step (d): FP64
1e-9 and mixed 1e-6 in all four block measures (tests/_checks.py); the centre
camera's FP64 bar is 1e-8 (its scaled matrix has a condition number of about
3e6, see test_gpu_centre.py).  Sizes: 40 observations on four cameras (one S
tile), 600 on a 300-camera scene (r = 1200 columns: ten 128-row blocks of S,
134 groups of nine columns with a ragged last group), anisotropic
per-observation covariances, and the centre camera."""
import numpy as np
import pytest

from _checks import FP64_TOL, MIXED_TOL, assert_blocks_close
from oracle import covariance
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu


def _aniso(sc, seed=5):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 2.0, size=(sc.t, 2))
    th = rng.uniform(0, np.pi, size=sc.t)
    c, s = np.cos(th), np.sin(th)
    Rr = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)
    C = np.einsum("tij,tj,tkj->tik", Rr, a, Rr)
    sc.obs_cov = 0.5 * (C + C.transpose(0, 2, 1))   # exactly symmetric
    return sc


def _update(sc, added, **kw):
    with ccov.from_scene(sc, **kw) as ctx:
        before = ctx.run()
        acov = None if added.obs_cov is None else added.obs_cov.reshape(-1, 4)
        got = ctx.ccov_update_observations(added.obs_records(), acov)
        stats = ctx.ccov_get_stats()
    return before, got, stats


@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, MIXED_TOL)])
def test_update_small_against_the_oracle(prec, tol):
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    merged, added = synth.added_observations(sc, 40, cams=[0, 1, 2, 3], seed=4)
    before, got, stats = _update(sc, added, precision=prec)
    assert_blocks_close(got, covariance.camera_covariance(merged), tol, "update")
    assert stats["update_launches"] > 0 and stats["ms_update"] > 0
    # the four cameras that got observations tighten
    for c in range(4):
        assert np.trace(got[c][6:9, 6:9]) < np.trace(before[c][6:9, 6:9])


@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, MIXED_TOL)])
def test_update_several_tiles_against_the_oracle(prec, tol):
    sc = synth.shell_scene(n=300, m=30000, seed=6)
    merged, added = synth.added_observations(sc, 600, seed=8)
    _, got, _ = _update(sc, added, precision=prec)
    assert_blocks_close(got, covariance.camera_covariance(merged), tol, "update")


def test_update_many_observations_on_a_small_scene():
    """2k columns wider than the scene's padded N (200 observations on 30
    cameras: 405 columns, Np = 384): the mixed form then takes Y = Z'^-1 V in
    double-single arithmetic and the small products in FP64 instead of the
    tensor-core panels, whose operand buffers hold Np rows."""
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    merged, added = synth.added_observations(sc, 200, seed=5)
    _, got, _ = _update(sc, added, precision=ccov.CCOV_PREC_MIXED)
    assert_blocks_close(got, covariance.camera_covariance(merged), MIXED_TOL, "update")


def test_update_anisotropic_against_the_oracle():
    sc = _aniso(synth.shell_scene(n=60, m=4000, seed=9))
    merged, added = synth.added_observations(sc, 120, seed=3)
    assert added.obs_cov is not None and merged.obs_cov is not None
    _, got, _ = _update(sc, added, precision=ccov.CCOV_PREC_FP64)
    assert_blocks_close(got, covariance.camera_covariance(merged), FP64_TOL, "update")


def test_update_centre_camera_against_the_oracle():
    sc = synth.centre_scene(synth.shell_scene(n=60, m=4000, seed=9))
    merged, added = synth.added_observations(sc, 80, seed=2)
    _, got, _ = _update(sc, added, precision=ccov.CCOV_PREC_FP64)
    want = covariance.camera_covariance(merged)
    g8 = got[:, :8, :8]
    rel = np.linalg.norm(g8 - want, axis=(1, 2)) / np.linalg.norm(want, axis=(1, 2))
    d = 1.0 / np.sqrt(np.einsum("nii->ni", want))
    D = d[:, :, None] * d[:, None, :]
    nrel = np.linalg.norm((g8 - want) * D, axis=(1, 2)) / np.linalg.norm(want * D, axis=(1, 2))
    assert rel.max() < 1e-8 and nrel.max() < 1e-8, (rel.max(), nrel.max())
    np.testing.assert_allclose(got[:, 8, 8], 1.0, rtol=1e-12)


def _with_extra(sc, cams, pts):
    """The scene with extra observations (cam, pt) appended in point order
    (pairs may repeat existing ones: the oracle adds their information)."""
    cam = np.concatenate([sc.obs_cam, np.asarray(cams, np.int32)])
    pt = np.concatenate([sc.obs_pt, np.asarray(pts, np.int32)])
    u = np.concatenate([sc.obs_u, np.zeros((len(cams), 2))])
    order = np.lexsort((cam, pt))
    return synth.Scene(sc.cams, sc.pts, cam[order].astype(np.int32), pt[order].astype(np.int32), u[order],
                       sc.sigma, None, dict(sc.meta))


@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, MIXED_TOL)])
def test_update_one_observation_and_a_repeated_pair(prec, tol):
    """k = 1, and an added observation of a (camera, point) pair that the scene
    already has (a second, independent measurement of the same projection)."""
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    c, j = int(sc.obs_cam[5]), int(sc.obs_pt[5])
    other = int(np.flatnonzero(~np.isin(np.arange(sc.n), sc.obs_cam[sc.obs_pt == 7]))[0])
    for cams, pts in (([other], [7]), ([c], [j])):
        add = np.zeros(len(cams), dtype=synth.OBS_DTYPE)
        add["cam"], add["pt"] = cams, pts
        with ccov.from_scene(sc, precision=prec) as ctx:
            ctx.run()
            got = ctx.ccov_update_observations(add)
        assert_blocks_close(got, covariance.camera_covariance(_with_extra(sc, cams, pts)), tol, "update")


def test_update_keeps_the_context_and_repeats_bit_exactly():
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    _, add_a = synth.added_observations(sc, 40, cams=[0, 1, 2, 3], seed=4)
    _, add_b = synth.added_observations(sc, 25, seed=9)
    with ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED) as ctx:
        before = ctx.run()
        none = ctx.ccov_update_observations(add_a.obs_records()[:0])
        np.testing.assert_array_equal(none, before)
        a1 = ctx.ccov_update_observations(add_a.obs_records())
        b1 = ctx.ccov_update_observations(add_b.obs_records())
        a2 = ctx.ccov_update_observations(add_a.obs_records())
        np.testing.assert_array_equal(a1, a2)
        assert not np.array_equal(a1, b1)
        # and the device-output form gives the same bits
        torch = pytest.importorskip("torch")
        out = torch.empty((sc.n, 9, 9), dtype=torch.float64, device="cuda")
        ctx.ccov_update_observations(add_a.obs_records(), out=out)
        np.testing.assert_array_equal(out.cpu().numpy(), a1)


def test_update_rejects_bad_calls():
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    _, added = synth.added_observations(sc, 10, seed=4)
    rec = added.obs_records()
    with ccov.from_scene(sc) as ctx:
        with pytest.raises(ccov.CcovError) as e:        # before ccov_covariance
            ctx.ccov_update_observations(rec)
        assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
        ctx.run()
        bad = rec.copy()
        bad["cam"][3] = sc.n
        with pytest.raises(ccov.CcovError) as e:
            ctx.ccov_update_observations(bad)
        assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
        bad = rec.copy()
        bad["pt"][0] = -1
        with pytest.raises(ccov.CcovError):
            ctx.ccov_update_observations(bad)
        with pytest.raises(ccov.CcovError):             # covariances the context was not made with
            ctx.ccov_update_observations(rec, np.tile(np.eye(2).ravel(), (10, 1)))
        # still usable
        assert np.isfinite(ctx.ccov_update_observations(rec)).all()
        ctx.ccov_information()                         # a new step (a) ends the state
        with pytest.raises(ccov.CcovError):
            ctx.ccov_update_observations(rec)
    with ccov.from_scene(sc, gauge=ccov.CCOV_GAUGE_ZPINV) as ctx:
        ctx.run()
        with pytest.raises(ccov.CcovError):
            ctx.ccov_update_observations(rec)
