"""The seeded scene generator: shapes, determinism and track statistics."""
import numpy as np

from paper_1808_02414_gb300 import synth


def test_ring_scene_shape_and_tracks():
    sc = synth.workload("ring20")
    assert (sc.n, sc.m, sc.t) == (20, 500, 2500)
    assert np.all(np.diff(sc.obs_pt) >= 0)
    for j in range(sc.m):
        cams = sc.obs_cam[sc.obs_pt == j]
        assert cams.size == 5 and np.unique(cams).size == 5
    np.testing.assert_allclose(np.linalg.norm(sc.cams[:, 3:6], axis=1), 10.0, rtol=1e-12)


def test_shell_scene_statistics_and_determinism():
    a = synth.shell_scene(n=200, m=20000, seed=3)
    b = synth.shell_scene(n=200, m=20000, seed=3)
    assert np.array_equal(a.obs_cam, b.obs_cam) and np.array_equal(a.cams, b.cams)
    lengths = np.bincount(a.obs_pt, minlength=a.m)
    assert lengths.min() >= 2
    assert abs(lengths.mean() - 8.0) < 0.2
    assert np.bincount(a.obs_cam, minlength=a.n).min() >= 5
    theta = np.linalg.norm(a.cams[:, :3], axis=1)
    assert theta.max() < np.pi - 0.1 + 1e-9
    rec = a.obs_records()
    assert rec.dtype.itemsize == 24


def test_subscene_keeps_tracks_of_at_least_two():
    sc = synth.shell_scene(n=60, m=3000, seed=4)
    sub = synth.subscene(sc, np.arange(0, 60, 2))
    assert sub.n == 30
    assert np.bincount(sub.obs_pt).min() >= 2
