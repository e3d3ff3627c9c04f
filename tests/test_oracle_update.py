"""Pins for adding observations (Sec. 5: M_{i+1} = M_i + M_Delta, Woodbury):
the reference of an update is the covariance of the scene with the added
observations, computed from scratch by the oracle.  What the paper states
about it is checked here: the added information subtracts positive
semi-definite terms, so the uncertainty decreases (Loewner order on the
gauge-invariant intrinsic blocks), and nothing changes when nothing is added."""
import numpy as np

from oracle import covariance
from paper_1808_02414_gb300 import synth


def test_added_observations_decrease_the_uncertainty():
    sc = synth.shell_scene(n=30, m=2000, seed=12)
    before = covariance.camera_covariance(sc)
    merged, added = synth.added_observations(sc, 40, cams=[0, 1, 2, 3], seed=4)
    assert merged.t == sc.t + 40 and added.t == 40
    after = covariance.camera_covariance(merged)
    for a, b in zip(before, after):
        d = a[6:9, 6:9] - b[6:9, 6:9]
        assert np.linalg.eigvalsh(0.5 * (d + d.T)).min() > -1e-9 * np.abs(a[6:9, 6:9]).max()
    # the cameras that got observations tighten visibly
    for c in range(4):
        assert np.trace(after[c][6:9, 6:9]) < np.trace(before[c][6:9, 6:9])


def test_added_observations_are_new_and_sorted():
    sc = synth.shell_scene(n=20, m=800, seed=13)
    merged, added = synth.added_observations(sc, 25, seed=5)
    old = set(zip(sc.obs_cam.tolist(), sc.obs_pt.tolist()))
    new = list(zip(added.obs_cam.tolist(), added.obs_pt.tolist()))
    assert len(set(new)) == 25 and not (set(new) & old)
    assert np.all(np.diff(merged.obs_pt) >= 0)
