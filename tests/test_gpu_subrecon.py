"""Uncertainty from sub-reconstructions (Sec. 5) through ccov_subrecon_covariance
against the oracle's pipeline (same plan, oracle covariance of every
sub-reconstruction, minimum-trace merge): the mixed form at its bar (1e-6,
four measures), the FP64 form at 1e-9; the cover counts exactly."""
import numpy as np
import pytest

from _checks import FP64_TOL, MIXED_TOL, assert_blocks_close
from oracle import subrecon
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_MIXED, MIXED_TOL), (ccov.CCOV_PREC_FP64, FP64_TOL)])
def test_subrecon_pipeline_against_the_oracle(prec, tol):
    sc = synth.local_scene(n=40, m=4000, seed=21)
    orders = synth.decomposition_orders(sc.n, 2, seed=5)
    want, want_cover, subs = subrecon.camera_covariance(sc, 10, orders)
    got, cover, nsub = ccov.subrecon_covariances(sc, 10, orders, precision=prec)
    assert nsub == len(subs)
    assert np.array_equal(cover, want_cover)
    assert_blocks_close(got, want, tol)


def test_whole_scene_neighbourhood_equals_the_single_scene_path():
    sc = synth.local_scene(n=20, m=2000, seed=22)
    got, cover, nsub = ccov.subrecon_covariances(sc, sc.n, synth.decomposition_orders(sc.n, 1),
                                                 precision=ccov.CCOV_PREC_MIXED)
    assert nsub == 1 and (cover == 1).all()
    assert np.array_equal(got, ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED))
