"""The comparison algorithms of Table 2 through the C ABI (ccov_options.gauge)
against their oracle: Alg. 4 (Moore-Penrose inverse of the reduced camera
matrix) and Alg. 5 (three points fixed), FP64 at 1e-9 and the mixed form at
1e-6 (four measures per block), on scenes of 20-100 cameras.  The mixed form
runs these with six digits by default: their Jacobi-scaled matrices have
condition numbers near 2e6 (2e4 for the method's), at which five 8-bit digits
leave errors of about 2e-6 in the scaled measure."""
import numpy as np
import pytest

from _checks import FP64_TOL, MIXED_TOL, assert_blocks_close
from oracle import alternatives, covariance, metrics
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu

CASES = [("ring20", None), ("shell60", (60, 4000, 9)), ("shell100", (100, 10000, 5))]


def _scene(name, spec):
    return synth.workload("ring20") if spec is None else synth.shell_scene(n=spec[0], m=spec[1], seed=spec[2])


@pytest.mark.parametrize("name,spec", CASES)
@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, MIXED_TOL)])
def test_alg4_zpinv(name, spec, prec, tol):
    sc = _scene(name, spec)
    got = ccov.camera_covariances(sc, precision=prec, gauge=ccov.CCOV_GAUGE_ZPINV)
    assert_blocks_close(got, alternatives.zpinv_covariance(sc), tol)


@pytest.mark.parametrize("name,spec", CASES)
@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, MIXED_TOL)])
def test_alg5_three_fixed_points(name, spec, prec, tol):
    sc = _scene(name, spec)
    got = ccov.camera_covariances(sc, precision=prec, gauge=ccov.CCOV_GAUGE_FIXED3)
    assert_blocks_close(got, alternatives.fixed_points_covariance(sc), tol)


def test_alg5_with_given_points():
    sc = synth.workload("ring20")
    pts = (7, 100, 333)
    got = ccov.camera_covariances(sc, gauge=ccov.CCOV_GAUGE_FIXED3, fixed_points=pts)
    assert_blocks_close(got, alternatives.fixed_points_covariance(sc, list(pts)), FP64_TOL)


def test_accuracy_ordering_on_a_scene():
    """Against the natural covariance of the oracle, the method is exact to
    rounding while Alg. 4 and 5 differ on the gauge-dependent entries."""
    sc = synth.shell_scene(n=60, m=4000, seed=9)
    nat = covariance.camera_covariance(sc)
    e = {g: metrics.paper_err(ccov.camera_covariances(sc, gauge=g), nat, sc.cams).mean()
         for g in (ccov.CCOV_GAUGE_NATURAL, ccov.CCOV_GAUGE_ZPINV, ccov.CCOV_GAUGE_FIXED3)}
    assert e[ccov.CCOV_GAUGE_NATURAL] < 1e-3 * min(e[ccov.CCOV_GAUGE_ZPINV], e[ccov.CCOV_GAUGE_FIXED3])
