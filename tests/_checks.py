"""Block comparison used by every GPU covariance test.

Each 9x9 block is compared by four measures (oracle.metrics): the relative
Frobenius error of the whole block, the same after the scaling
D = diag(R)^-1/2, and the relative Frobenius errors of the 6x6 pose and the
3x3 intrinsic sub-blocks.  The whole-block measure alone is dominated by the
k2 variance and cannot see the pose entries, which are about 1e-7 of a
block's norm.  One tolerance bounds all four:
- FP64 path: 1e-9.  FP64 rounding amplified by the condition number of the
  Jacobi-scaled matrix (about 2e4 on these scenes) gives errors near 1e-12
  in every measure.
- mixed path: 1e-6.  Its operands carry 39-bit digits; a relative
  perturbation of 2^-39 of the scaled matrix gives at most 2e-8 in the
  scaled and the pose measures on 20-300-camera scenes (numpy emulation),
  so 1e-6 leaves a factor of 50.
"""
import numpy as np

from oracle import metrics

FP64_TOL = 1e-9
MIXED_TOL = 1e-6


def block_errors(got, want):
    return {k: float(v.max()) for k, v in metrics.all_errors(np.asarray(got), np.asarray(want)).items()}


def assert_blocks_close(got, want, tol, what=""):
    errs = block_errors(got, want)
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, f"{what}: {bad} not below {tol:.0e} (all: {errs})"
    return errs
