"""The allocation-free entry point ccov_spd_inverse_blocks_noalloc.

It serves callers that cannot call cudaMalloc (a real-time loop that must not
allocate; a process whose device memory is owned by another allocator), so all
of its workspace is a fixed static device array.  Checked against the regular
ccov_covariance path on the same scene, on two calls in a row (the second call
reuses the array that the first one left behind)."""
import numpy as np
import pytest

from oracle import metrics
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def test_noalloc_blocks_match_covariance_path_twice():
    torch = pytest.importorskip("torch")
    sc = synth.workload("ring20")
    with ccov.from_scene(sc) as ctx:
        ctx.ccov_information()
        ctx.ccov_schur()
        ctx.ccov_nullspace()
        Z, G, W7 = ctx.ccov_get_schur()
        want = ctx.ccov_covariance()
    # the camera block of Z_p^-1 is (Z + G W7^-1 G^T)^-1 (block inversion of Z_p)
    Zl = np.tril(Z)
    A = Zl + np.tril(Zl, -1).T + G @ np.linalg.solve(W7, G.T)
    N = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    out = torch.empty((N // 9, 9, 9), dtype=torch.float64, device="cuda")
    fn = ccov.load().ccov_spd_inverse_blocks_noalloc
    torch.cuda.synchronize()
    for _ in range(2):
        out.fill_(np.nan)
        torch.cuda.synchronize()
        st = fn(dA.data_ptr(), N, N, out.data_ptr(), None)
        assert st == ccov.CCOV_OK
        got = out.cpu().numpy()
        assert metrics.rel_fro(got, want).max() < FP64_TOL


def test_noalloc_rejects_sizes_beyond_its_workspace():
    fn = ccov.load().ccov_spd_inverse_blocks_noalloc
    # checked before any device work: the pointers are never touched
    assert fn(8, 585, 585, 8, None) == ccov.CCOV_ERR_INVALID_ARG
    assert fn(8, 20, 20, 8, None) == ccov.CCOV_ERR_INVALID_ARG   # not a multiple of 9
