"""The allocation-free entry point ccov_spd_inverse_blocks_noalloc.

It serves callers that cannot call cudaMalloc (a real-time loop that must not
allocate; a process whose device memory is owned by another allocator), so all
of its workspace is a fixed static device array.  Checked against the regular
ccov_covariance path on the same scene, on two calls in a row (the second call
reuses the array that the first one left behind)."""
import numpy as np
import pytest

from _checks import assert_blocks_close
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
        assert_blocks_close(got, want, FP64_TOL)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    fn = ccov.load().ccov_spd_inverse_blocks_noalloc
    # checked before any device work: the pointers are never touched
    assert fn(8, 585, 585, 8, None) == ccov.CCOV_ERR_INVALID_ARG
    assert fn(8, 20, 20, 8, None) == ccov.CCOV_ERR_INVALID_ARG   # not a multiple of 9


def test_noalloc_at_its_size_limit_with_a_leading_dimension_beyond_n():
    """N = 576 (the maximum: five 128-row blocks after padding) read from a
    larger buffer (lda > N), against numpy's inverse, on two calls in a row."""
    torch = pytest.importorskip("torch")
    N, lda = 576, 600
    rng = np.random.default_rng(3)
    B = rng.standard_normal((N, N))
    A = B @ B.T / N + np.diag(rng.uniform(0.5, 2.0, N))   # SPD, condition number about 10
    buf = np.full((N, lda), np.nan)                        # the columns beyond N are never read
    buf[:, :N] = A
    want = np.linalg.inv(A)
    want = np.stack([want[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(N // 9)])
    dA = torch.from_numpy(buf).cuda()
    out = torch.empty((N // 9, 9, 9), dtype=torch.float64, device="cuda")
    fn = ccov.load().ccov_spd_inverse_blocks_noalloc
    for _ in range(2):
        out.fill_(np.nan)
        torch.cuda.synchronize()
        assert fn(dA.data_ptr(), lda, N, out.data_ptr(), None) == ccov.CCOV_OK
        assert_blocks_close(out.cpu().numpy(), want, FP64_TOL)
