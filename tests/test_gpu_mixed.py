"""The tensor-core (digit-split, emulated FP64) path of step (d).

The GEMM kernel is checked bit-exactly against the integer definition of
its output; the full mixed path against the oracle at the 1e-6 relative
Frobenius bar per camera block, and against the FP64 GPU path."""
import numpy as np
import pytest

from _checks import assert_blocks_close
from oracle import covariance, metrics
from paper_1808_02414_gb300 import ccov, synth

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def _bf16_bits(d):
    f = d.astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def _expected(dA, eA, dB, eB, s, Fc, sub, lower, C0):
    """Integer definition of the kernel's result: T = sum_g P_g 2^(8 (s-1-g)),
    P_g = sum_{a+b=g} A_a B_b^T (exact), shifted once to Q(Fc) with the row
    and column exponents (round half up on right shifts, wrap-around on left)."""
    M, N = dA.shape[1], dB.shape[1]
    T = np.zeros((M, N), dtype=np.int64)
    for g in range(s):
        P = np.zeros((M, N), dtype=np.int64)
        for a in range(g + 1):
            P += dA[a] @ dB[g - a].T
        with np.errstate(over="ignore"):
            T = (T << 8) + P
    sh = eA[:, None] + eB[None, :] + Fc - 14 - 8 * (s - 1)
    pos = sh >= 0
    with np.errstate(over="ignore"):
        left = T << np.where(pos, sh, 0)
        rs = np.where(pos, 0, -sh)
        right = (T + (np.int64(1) << np.maximum(rs - 1, 0))) >> rs
        S = np.where(pos, left, np.where(rs > 0, right, T))
    out = C0 - S if sub else S
    if lower:
        ti = np.arange(M)[:, None] // 128
        tj = np.arange(N)[None, :] // 64
        keep = tj * 64 <= ti * 128 + 127
        out = np.where(keep, out, C0)
    return out


def _run(s, M, N, Fc, sub, lower, seed, with_exp=True, K=128):
    rng = np.random.default_rng(seed)
    dA = rng.integers(-128, 129, size=(s, M, K)).astype(np.int64)
    dB = rng.integers(-128, 129, size=(s, N, K)).astype(np.int64)
    eA = rng.integers(-3, 4, size=M).astype(np.int32) if with_exp else np.zeros(M, np.int32)
    eB = rng.integers(-3, 4, size=N).astype(np.int32) if with_exp else np.zeros(N, np.int32)
    C0 = rng.integers(-(1 << 50), 1 << 50, size=(M, N)).astype(np.int64)
    Cg = C0.copy()
    fn = ccov.load().ccov_test_ozaki_gemm
    ba, bb = _bf16_bits(dA), _bf16_bits(dB)
    st = fn(s, K, M, N, ba.ctypes.data, eA.ctypes.data if with_exp else None, bb.ctypes.data,
            eB.ctypes.data if with_exp else None, Fc, sub, lower, Cg.ctypes.data)
    assert st == 0
    want = _expected(dA, eA.astype(np.int64), dB, eB.astype(np.int64), s, Fc, sub, lower, C0)
    return Cg, want


@pytest.mark.parametrize("s", [4, 5, 6])
@pytest.mark.parametrize("K", [128, 256])
def test_ozaki_gemm_single_tile_bit_exact(s, K):
    got, want = _run(s, 128, 128, 60, 1, 0, seed=s, with_exp=False, K=K)
    assert np.array_equal(got, want)


def test_ozaki_gemm_extreme_digits_exact():
    """All digits +-128: the largest digit orders reach the fp32 exactness limit."""
    for K in (128, 256):
        s, M, N = 6, 128, 128
        dA = np.full((s, M, K), 128, dtype=np.int64)
        dB = np.full((s, N, K), -128, dtype=np.int64)
        C0 = np.zeros((M, N), dtype=np.int64)
        Cg = C0.copy()
        fn = ccov.load().ccov_test_ozaki_gemm
        ba, bb = _bf16_bits(dA), _bf16_bits(dB)   # keep the buffers alive across the call
        st = fn(s, K, M, N, ba.ctypes.data, None, bb.ctypes.data, None, 60, 1, 0, Cg.ctypes.data)
        assert st == 0
        want = _expected(dA, np.zeros(M, np.int64), dB, np.zeros(N, np.int64), s, 60, 1, 0, C0)
        assert np.array_equal(Cg, want)


@pytest.mark.parametrize("sub,Fc", [(1, 60), (0, 42)])
def test_ozaki_gemm_with_exponents_bit_exact(sub, Fc):
    got, want = _run(5, 256, 384, Fc, sub, 0, seed=11 + sub)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("K", [128, 256])
def test_ozaki_gemm_many_tiles_persistent_bit_exact(K):
    # 16 x 20 = 320 tiles: every CTA runs several tiles through the smem ring
    got, want = _run(5, 2048, 1280, 60, 1, 0, seed=5, with_exp=False, K=K)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("K", [128, 256])
def test_ozaki_gemm_lower_tiles_bit_exact(K):
    got, want = _run(6, 640, 640, 60, 1, 1, seed=7, with_exp=False, K=K)
    assert np.array_equal(got, want)


def test_ozaki_gemm_overwrite_with_exponents_k256():
    got, want = _run(5, 384, 256, 42, 0, 0, seed=21, K=256)
    assert np.array_equal(got, want)


# K = 512 (the trailing updates of four sub-panels): eight accumulators.  With
# four digits every one is exact; with five, the second accumulator of the
# lowest order takes three products and may round once its sum passes 2^24,
# which uniform digits never reach (their sums stay near 2^17).
@pytest.mark.parametrize("s", [4, 5])
def test_ozaki_gemm_k512_single_tile_bit_exact(s):
    got, want = _run(s, 128, 128, 60, 1, 0, seed=30 + s, with_exp=False, K=512)
    assert np.array_equal(got, want)


def test_ozaki_gemm_k512_many_tiles_lower_and_exponents():
    got, want = _run(5, 1280, 1280, 60, 1, 1, seed=33, with_exp=False, K=512)
    assert np.array_equal(got, want)
    got, want = _run(5, 384, 640, 42, 0, 0, seed=34, K=512)
    assert np.array_equal(got, want)


def test_ozaki_gemm_k512_extreme_digits_within_the_rounding_bound():
    """Digits near +-128 with odd products, so that every accumulator sum
    passes 2^23 and the lowest order's second one (three products) passes
    2^24 with odd partial sums: every other order stays exact, and the
    lowest order's rounding (at most one unit of 2 per accumulation into
    an fp32 value below 2^25: 32 K-steps x 3 MMAs) enters T with weight 1,
    shifted to Q60 by 2^(60 - 14 - 32)."""
    s, K, M, N = 5, 512, 128, 128
    dA = np.full((s, M, K), 128, dtype=np.int64)
    dB = np.full((s, N, K), 128, dtype=np.int64)
    dA[:, :, ::16] = 127                    # one odd product per 16-wide K step
    dB[:, :, ::16] = 127
    C0 = np.zeros((M, N), dtype=np.int64)
    Cg = C0.copy()
    fn = ccov.load().ccov_test_ozaki_gemm
    ba, bb = _bf16_bits(dA), _bf16_bits(dB)
    assert fn(s, K, M, N, ba.ctypes.data, None, bb.ctypes.data, None, 60, 1, 0, Cg.ctypes.data) == 0
    want = _expected(dA, np.zeros(M, np.int64), dB, np.zeros(N, np.int64), s, 60, 1, 0, C0)
    bound = 32 * 3 * 2 * 2 ** (60 - 14 - 32)
    assert np.abs(Cg - want).max() <= bound
    # the rest of T is exact: the error is below one unit of the next order up
    assert np.abs(Cg - want).max() < 2 ** 8 * 2 ** (60 - 14 - 32)


@pytest.mark.parametrize("case", ["ring20", "shell10", "shell30", "shell100", "shell300"])
def test_mixed_covariance_vs_oracle(case):
    # shell10: one 128-column block; shell30: three (an odd count: the last
    # sub-panel has no partner); the others span 2, 8 and 22 blocks
    if case == "ring20":
        sc = synth.workload("ring20")
    elif case == "shell10":
        sc = synth.shell_scene(n=10, m=1000, seed=3)
    elif case == "shell30":
        sc = synth.shell_scene(n=30, m=3000, seed=4)
    elif case == "shell100":
        sc = synth.shell_scene(n=100, m=10000, seed=5)
    else:
        sc = synth.shell_scene(n=300, m=30000, seed=6)
    want = covariance.camera_covariance(sc)
    got = ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED)
    assert_blocks_close(got, want, MIXED_TOL)


def test_mixed_six_digits_tighter():
    sc = synth.shell_scene(n=100, m=10000, seed=5)
    want = ccov.camera_covariances(sc)
    got = ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED, mixed_slices=6)
    assert_blocks_close(got, want, 1e-8)


def test_mixed_repeatable_on_a_user_stream_and_after_reload():
    """The mixed form forks its Cholesky and triangular inverse onto internal
    streams and joins them back onto the context stream: repeated calls, a
    user-provided stream and new inputs give the same blocks."""
    torch = pytest.importorskip("torch")
    sc = synth.shell_scene(n=60, m=3000, seed=12)
    want = covariance.camera_covariance(sc)
    user = torch.cuda.Stream()
    with ccov.from_scene(sc, precision=ccov.CCOV_PREC_MIXED, stream=user.cuda_stream) as ctx:
        a = ctx.run()
        b = ctx.run()
        moved = sc.cams.copy()
        moved[:, 3:6] *= 1.5            # a scaled scene: covariances of t change by 1.5^2
        ctx.ccov_load(moved, sc.pts * 1.5, sc.obs_records())
        c = ctx.run()
        ctx.ccov_load(sc.cams, sc.pts, sc.obs_records())
        d = ctx.run()
    assert_blocks_close(a, want, 1e-6)
    # every sum runs in a fixed order (no atomics; integer reduce-adds of the
    # digit products commute exactly): identical bits
    assert np.array_equal(a, b)
    assert np.array_equal(a, d)
    scaled = covariance.camera_covariance(synth.Scene(cams=moved, pts=sc.pts * 1.5, obs_cam=sc.obs_cam,
                                                      obs_pt=sc.obs_pt, obs_u=sc.obs_u, sigma=sc.sigma))
    assert_blocks_close(c, scaled, 1e-6)


def test_gemm_wait_limit_runs_out_and_the_library_stays_usable():
    """The producer of every CTA leaves out one pipeline fill, so the MMA
    issuer waits for operands that never arrive: with a 2 ms limit the wait
    gives up, the kernel leaves every loop, drains its MMAs, frees TMEM and
    the call returns TIMEOUT.  The next calls (the same GEMM without the gap,
    and a whole covariance) are exact again."""
    s, K, M, N = 5, 128, 256, 256
    rng = np.random.default_rng(31)
    dA = rng.integers(-128, 129, size=(s, M, K)).astype(np.int64)
    dB = rng.integers(-128, 129, size=(s, N, K)).astype(np.int64)
    C0 = rng.integers(-(1 << 50), 1 << 50, size=(M, N)).astype(np.int64)
    ba, bb = _bf16_bits(dA), _bf16_bits(dB)
    L = ccov.load()
    for skip in (0, 3, 7):      # the first fill, a middle one, the last of the tile
        Cg = C0.copy()
        st = L.ccov_test_ozaki_gemm_wait(s, K, M, N, ba.ctypes.data, None, bb.ctypes.data, None, 60, 1, 0,
                                         Cg.ctypes.data, skip, 2_000_000)
        assert st == ccov.CCOV_ERR_TIMEOUT
        assert np.array_equal(Cg, C0)           # nothing copied back on failure
    Cg = C0.copy()
    st = L.ccov_test_ozaki_gemm_wait(s, K, M, N, ba.ctypes.data, None, bb.ctypes.data, None, 60, 1, 0,
                                     Cg.ctypes.data, -1, 2_000_000)
    assert st == ccov.CCOV_OK
    want = _expected(dA, np.zeros(M, np.int64), dB, np.zeros(N, np.int64), s, 60, 1, 0, C0)
    assert np.array_equal(Cg, want)
    sc = synth.workload("ring20")
    assert_blocks_close(ccov.camera_covariances(sc, precision=ccov.CCOV_PREC_MIXED),
                        covariance.camera_covariance(sc), MIXED_TOL)
