"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: information blocks, nullspace and Schur blocks are FP64 sums of a
few hundred terms of magnitude up to |Z|: 1e-11 relative to the largest entry
covers rounding-order differences.  Camera covariance blocks: 1e-9 relative
Frobenius error per block for the FP64 path."""
import numpy as np
import pytest

from _checks import assert_blocks_close
from oracle import camera, covariance, information, metrics, nullspace
from paper_1808_02414_gb300 import ccov, synth

from _scenes import golden_entries

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def _ctx(sc, **kw):
    return ccov.from_scene(sc, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("aniso", [False, True])
def test_information_blocks(aniso):
    sc = synth.tiny_scene(n=6, m=60, track_len=4, seed=2, anisotropic=aniso)
    U, A, W, Jc, Jp = information.blocks(sc)
    with _ctx(sc) as ctx:
        ctx.ccov_information()
        Ug, Ag, Wg = ctx.ccov_get_blocks()
    assert _rel(Ug, U) < 1e-12
    assert _rel(Ag, np.linalg.inv(A)) < 1e-11
    assert _rel(Wg, W) < 1e-12


@pytest.mark.parametrize("route", [ccov.CCOV_NULL_PAPER, ccov.CCOV_NULL_CLOSED])
def test_nullspace_camera_rows(route):
    sc = synth.workload("ring20")
    Jc, Jp = camera.jacobians(sc.cams, sc.pts, sc.obs_cam, sc.obs_pt)
    want = nullspace.camera_rows(sc, Jc, Jp)
    with _ctx(sc, nullspace_route=route) as ctx:
        got = ctx.ccov_nullspace(want_hp=True)
    assert np.abs(got - want).max() < 1e-11


@pytest.mark.parametrize("n,m", [(20, 500), (100, 8000)])
def test_schur_blocks(n, m):
    sc = synth.workload("ring20") if n == 20 else synth.shell_scene(n=n, m=m, seed=5)
    Z, G, W7 = covariance.schur_blocks_unscaled(sc)
    with _ctx(sc) as ctx:
        ctx.ccov_information()
        ctx.ccov_schur()
        ctx.ccov_nullspace()
        Zg, Gg, W7g = ctx.ccov_get_schur()
    low = np.tril_indices(Z.shape[0])
    assert np.abs(Zg[low] - Z[low]).max() / np.abs(Z).max() < 1e-11
    assert _rel(Gg, G) < 1e-11
    assert _rel(W7g, W7) < 1e-11


@pytest.mark.parametrize("name,sc,gt", golden_entries(), ids=lambda x: x if isinstance(x, str) else "")
def test_covariance_vs_extended_precision_ground_truth(name, sc, gt):
    got = ccov.camera_covariances(sc)
    assert_blocks_close(got, gt, FP64_TOL)


@pytest.mark.parametrize("case", ["ring20", "aniso", "shell100", "shell300"])
def test_covariance_vs_oracle(case):
    if case == "ring20":
        sc = synth.workload("ring20")
    elif case == "aniso":
        sc = synth.tiny_scene(n=12, m=300, track_len=4, seed=7, anisotropic=True)
    elif case == "shell100":
        sc = synth.shell_scene(n=100, m=10000, seed=5)
    else:
        sc = synth.shell_scene(n=300, m=30000, seed=6)   # N = 2700: 22 tiles, ragged tail
    want = covariance.camera_covariance(sc)
    got = ccov.camera_covariances(sc)
    assert_blocks_close(got, want, FP64_TOL)
    np.testing.assert_allclose(got, np.transpose(got, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(got).max())


@pytest.mark.parametrize("prec,tol", [(ccov.CCOV_PREC_FP64, FP64_TOL), (ccov.CCOV_PREC_MIXED, 1e-6)])
def test_three_cameras_one_padded_block(prec, tol):
    """The smallest well-posed scene: three cameras (N = 27 in one 128-row
    block, 101 rows of padding; with two cameras the intrinsics are not
    determined and the system is singular beyond the gauge)."""
    sc = synth.ring_scene(n=3, m=40, track_len=3, seed=3)
    assert_blocks_close(ccov.camera_covariances(sc, precision=prec), covariance.camera_covariance(sc), tol)


def test_paper_route_and_closed_form_nullspace_agree_on_covariance():
    sc = synth.shell_scene(n=60, m=4000, seed=9)
    a = ccov.camera_covariances(sc, nullspace_route=ccov.CCOV_NULL_PAPER)
    b = ccov.camera_covariances(sc, nullspace_route=ccov.CCOV_NULL_CLOSED)
    assert_blocks_close(a, b, FP64_TOL)


def test_repeatable_and_reloadable():
    sc = synth.shell_scene(n=40, m=2000, seed=10)
    with _ctx(sc) as ctx:
        a = ctx.run()
        b = ctx.run()
        ctx.ccov_load(sc.cams, sc.pts, sc.obs_records())
        c = ctx.run()
    # every sum of the path runs in a fixed order: identical bits
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


def test_device_resident_inputs_and_outputs():
    torch = pytest.importorskip("torch")
    sc = synth.shell_scene(n=30, m=1500, seed=11)
    cams = torch.from_numpy(sc.cams).cuda()
    pts = torch.from_numpy(sc.pts).cuda()
    obs = torch.from_numpy(sc.obs_records().view(np.uint8)).cuda()
    out = torch.empty((sc.n, 9, 9), dtype=torch.float64, device="cuda")
    with ccov.Context(cams, pts, obs, sc.sigma) as ctx:
        ctx.run(out=out)
    want = ccov.camera_covariances(sc)
    assert np.array_equal(out.cpu().numpy(), want)


def test_degenerate_and_invalid_inputs_are_rejected():
    sc = synth.ring_scene(n=6, m=40, track_len=3, seed=1)
    rec = sc.obs_records()
    # a point seen once (point 0 has three observations: drop two)
    bad = rec[2:].copy()
    with pytest.raises(ccov.CcovError) as e:
        ccov.Context(sc.cams, sc.pts, bad, 1.0)
    assert e.value.status == ccov.CCOV_ERR_DEGENERATE
    # unsorted observations
    with pytest.raises(ccov.CcovError) as e:
        ccov.Context(sc.cams, sc.pts, rec[::-1].copy(), 1.0)
    assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
    # camera index out of range
    bad = rec.copy()
    bad["cam"][0] = 99
    with pytest.raises(ccov.CcovError) as e:
        ccov.Context(sc.cams, sc.pts, bad, 1.0)
    assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
    # a point behind its cameras
    pts = sc.pts.copy()
    i = sc.obs_cam[0]
    center = -camera.rotation_matrix(sc.cams[i, :3]).T @ sc.cams[i, 3:6]
    pts[sc.obs_pt[0]] = 2.0 * center          # beyond the camera, opposite its view
    with ccov.Context(sc.cams, pts, rec, 1.0) as ctx:
        with pytest.raises(ccov.CcovError) as e:
            ctx.ccov_information()
    assert e.value.status == ccov.CCOV_ERR_DEGENERATE
    # calls out of order
    with ccov.Context(sc.cams, sc.pts, rec, 1.0) as ctx:
        with pytest.raises(ccov.CcovError) as e:
            ctx.ccov_covariance()
    assert e.value.status == ccov.CCOV_ERR_INVALID_ARG
