"""Pins of the sub-reconstruction oracle (Sec. 5) against what the paper and
the mathematics fix: a neighbourhood that holds the whole scene reproduces
the full result; the intrinsic (f, k1, k2) blocks of a sub-reconstruction
bound the full scene's from above (less information, larger marginal
covariance, Loewner order); every decomposition covers every camera; the
approximation error falls as the neighbourhoods grow (Fig. 5-6); the merge
keeps the smallest trace."""
import numpy as np

from oracle import covariance, metrics, subrecon
from paper_1808_02414_gb300 import synth


def test_grow_on_a_hand_made_graph():
    # weights: 0-1:5, 0-2:1, 1-3:4, 2-3:1, 3-4:9, 2-4:1
    adj = [dict() for _ in range(5)]
    for a, b, w in [(0, 1, 5), (0, 2, 1), (1, 3, 4), (2, 3, 1), (3, 4, 9), (2, 4, 1)]:
        adj[a][b] = w
        adj[b][a] = w
    # from 0: take 1 (5); then 3 (4 via 1) over 2 (1); then 4 (9 via 3); then 2
    assert subrecon.grow(0, 2, adj) == [0, 1]
    assert subrecon.grow(0, 3, adj) == [0, 1, 3]
    assert subrecon.grow(0, 4, adj) == [0, 1, 3, 4]
    assert subrecon.grow(0, 9, adj) == [0, 1, 2, 3, 4]
    # ties go to the smaller index: from 2 all neighbours weigh 1
    assert subrecon.grow(2, 2, adj) == [0, 2]


def test_view_graph_counts_shared_points():
    sc = synth.local_scene(n=12, m=300, seed=4)
    adj = subrecon.view_graph(sc.n, sc.obs_cam, sc.obs_pt)
    for i, k in [(0, 1), (3, 7), (5, 11)]:
        pi = set(sc.obs_pt[sc.obs_cam == i])
        pk = set(sc.obs_pt[sc.obs_cam == k])
        assert adj[i].get(k, 0) == len(pi & pk) == adj[k].get(i, 0)


def test_plan_covers_every_camera_in_every_decomposition():
    sc = synth.local_scene(n=40, m=3000, seed=5)
    orders = synth.decomposition_orders(sc.n, 3, seed=2)
    subs = subrecon.plan(sc, 8, orders)
    assert all(len(S) <= 8 for S in subs)
    # the sub-reconstructions of each decomposition, in order, cover 0..n-1
    covered, d, seen = set(), 0, []
    for S in subs:
        covered |= set(S)
        if len(covered) == sc.n:
            seen.append(d)
            covered, d = set(), d + 1
    assert seen == [0, 1, 2]


def test_whole_scene_neighbourhood_reproduces_the_full_result():
    sc = synth.local_scene(n=15, m=1500, seed=6)
    full = covariance.camera_covariance(sc)
    out, cover, subs = subrecon.camera_covariance(sc, sc.n, synth.decomposition_orders(sc.n, 1))
    assert len(subs) == 1 and subs[0] == list(range(sc.n))
    assert np.array_equal(cover, np.ones(sc.n, np.int32))
    assert np.array_equal(out, full)


def test_sub_reconstructions_bound_the_intrinsics_from_above():
    sc = synth.local_scene(n=30, m=3000, seed=7)
    full = covariance.camera_covariance(sc)
    for S in subrecon.plan(sc, 8, synth.decomposition_orders(sc.n, 1, seed=3)):
        sub, ids = subrecon.extract(sc, S)
        blocks = covariance.camera_covariance(sub)
        for c, b in zip(ids, blocks):
            d = b[6:9, 6:9] - full[c][6:9, 6:9]
            ev = np.linalg.eigvalsh(0.5 * (d + d.T))
            assert ev.min() > -1e-9 * np.abs(full[c][6:9, 6:9]).max()


def test_error_falls_as_the_neighbourhoods_grow():
    sc = synth.local_scene(n=48, m=4800, seed=8)
    full = covariance.camera_covariance(sc)
    orders = synth.decomposition_orders(sc.n, 2, seed=4)
    errs = []
    for k in (6, 12, 24):
        out, cover, _ = subrecon.camera_covariance(sc, k, orders)
        assert cover.min() >= 2
        errs.append(np.mean(metrics.intr_err(out, full)))
    assert errs[0] > errs[1] > errs[2]


def test_merge_keeps_the_smallest_trace():
    a = np.eye(9)[None] * 2.0
    b = np.eye(9)[None] * 1.0
    out, cover = subrecon.merge(3, [(np.array([1]), a), (np.array([1]), b), (np.array([2]), a)])
    assert np.array_equal(out[1], b[0]) and np.array_equal(out[2], a[0])
    assert np.isnan(out[0]).all() and cover.tolist() == [0, 2, 1]
