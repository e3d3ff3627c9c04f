"""The library's sub-reconstruction planner (host logic of ccov_subrecon_plan,
no GPU work) against the oracle's: identical camera sets, bit for bit."""
import numpy as np
import pytest

from oracle import subrecon
from paper_1808_02414_gb300 import ccov, synth


@pytest.mark.parametrize("n,m,k,d", [(40, 3000, 8, 3), (60, 5000, 20, 2), (25, 2000, 100, 1)])
def test_plan_matches_the_oracle(n, m, k, d):
    sc = synth.local_scene(n=n, m=m, seed=n)
    orders = synth.decomposition_orders(n, d, seed=k)
    assert ccov.subrecon_plan(sc, k, orders) == subrecon.plan(sc, k, orders)


def test_plan_on_a_scene_without_locality():
    sc = synth.shell_scene(n=30, m=2000, seed=9)
    orders = synth.decomposition_orders(30, 2, seed=1)
    assert ccov.subrecon_plan(sc, 6, orders) == subrecon.plan(sc, 6, orders)


def test_plan_rejects_an_order_that_is_not_a_permutation():
    sc = synth.local_scene(n=12, m=500, seed=2)
    orders = synth.decomposition_orders(12, 1)
    orders[0, 3] = orders[0, 4]
    with pytest.raises(ccov.CcovError):
        ccov.subrecon_plan(sc, 4, orders)
