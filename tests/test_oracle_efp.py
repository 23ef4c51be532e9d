"""The extended feasibility pump orchestration oracle (oracle/efp.py, Algorithm 2): its own
steps by hand, and end to end: a reported feasible point satisfies every row."""
import numpy as np
import pytest

from oracle import efp, local_mip
from paper_2510_20499_gb300 import synth


def test_snap_and_nearest():
    lb, ub = np.array([0.0, 0.0, -1.0]), np.array([1.0, 5.0, 1.0])
    x = np.array([0.3 + 2.0 ** -22, 4.75 + 2.0 ** -21, -2.0])   # a tie at 2^-21 rounds to even
    s = efp.snap(x, lb, ub)
    assert s[0] == np.round(0.3 * 2 ** 20) / 2 ** 20 and s[1] == 4.75 and s[2] == -1.0
    assert np.array_equal(efp.nearest([1, 1, 0], np.array([0.5, 2.49, 0.3]), lb, ub), [1.0, 2.0, 0.3])


def test_projection_objective_and_distance():
    is_int = [1, 1, 1, 0, 1]
    lb = np.array([0.0, 0.0, 0.0, 0.0, 2.0])
    ub = np.array([1.0, 3.0, 3.0, 1.0, 2.0])
    s = np.array([0.0, 3.0, 1.0, 0.0, 2.0])
    # at lower bound: +1; at upper: -1; inside or continuous or fixed: 0
    assert np.array_equal(efp.projection_objective(is_int, s, lb, ub), [1.0, -1.0, 0.0, 0.0, 0.0])
    x = np.array([0.25, 2.5, 1.0, 0.75, 2.0])
    assert efp.distance(is_int, x, s) == 0.25 + 0.5   # continuous variables do not count


def test_cycle_rule():
    h = [10.0, 8.0, 6.0]
    assert not efp.cycle(h[:2], 5.0, 3, 0.1)            # fewer than N earlier distances
    assert not efp.cycle(h, 7.0 - 0.71, 3, 0.1)         # mean 8: improves by 1.71 > 0.8
    assert efp.cycle(h, 7.2, 3, 0.1)                    # improves by 0.8 <= 0.1 * 8
    assert efp.cycle(h, 9.0, 3, 0.1)                    # worse than the mean


@pytest.mark.parametrize("seed", range(4))
def test_end_to_end_sound(seed):
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).normal(0, 1, p.n)
    x, r = efp.run(p, p.lb, p.ub, rounds=6, lp_iterations=200, ls_iterations=100, seed=seed + 1)
    assert (x >= p.lb).all() and (x <= p.ub).all()
    assert (x[p.is_int == 1] == np.round(x[p.is_int == 1])).all()
    if r["status"] == 0:
        L = local_mip.activities(p, x)
        fin = np.isfinite(p.g)
        assert (L[fin] <= p.g[fin]).all()
    assert r["found_at"] in (-3, -2, -1) or 0 <= r["found_at"] < 6
