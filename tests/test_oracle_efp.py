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
    assert efp.cycle([10.0, 10.0, 10.0], 9.0, 3, 0.1)   # improves by exactly 10% of the mean: a cycle
    assert efp.cycle([100.0, 10.0, 10.0, 10.0], 9.5, 3, 0.1)   # the mean of the last N only (10, not 32.5)


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


# --- improvement mode (the objective cut at each feasible point) ---


def test_with_cut_row():
    """The cut problem appends one row: the nonzero costs in column order, right-hand side
    c x* - delta; its other rows are the problem's."""
    p = synth.knapsack_cover(seed=711, m=30, n=60, nnz=300)
    p.c = np.zeros(p.n)
    p.c[[3, 17, 40]] = [2.0, -1.0, 5.0]
    xb = np.zeros(p.n)
    xb[[3, 40]] = 1.0
    q = efp.with_cut(p, xb)
    assert q.m == p.m + 1 and q.nnz == p.nnz + 3
    np.testing.assert_array_equal(q.col[p.nnz:], [3, 17, 40])
    np.testing.assert_array_equal(q.val[p.nnz:], [2.0, -1.0, 5.0])
    assert q.g[-1] == 7.0 - 1.0                         # c x* = 7, integral objective: delta = 1
    np.testing.assert_array_equal(q.g[:-1], p.g)
    np.testing.assert_array_equal(q.col[:p.nnz], p.col)
    p.c[17] = -0.5                                      # a fractional cost: delta = 1e-4
    assert efp.with_cut(p, xb).g[-1] == 7.0 - 1e-4


def _rows_ok(p, x):
    L = local_mip.activities(p, x)
    fin = np.isfinite(p.g)
    return bool((L[fin] <= p.g[fin]).all())


@pytest.mark.parametrize("seed", range(4))
def test_improvement_mode(seed):
    """The first incumbent is generation mode's point; every incumbent satisfies every row of
    the problem, is integral on integer variables, and improves on the previous one by at least
    delta (1: integral costs); the returned point is the last incumbent."""
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    kw = dict(rounds=6, lp_iterations=200, ls_iterations=100, seed=seed + 1)
    xg, rg = efp.run(p, p.lb, p.ub, **kw)
    xi, ri = efp.run(p, p.lb, p.ub, improve=True, **kw)
    assert ri["status"] == rg["status"] and ri["found_at"] == rg["found_at"]
    if rg["status"] != 0:
        assert ri["improvements"] == 0 and ri["rounds"] == kw["rounds"]
        return
    inc = ri["incumbents"]
    assert len(inc) == ri["improvements"] >= 1
    np.testing.assert_array_equal(inc[0], xg)
    np.testing.assert_array_equal(inc[-1], xi)
    prev = np.inf
    for x in inc:
        assert _rows_ok(p, x)
        assert (x >= p.lb).all() and (x <= p.ub).all()
        assert (x[p.is_int == 1] == np.round(x[p.is_int == 1])).all()
        f = float(p.c @ x)
        assert f <= prev - 1.0
        prev = f
    assert ri["best_objective"] == prev


@pytest.mark.parametrize("seed", [0, 2, 4])
def test_improvement_mode_polish(seed):
    """With the polish, the first incumbent is the local search's best from generation mode's
    point (never worse than it), every incumbent satisfies every row and improves on the last by
    at least delta, and the polish replaced at least one incumbent on these instances."""
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    kw = dict(rounds=6, lp_iterations=200, ls_iterations=100, seed=seed + 1)
    xg, rg = efp.run(p, p.lb, p.ub, **kw)
    xi, ri = efp.run(p, p.lb, p.ub, improve=True, polish=True, **kw)
    assert ri["status"] == rg["status"] == 0 and ri["found_at"] == rg["found_at"]
    assert ri["polished"] >= 1
    inc = ri["incumbents"]
    assert float(p.c @ inc[0]) <= float(p.c @ xg)
    _, _, xb, rr = local_mip.search_objective(p, p.lb, p.ub, xg, np.ones(p.m), kw["ls_iterations"])
    np.testing.assert_array_equal(inc[0], xb if rr["improvements"] > 1 else xg)
    prev = np.inf
    for x in inc:
        assert _rows_ok(p, x) and (x[p.is_int == 1] == np.round(x[p.is_int == 1])).all()
        f = float(p.c @ x)
        assert f <= prev - 1.0
        prev = f
    np.testing.assert_array_equal(inc[-1], xi)
