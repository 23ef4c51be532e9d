"""The oracle's repair of fix-and-propagate (Section 2.3, the repair branch of Algorithm 1) against
a hand-worked case and brute force on tiny integer problems."""
import itertools

import numpy as np
import pytest

import oracle
from tests.helpers import load_golden, milp_from_dense


def _golden():
    d = load_golden("fp_repair.json")
    p = milp_from_dense(d["A"], d["g"], d["lb"], d["ub"], [1] * d["n"])
    return d, p


@pytest.mark.parametrize("seed", range(1, 9))
def test_hand_worked_case(seed):
    d, p = _golden()
    P = oracle.Problem(p)
    x = np.array(d["x"])
    out, r = P.fix_and_propagate(x, p.lb, p.ub, seed=seed)
    want = d["without_repair"]
    assert r["status"] == want["status"] and r["bulks"] == want["bulks"] and r["repairs"] == 0
    np.testing.assert_array_equal(out, want["x_out"])
    out, r = P.fix_and_propagate(x, p.lb, p.ub, seed=seed, repair_max=4)
    # x1 is bulk 1's variable (index 1), drawn up when its uniform falls below P(up) = 0.7
    up = oracle.uniform(seed, 1, 1, 0) < d["p_up_x1"]
    want = d["with_repair"]["x1_drawn_up" if up else "x1_drawn_down"]
    for k in ("status", "bulks", "fixed_by_choice", "repairs", "repair_runs", "bp_runs"):
        assert r[k] == want[k], (k, r, want)
    np.testing.assert_array_equal(out, want["x_out"])
    assert r["fragile"] == 0


@pytest.mark.parametrize("seed", range(1, 9))
def test_hand_worked_case_with_implied_fixing(seed):
    """An implied bound of a fixing the repair moves must not survive it: every repair
    propagation starts from the caller's bounds."""
    d = load_golden("fp_repair.json")
    c = d["with_implied"]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], [1] * 4)
    P = oracle.Problem(p)
    x = np.array(c["x"])
    out, r = P.fix_and_propagate(x, p.lb, p.ub, seed=seed)
    assert r["status"] == c["without_repair"]["status"] and r["bulks"] == c["without_repair"]["bulks"]
    np.testing.assert_array_equal(out, c["without_repair"]["x_out"])
    out, r = P.fix_and_propagate(x, p.lb, p.ub, seed=seed, repair_max=4)
    up = oracle.uniform(seed, 1, 1, 0) < d["p_up_x1"]
    want = c["with_repair"]["x1_drawn_up" if up else "x1_drawn_down"]
    for k in ("status", "bulks", "fixed_by_choice", "repairs", "repair_runs", "bp_runs"):
        assert r[k] == want[k], (k, r, want)
    np.testing.assert_array_equal(out, want["x_out"])


@pytest.mark.parametrize("case", range(5))
def test_repair_step(case):
    d = load_golden("fp_repair.json")["steps"]
    c = d["cases"][case]
    p = milp_from_dense([c["row"]], [c["g"]], d["lb"], d["ub"], [1, 1])
    moved, cval, fragile = oracle.Problem(p).repair_step(c["l"], c["u"], 0, -1, d["lb"], d["ub"], c["chosen"],
                                                         c["cval"])
    assert moved == c["moved"] and fragile == 0
    np.testing.assert_array_equal(cval, c["cval_out"])


def test_both_draws_occur():
    d, _ = _golden()
    ups = {oracle.uniform(s, 1, 1, 0) < d["p_up_x1"] for s in range(1, 9)}
    assert ups == {True, False}


def test_repair_cycles_bound():
    """With one repair propagation allowed the hand-worked repair cannot finish."""
    d, p = _golden()
    out, r = oracle.Problem(p).fix_and_propagate(np.array(d["x"]), p.lb, p.ub, seed=1, repair_max=4,
                                                 repair_cycles=1)
    assert r["status"] == 1 and r["repairs"] == 0 and r["repair_runs"] == 1


def test_repair_needs_no_cache():
    d, p = _golden()
    cache = {"pairs": np.array([0], np.int32), "boxes": np.array([[0, 0, 1, 1]], float),
             "status": np.array([0, 0], np.int32), "offsets": np.array([0, 0, 0], np.int64),
             "var": np.zeros(0, np.int32), "l": np.zeros(0), "u": np.zeros(0)}
    with pytest.raises(ValueError):
        oracle.Problem(p).fix_and_propagate(np.array(d["x"]), p.lb, p.ub, cache=cache, repair_max=1)


def _tiny(rng, n, m, ub_max):
    """Random small integer rows over n integer variables in [0, ub], right-hand sides that a
    planted integer point satisfies (with random slack 0 or 1)."""
    ub = rng.integers(1, ub_max + 1, n).astype(float)
    x0 = np.array([rng.integers(0, int(u) + 1) for u in ub], dtype=float)
    A = np.zeros((m, n))
    for k in range(m):
        cols = rng.choice(n, size=rng.integers(2, n + 1), replace=False)
        A[k, cols] = rng.integers(-3, 4, len(cols))
        if not A[k].any():
            A[k, cols[0]] = 1
    g = A @ x0 + rng.integers(0, 2, m)
    if rng.random() < 0.3:   # sometimes no integer point at all
        g = g - rng.integers(1, 4, m)
    return milp_from_dense(A, g, np.zeros(n), ub, np.ones(n)), A, g, ub


def _integer_points(ub):
    return itertools.product(*[range(int(u) + 1) for u in ub])


def _tiny_planted(rng, n, m, eq_frac, ub_max):
    """Rows over 2-4 variables with coefficients in {-2, -1, 1, 2} that a planted integer point
    satisfies, a share of them as equality pairs; the point to round lies near the opposite
    corner (ub - planted), so the early fixings tend to be wrong."""
    ub = rng.integers(1, ub_max + 1, n).astype(float)
    x0 = np.array([rng.integers(0, int(u) + 1) for u in ub], dtype=float)
    rows, rhs = [], []
    for _ in range(m):
        cols = rng.choice(n, size=rng.integers(2, min(n, 4) + 1), replace=False)
        a = np.zeros(n)
        a[cols] = rng.choice([-2, -1, 1, 2], len(cols))
        b = a @ x0
        if rng.random() < eq_frac:
            rows += [a, -a]
            rhs += [b, -b]
        else:
            rows.append(a)
            rhs.append(b + rng.integers(0, 2))
    A, g = np.array(rows), np.array(rhs, dtype=float)
    x = np.clip(ub - x0 + rng.uniform(-0.2, 0.2, n), 0, ub)
    return milp_from_dense(A, g, np.zeros(n), ub, np.ones(n)), A, g, ub, x


def _check_tiny(p, A, g, ub, x, seed, exists):
    P = oracle.Problem(p)
    o0, r0 = P.fix_and_propagate(x, p.lb, p.ub, seed=seed)
    oz, rz = P.fix_and_propagate(x, p.lb, p.ub, seed=seed, repair_max=0)
    o1, r1 = P.fix_and_propagate(x, p.lb, p.ub, seed=seed, repair_max=6)
    # repair off is the default
    assert r0 == rz and np.array_equal(o0, oz)
    # a repair run that never needed one equals the plain run
    if r1["repair_runs"] == 0:
        assert r1 == r0 and np.array_equal(o1, o0), (r0, r1)
    # sound: a feasible verdict is an integer point inside the bounds satisfying every row
    for o, r in ((o0, r0), (o1, r1)):
        assert (o == np.round(o)).all() and (o >= 0).all() and (o <= ub).all()
        if r["status"] == 0:
            assert (A @ o <= g + 1e-9).all(), (o, r)
    if not exists:
        assert r1["status"] == 1
    assert r1["repairs"] <= 6 and r1["repair_runs"] <= 6 * 8
    assert r0["fragile"] == 0 and r1["fragile"] == 0   # integer data: every decision exact
    return r0, r1


def test_brute_force_random_rows():
    """Random integer rows, a third of the problems without any integer point."""
    rng = np.random.default_rng(2024)
    infeasible = 0
    for _ in range(300):
        n = int(rng.integers(3, 7))
        p, A, g, ub = _tiny(rng, n, int(rng.integers(2, 6)), 2)
        exists = any((A @ np.array(pt) <= g + 1e-9).all() for pt in _integer_points(ub))
        infeasible += not exists
        _check_tiny(p, A, g, ub, rng.uniform(0, ub), int(rng.integers(1, 1000)), exists)
    assert infeasible > 30


def test_brute_force_planted_dead_ends():
    """Planted feasible problems rounded from the opposite corner: the repair turns some failed
    roundings into feasible ones (and only sound ones, checked row by row)."""
    rng = np.random.default_rng(11)
    helped = tried = 0
    for _ in range(300):
        n = int(rng.integers(4, 9))
        p, A, g, ub, x = _tiny_planted(rng, n, int(rng.integers(3, 7)), 0.3, 2)
        r0, r1 = _check_tiny(p, A, g, ub, x, int(rng.integers(1, 1000)), True)
        tried += r1["repair_runs"] > 0
        helped += r0["status"] == 1 and r1["status"] == 0
    assert helped >= 3 and tried > helped, (helped, tried)


def test_repair_step_skips_a_row_with_an_infinite_minimal_activity():
    """A target row whose minimal activity is -inf (an unbounded-below variable in it) is not
    violated, so no fixing shifts: x0 + y <= 1 with x0 chosen at 5 in [0, 10] and y unbounded
    below (counting only x0's finite part, the row would look violated by 4)."""
    lb = np.array([0.0, -np.inf])
    ub = np.array([10.0, 10.0])
    p = milp_from_dense([[1.0, 1.0]], [1.0], lb, ub, [1, 0])
    l = np.array([5.0, -np.inf])
    u = np.array([5.0, 10.0])
    moved, cval, fragile = oracle.Problem(p).repair_step(l, u, 0, -1, lb, ub, [1, 0], [5.0, 0.0])
    assert moved == -1
    np.testing.assert_array_equal(cval, [5.0, 0.0])
