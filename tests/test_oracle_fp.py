"""Pins of the oracle's fix-and-propagate rounding (Algorithm 1, Section 2.3)."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.helpers import dense, feasible_points, load_golden, milp_from_dense


def test_splitmix64_reference_values():
    """The generator's published reference outputs for the state 1234567 (SplitMix64, Steele,
    Lea and Flood 2014; the same values as the reference C implementation's test)."""
    gamma = 0x9E3779B97F4A7C15
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    s = 1234567
    for w in want:
        assert oracle.splitmix64(s) == w
        s = (s + gamma) % (1 << 64)


def test_uniform_range_and_independence():
    u = np.array([oracle.uniform(7, b, j, d) for b in range(20) for j in range(50) for d in range(2)])
    assert ((u >= 0) & (u < 1)).all()
    assert abs(u.mean() - 0.5) < 0.03
    assert len(set(u.tolist())) == len(u)


@pytest.mark.parametrize("case", range(5))
def test_golden(case):
    c = load_golden("fp_small.json")["cases"][case]
    p = synth.Milp(c["m"], c["n"], np.array(c["row_ptr"], dtype=np.int64), np.array(c["col"], dtype=np.int32),
                   np.array(c["val"], float), np.array(c["g"], float), np.array(c["lb"], float),
                   np.array(c["ub"], float), np.array(c["is_int"], dtype=np.uint8), np.zeros(c["n"]))
    for seed in (1, 2, 3):
        x, r = oracle.Problem(p).fix_and_propagate(c["x"], p.lb, p.ub, seed=seed)
        assert r["status"] == c["status"], c["note"]
        np.testing.assert_array_equal(x, c["x_out"])
        assert r["bulks"] == c["bulks"] and r["bp_runs"] == c["bp_runs"] and r["recoveries"] == c["recoveries"]


@pytest.mark.parametrize("f,p_up", [(0.1, 0.0), (0.25, 0.0), (0.28, 0.06), (0.3, 0.1), (0.5, 0.5), (0.7, 0.9), (0.72, 0.94), (0.75, 1.0), (0.9, 1.0)])
def test_rounding_distribution(f, p_up):
    """P(round up) = 0 up to f = .25, 1 from f = .75, linear between (random near .5, nearest
    away from .5).  Measured on a problem without rows: every fixing succeeds, so x_out is the
    first draw of each variable."""
    n = 2000
    p = milp_from_dense(np.zeros((0, n)), [], np.zeros(n), np.full(n, 5.0), np.ones(n))
    x = np.full(n, 2.0 + f)
    out, r = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, seed=11, last_single=0)
    assert r["status"] == 0
    up = (out == 3.0).mean()
    assert set(np.unique(out)) <= {2.0, 3.0}
    sd = math.sqrt(max(p_up * (1 - p_up), 1e-12) / n)
    assert abs(up - p_up) <= 5 * sd + 1e-12


def test_bulk_sizes_without_rows():
    """Without rows every candidate is feasible: bulk sizes follow ceil(sqrt(remaining)) down
    to 36 remaining, then one variable per bulk."""
    n = 1000
    p = milp_from_dense(np.zeros((0, n)), [], np.zeros(n), np.ones(n), np.ones(n))
    _, r = oracle.Problem(p).fix_and_propagate(np.full(n, 0.5), p.lb, p.ub)
    rem, bulks = n, 0
    while rem > 36:
        rem -= math.isqrt(rem - 1) + 1     # ceil(sqrt(rem))
        bulks += 1
    bulks += rem
    assert r["bulks"] == bulks and r["status"] == 0 and r["bp_runs"] == 1 + 2 * bulks
    _, r = oracle.Problem(p).fix_and_propagate(np.full(n, 0.5), p.lb, p.ub, bulk_rule=1, fraction=0.05)
    rem, bulks = n, 0
    while rem > 36:
        rem -= 50
        bulks += 1
    assert r["bulks"] == bulks + rem


@pytest.mark.parametrize("seed", range(25))
def test_brute_force_soundness(seed):
    """A FEASIBLE result is an integer point satisfying every row; a problem without integer
    points never ends FEASIBLE."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(3, 8)), int(rng.integers(1, 6))
    A = rng.integers(-4, 5, size=(m, n)).astype(float)
    A[rng.uniform(size=(m, n)) < 0.3] = 0.0
    for k in range(m):
        if not A[k].any():
            A[k, rng.integers(0, n)] = 1.0
    ub = rng.integers(1, 4, size=n).astype(float)
    g = rng.integers(-2, 8, size=m).astype(float)
    p = milp_from_dense(A, g, np.zeros(n), ub, np.ones(n))
    pts = feasible_points(p, p.lb, p.ub)
    for s in range(3):
        x, r = oracle.Problem(p).fix_and_propagate(rng.uniform(0, ub), p.lb, p.ub, seed=s)
        if r["status"] == 0:
            assert (A @ x <= g + 1e-6).all() and (x >= 0).all() and (x <= ub).all()
            assert (x == np.round(x)).all()
        if len(pts) == 0:
            assert r["status"] == 1


def test_cache_keeps_only_consistent_fixings():
    """With the probing cache of every binary, a result marked FEASIBLE is feasible and no
    fixing whose cached branch is infeasible is used (checked by brute force)."""
    for seed in range(10):
        p = synth.knapsack_cover(seed=seed, m=8, n=12, nnz=40)
        P = oracle.Problem(p)
        rl, ru, r, _ = P.bp(p.lb, p.ub)
        if r["status"] != 0:
            continue
        var = np.array([j for j in range(p.n) if rl[j] < ru[j]], dtype=np.int32)
        boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=float).reshape(-1, 4)
        cache = P.probe_batch(rl, ru, var, boxes)
        cache["pairs"], cache["boxes"] = var, boxes
        A = dense(p)
        for s in range(3):
            x0 = np.random.default_rng(s).uniform(0, 1, p.n)
            x, r = P.fix_and_propagate(x0, p.lb, p.ub, seed=s, cache=cache)
            if r["status"] == 0:
                assert (A @ x <= p.g + 1e-6).all()


def test_deterministic_per_seed():
    p = synth.random_milp(3, 300, 400, len_lo=2, len_hi=10, integer_coefs=True, int_fraction=1.0, slack_scale=0.3)
    x0 = np.random.default_rng(0).uniform(0, 20, p.n)
    a = oracle.Problem(p).fix_and_propagate(x0, p.lb, p.ub, seed=5)
    b = oracle.Problem(p).fix_and_propagate(x0, p.lb, p.ub, seed=5)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1]


def test_up_prob_hook_only_inside_band():
    n = 400
    p = milp_from_dense(np.zeros((0, n)), [], np.zeros(n), np.full(n, 5.0), np.ones(n))
    x = np.where(np.arange(n) % 2 == 0, 2.5, 2.1)          # in band / below band
    for pu, want in ((1.0, 3.0), (0.0, 2.0)):
        out, r = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, seed=3, last_single=0, up_prob=np.full(n, pu))
        assert (out[0::2] == want).all()                   # f = 0.5: the hook decides
        assert (out[1::2] == 2.0).all()                    # f = 0.1: nearest, hook ignored


def test_order_score_hook():
    """Two binaries with equal fractionality and y + z <= 1: the first fixed wins.  Without a
    score the lower index goes first; a higher score for z puts z first."""
    p = milp_from_dense(np.array([[1.0, 1.0]]), [1.0], np.zeros(2), np.ones(2), np.ones(2))
    x = np.array([0.8, 0.8])
    out, _ = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub)
    np.testing.assert_array_equal(out, [1.0, 0.0])
    out, _ = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, order_score=np.array([0.0, 1.0]))
    np.testing.assert_array_equal(out, [0.0, 1.0])


def test_order_score_replaces_implied_slack_order():
    """Binaries y1..y4, all at x = 0.8 (always rounded up), rows 10 y1 + 10 y2 <= 10 and
    y3 + y4 <= 1.5, no single-variable tail.  Implied slack: S = (10/10)^2 = 1 for y1, y2 and
    (1/1.5)^2 = 0.44 for y3, y4, so the plain order puts {y1, y2} in the first bulk of
    ceil(sqrt(4)) = 2: both vectors set y1 = y2 = 1 and fail, the recovery fixes y1 = 1
    (propagation then fixes y2 = 0), and the next bulk {y3, y4} fails the same way before y3 = 1
    fixes y4 = 0: 4 bulks, 2 recoveries.  A score ranking y1, y3, y4, y2 replaces the
    implied-slack order: the first bulk {y1, y3} succeeds and propagation fixes the others
    (1 bulk, no recovery)."""
    A = np.array([[10.0, 10.0, 0.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    p = milp_from_dense(A, [10.0, 1.5], np.zeros(4), np.ones(4), np.ones(4))
    x = np.full(4, 0.8)
    out, r = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, last_single=0)
    np.testing.assert_array_equal(out, [1.0, 0.0, 1.0, 0.0])
    assert (r["bulks"], r["recoveries"], r["status"]) == (4, 2, 0)
    out, r = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, last_single=0,
                                                 order_score=np.array([3.0, 0.0, 2.0, 1.0]))
    np.testing.assert_array_equal(out, [1.0, 0.0, 1.0, 0.0])
    assert (r["bulks"], r["recoveries"], r["status"]) == (1, 0, 0)


def test_recovery_one_variable_at_a_time():
    """Hand-worked recovery (Section 2.3: a bulk that fails both ways is retried one variable at
    a time). Binaries x1, x2 at x = (0.9, 0.9), row x1 + x2 <= 1, one bulk of both (bulk rule
    fraction 1.0, no single-variable tail). f = 0.9 >= 0.75 draws 1 in both vectors, so both
    candidates are (1, 1) and the row is violated: the bulk fails both ways. Recovery takes x1
    alone: it draws 1, which propagates x2 <= 0, and every variable is fixed.
    Counts: bulks 2 (the failed pair, then x1), propagations 5 (start, two per bulk), one
    recovery, one fixing by choice. Nonzeros: start 2 (one round over the row); each failed
    candidate 2; x1 = 1 takes two rounds (the row, then the row again for x2) = 4; x1 = 0 takes
    one round = 2; total 12."""
    p = milp_from_dense(np.array([[1.0, 1.0]]), [1.0], np.zeros(2), np.ones(2), np.ones(2))
    for seed in (1, 2, 3):
        xo, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 0.9]), p.lb, p.ub, seed=seed, bulk_rule=1,
                                                    fraction=1.0, last_single=0)
        assert r["status"] == 0
        assert list(xo) == [1.0, 0.0]
        assert (r["bulks"], r["bp_runs"], r["recoveries"], r["fixed_by_choice"], r["nnz_updates"]) == (2, 5, 1, 1, 12)


def _golden_slack_case():
    c = load_golden("fp_slack_order.json")
    p = synth.Milp(c["m"], c["n"], np.array(c["row_ptr"], dtype=np.int64), np.array(c["col"], dtype=np.int32),
                   np.array(c["val"], float), np.array(c["g"], float), np.array(c["lb"], float),
                   np.array(c["ub"], float), np.array(c["is_int"], dtype=np.uint8), np.zeros(c["n"]))
    return c, p


def test_implied_slack_values():
    """Implied slack of the hand-worked case (Section 2.3): squares of a / slack summed over the
    variable's rows, the slack floored at the tolerance (the 2^-21 row)."""
    c, p = _golden_slack_case()
    S = oracle.Problem(p).implied_slack(p.lb, p.ub)
    np.testing.assert_allclose(S, c["S"], rtol=1e-12, atol=0)


def test_implied_slack_special_rows():
    """Rows whose minimal activity has an infinite term, and free rows (g = +inf), add nothing;
    a row violated within the tolerance has its slack raised to the tolerance; a negative
    coefficient takes the upper bound in L_min and adds its square.  Variables x (integer [0, 1]),
    y (continuous, lower bound -inf), z (integer [0, 1]), w (integer [0, 4]):
      x + y <= 3            L_min has the infinite term of y: skipped
      x + z <= inf          free row: skipped
      x <= -5e-7            L_min = 0, slack -5e-7 -> 1e-6: x gets (1 / 1e-6)^2 = 1e12
      -2 z + w <= 1         L_min = -2, slack 3: z gets (-2/3)^2 = 4/9, w gets 1/9
    """
    inf = np.inf
    A = np.array([[1.0, 1.0, 0, 0], [1.0, 0, 1.0, 0], [1.0, 0, 0, 0], [0, 0, -2.0, 1.0]])
    p = milp_from_dense(A, [3.0, inf, -5e-7, 1.0], np.array([0.0, -inf, 0.0, 0.0]),
                        np.array([1.0, 10.0, 1.0, 4.0]), np.array([1, 0, 1, 1]))
    S = oracle.Problem(p).implied_slack(p.lb, p.ub)
    np.testing.assert_allclose(S, [1e12, 0.0, 4.0 / 9.0, 1.0 / 9.0], rtol=1e-12, atol=0)


def test_implied_slack_order_golden():
    """The asymmetric hand-worked case: decreasing implied slack puts {B, A} in the first bulk
    and C is propagated to 0.  Increasing order, |a / slack| instead of its square, or an
    unfloored slack each change the first bulk and the result (see the fixture's note)."""
    c, p = _golden_slack_case()
    for seed in (1, 2, 3):
        x, r = oracle.Problem(p).fix_and_propagate(np.array(c["x"], float), p.lb, p.ub, seed=seed,
                                                   last_single=c["last_single"])
        np.testing.assert_array_equal(x, c["x_out"])
        assert (r["status"], r["bulks"], r["bp_runs"], r["recoveries"], r["fixed_by_choice"]) == \
            (c["status"], c["bulks"], c["bp_runs"], c["recoveries"], c["fixed_by_choice"])


@pytest.mark.parametrize("coef,fragile", [(0.1, True), (1.0, False)])
def test_fragile_counts_implied_slack_ties_at_the_bulk_boundary(coef, fragile):
    """Integer variables X, A, B (at x = 0.8, so every draw rounds up) and rows
    2X <= 3, coef A + 2 Y <= 5, coef B + 2 Z <= 5 (Y, Z continuous in [0, 1], never tightened):
    S_X = 4/9 > S_A = S_B = (coef / 5)^2, and the first bulk of ceil(sqrt(3)) = 2 takes X and A,
    so the tie A = B sits on the bulk boundary.  With coef = 0.1 the rows' activities are sums
    another implementation may round differently (their windows are nonzero), so an order that
    breaks the tie the other way is as valid: the oracle counts the boundary as fragile.  With
    coef = 1 every term is an integer, every summation order is exact, and the tie is not
    fragile (the stable order holds everywhere)."""
    A = np.array([[2.0, 0, 0, 0, 0], [0, coef, 0, 2.0, 0], [0, 0, coef, 0, 2.0]])
    p = milp_from_dense(A, [3.0, 5.0, 5.0], np.zeros(5), np.ones(5), np.array([1, 1, 1, 0, 0]))
    x, r = oracle.Problem(p).fix_and_propagate(np.array([0.8, 0.8, 0.8, 0.5, 0.5]), p.lb, p.ub, last_single=0)
    assert r["bulks"] == 2 and r["status"] == 0
    assert (r["fragile"] > 0) == fragile, r


def test_final_check_refutes_an_incremental_verdict():
    """Hand-worked (Sections 2.1 and 2.3): binaries x1, x2 at 0.8 (rounded up), continuous
    y in [0, 100], z in [0, 10], rows 50 x1 + y <= 100, 0.02 x2 + y <= 50.01, -y <= -49.985,
    z - y <= -49.985, -z <= -0.01.  The start propagation gives y in [49.985, 50.01],
    z in [0.01, 0.025].  Fixing x1 = 1 proposes y <= 50 and then x2 = 1 proposes y <= 49.99:
    improvements of 0.01 and 0.02, below the threshold 1e-3 * 50.01, so both are rejected and
    every propagation of the rounding is feasible.  From the start bounds with x1 = x2 = 1 the
    same rows move y's upper bound from 100 to 49.99 in one accepted step, then z <= 0.005 < 0.01:
    row 3 is infeasible in round 2.  No continuous completion exists (z <= y - 49.985 <= 0.005),
    so the result is INFEASIBLE, marked refuted; x_out keeps the rounded point."""
    A = np.array([[50.0, 0, 1, 0], [0, 0.02, 1, 0], [0, 0, -1, 0], [0, 0, -1, 1], [0, 0, 0, -1]])
    p = milp_from_dense(A, [100, 50.01, -49.985, -49.985, -0.01], np.zeros(4), np.array([1, 1, 100, 10.0]),
                        np.array([1, 1, 0, 0]))
    P = oracle.Problem(p)
    out, r = P.fix_and_propagate(np.array([0.8, 0.8, 50.0, 0.02]), p.lb, p.ub, seed=1)
    assert (r["status"], r["refuted"], r["bulks"], r["bp_runs"], r["fragile"]) == (1, 1, 2, 5, 0)
    np.testing.assert_array_equal(out, [1.0, 1.0, 50.0, 0.02])
    # one propagation from the start bounds with x1 = x2 = 1 reaches the contradiction
    lo, hi = p.lb.copy(), p.ub.copy()
    lo[:2] = hi[:2] = 1.0
    _, _, rb, _ = P.bp(lo, hi)
    assert rb["status"] == oracle.INFEASIBLE and rb["first_infeasible_row"] == 3 and rb["rounds"] == 2


def test_last_single_boundary():
    """Exactly last_single = 36 remaining variables are fixed one per bulk (36 bulks); 37 take
    one bulk of ceil(sqrt(37)) = 7 and then 30 singles (31 bulks)."""
    for n, want in ((36, 36), (37, 31)):
        p = milp_from_dense(np.zeros((0, n)), [], np.zeros(n), np.ones(n), np.ones(n))
        _, r = oracle.Problem(p).fix_and_propagate(np.full(n, 0.5), p.lb, p.ub)
        assert r["bulks"] == want, (n, r["bulks"])


def test_ternary_class_before_general_integers():
    """The initial order puts a ternary variable (u - l = 2) before a general integer whatever
    their fractionality (Section 2.3: binary and ternary first).  z in [0, 2] at 1.8, v in [0, 5]
    at 4.9, z + v <= 5 (the start propagation changes nothing): z goes first and rounds up to 2
    (fraction 0.8), propagation gives v <= 3, and v's upward rounding is clamped to 3: (2, 3).
    Ordered by fractionality alone, v (0.1 from an integer) would go first: v = 5 and
    propagation fixes z = 0."""
    p = milp_from_dense(np.array([[1.0, 1.0]]), [5.0], np.array([0.0, 0.0]), np.array([2.0, 5.0]), np.ones(2))
    out, r = oracle.Problem(p).fix_and_propagate(np.array([1.8, 4.9]), p.lb, p.ub)
    np.testing.assert_array_equal(out, [2.0, 3.0])
    assert r["status"] == 0


# --- the probing cache inside a bulk (Section 2.2 and 2.3, readings R15 and R16), hand-made caches ---


def _cache(pairs, boxes, status, entries):
    """A probing cache written by hand: `entries[b]` lists (var, l, u) for branch b (2i: down,
    2i + 1: up of pair i)."""
    off, var, lo, hi = [0], [], [], []
    for b in range(2 * len(pairs)):
        for w, l, u in entries.get(b, []):
            var.append(w)
            lo.append(l)
            hi.append(u)
        off.append(len(var))
    return {"pairs": np.array(pairs, dtype=np.int32), "boxes": np.array(boxes, dtype=float),
            "status": np.array(status, dtype=np.int32), "offsets": np.array(off, dtype=np.int64),
            "var": np.array(var, dtype=np.int32), "l": np.array(lo, dtype=float), "u": np.array(hi, dtype=float)}


def test_cache_infeasible_branch_drops_the_fixing():
    """Two free binaries, no rows; x0 at 0.9 rounds up, but the cache marks x0 = 1 infeasible:
    that fixing is dropped, the other neighbour x0 = 0 is kept."""
    p = milp_from_dense(np.zeros((0, 2)), [], np.zeros(2), np.ones(2), np.ones(2))
    cache = _cache([0], [[0, 0, 1, 1]], [0, 1], {})
    out, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 0.1]), p.lb, p.ub, cache=cache)
    np.testing.assert_array_equal(out, [0.0, 0.0])
    out, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 0.1]), p.lb, p.ub)
    np.testing.assert_array_equal(out, [1.0, 0.0])       # without the cache it rounds up


def test_cache_implications_warm_start_the_fixing():
    """The cache says x0 = 1 implies x1 = 1: fixing x0 = 1 starts from x1 in [1, 1], so x1 (at
    0.1, which alone rounds down) ends at 1."""
    p = milp_from_dense(np.zeros((0, 2)), [], np.zeros(2), np.ones(2), np.ones(2))
    cache = _cache([0], [[0, 0, 1, 1]], [0, 0], {1: [(1, 1.0, 1.0)]})
    out, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 0.1]), p.lb, p.ub, cache=cache)
    np.testing.assert_array_equal(out, [1.0, 1.0])


def test_cache_implication_that_empties_a_domain_drops_the_fixing():
    """The cache says x0 = 1 implies x1 = 1 while x1 is fixed at 0: the implication leaves x1
    no value, so the fixing x0 = 1 is dropped before any propagation: two propagation runs (the
    start and the kept candidate x0 = 0) where trying it would take three."""
    lb, ub = np.zeros(2), np.array([1.0, 0.0])
    p = milp_from_dense(np.zeros((0, 2)), [], lb, ub, np.ones(2))
    cache = _cache([0], [[0, 0, 1, 1]], [0, 0], {1: [(1, 1.0, 1.0)]})
    out, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 0.0]), lb, ub, cache=cache)
    np.testing.assert_array_equal(out, [0.0, 0.0])
    assert r["bp_runs"] == 2 and r["status"] == 0


def test_continuous_values_are_clamped_to_the_final_bounds():
    """x0 binary at 0.9 rounds up; x0 + y <= 1 then gives y <= 0, so the continuous y given at 3
    is returned as 0."""
    lb, ub = np.zeros(2), np.array([1.0, 5.0])
    p = milp_from_dense(np.array([[1.0, 1.0]]), [1.0], lb, ub, np.array([1, 0]))
    out, r = oracle.Problem(p).fix_and_propagate(np.array([0.9, 3.0]), lb, ub)
    np.testing.assert_array_equal(out, [1.0, 0.0])
