"""The local search oracle (oracle/local_mip.py: mixed tight moves and the objective moves,
Section 2.4) against hand-worked steps, from-scratch recomputation and brute force on random
integer problems."""
import numpy as np
import pytest

from oracle import local_mip as lm
from paper_2510_20499_gb300 import synth
from tests.helpers import load_golden, milp_from_dense


def _case(c):
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], c["is_int"])
    p.c = np.array(c["c"], dtype=float)
    return p


@pytest.mark.parametrize("case", range(2))
def test_hand_worked_steps(case):
    c = load_golden("local_mip_small.json")["cases"][case]
    p = _case(c)
    for k, (want_x, want_w) in enumerate(c["steps"]):
        x, w, r = lm.search(p, p.lb, p.ub, c["x0"], c["w0"], k + 1)
        np.testing.assert_array_equal(x, want_x)
        np.testing.assert_array_equal(w, want_w)
    assert r["moves"] == c["moves"] and r["bumps"] == c["bumps"]


def _problem(seed, m=40, n=30):
    p = synth.random_milp(seed, m, n, len_lo=2, len_hi=6, int_fraction=1.0, slack_scale=0.3, integer_coefs=True)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -5.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 5.0)
    return p


def _F(p, x, w):
    return float(w @ lm.violation(lm.activities(p, x), p.g))


@pytest.mark.parametrize("seed", range(6))
def test_scores_and_steps_from_scratch(seed):
    """Every candidate's score equals the drop of F recomputed from scratch; a step moves the
    best candidate only when its score is positive (and F then drops by it), else it bumps the
    weights of exactly the violated rows; a zero violation is a feasible point."""
    p = _problem(300 + seed)
    rng = np.random.default_rng(seed)
    x = np.clip(np.round(rng.normal(0, 3, p.n)), p.lb, p.ub)
    w = np.ones(p.m)
    cols = lm._csc(p)
    for _ in range(25):
        L = lm.activities(p, x)
        cands = lm.candidates(p, x, L, p.lb, p.ub)
        best = None
        for k, j, t in cands:
            sc = lm.score(cols, p.g, w, x, L, j, t)
            x2 = x.copy()
            x2[j] = t
            assert abs(sc - (_F(p, x, w) - _F(p, x2, w))) <= 1e-9 * (1 + abs(sc))
            assert lm.violation(L, p.g)[k] > 0 and p.lb[j] <= t <= p.ub[j] and t != x[j]
            a = dict((r, v) for r, v in cols[j])[k]
            if p.lb[j] < t < p.ub[j]:
                # the move alone satisfies its row, by the smallest integer step that does
                assert L[k] + a * (t - x[j]) <= p.g[k]
                assert L[k] + a * (t - x[j] + (1 if a > 0 else -1)) > p.g[k]
            if best is None or (-sc, j, t) < best[0]:
                best = ((-sc, j, t), j, t, sc)
        xn, wn, r = lm.search(p, p.lb, p.ub, x, w, 1)
        if best is not None and best[3] > 0:
            assert r["moves"] == 1 and xn[best[1]] == best[2] and np.array_equal(wn, w)
            assert _F(p, xn, w) < _F(p, x, w)
        else:
            viol = lm.violation(L, p.g) > 0
            assert r["moves"] == 0 and np.array_equal(wn, w + viol)
        x, w = xn, wn
    if r["violated"] == 0:
        assert (lm.activities(p, x)[np.isfinite(p.g)] <= p.g[np.isfinite(p.g)]).all()


def test_reaches_feasibility_on_planted_problems():
    found = 0
    for seed in range(10):
        p = _problem(400 + seed, m=30, n=30)
        x0 = np.clip(np.round(p.x0 + np.random.default_rng(seed).normal(0, 2, p.n)), p.lb, p.ub)
        x, w, r = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 300)
        if r["violated"] == 0:
            assert (lm.activities(p, x)[np.isfinite(p.g)] <= p.g[np.isfinite(p.g)]).all()
            found += 1
    assert found >= 5


# --- objective moves (Section 2.4: lift and breakthrough moves, the weighted objective) ---


@pytest.mark.parametrize("case", range(2))
def test_objective_hand_worked_steps(case):
    c = load_golden("local_mip_objective.json")["cases"][case]
    p = _case(c)
    for k, st in enumerate(c["steps"]):
        x, w, best, r = lm.search_objective(p, p.lb, p.ub, c["x0"], c["w0"], k + 1, obj_weight=c["obj_weight"])
        np.testing.assert_array_equal(x, st["x"])
        np.testing.assert_array_equal(w, st["w"])
        np.testing.assert_array_equal(best, st["best"])
        assert r["obj_weight"] == st["w0"]
    for key in ("moves", "bumps", "lifts", "breakthroughs", "improvements", "best_objective"):
        assert r[key] == c[key], key


@pytest.mark.parametrize("seed", range(4))
def test_zero_cost_is_the_mixed_tight_move_core(seed):
    """With c = 0 no lift or breakthrough move exists and the objective row never scores: the
    search is the mixed-tight-move core, step for step."""
    p = _problem(700 + seed)
    p.c = np.zeros(p.n)
    x0 = np.clip(np.round(np.random.default_rng(seed).normal(0, 3, p.n)), p.lb, p.ub)
    for it in (10, 40):
        ax, aw, ar = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), it)
        bx, bw, best, br = lm.search_objective(p, p.lb, p.ub, x0, np.ones(p.m), it)
        np.testing.assert_array_equal(ax, bx)
        np.testing.assert_array_equal(aw, bw)
        assert br["lifts"] == 0 and br["breakthroughs"] == 0
        assert ar["moves"] == br["moves"]
        # a bump at a feasible point raises w0 instead of a row weight
        assert ar["bumps"] + (br["obj_weight"] - 1.0) == br["bumps"]


def _feasible_start(p, rng):
    """The generator's planted point satisfies every row."""
    x = np.asarray(p.x0, dtype=np.float64)
    assert (lm.violation(lm.activities(p, x), p.g) == 0).all()
    return x


def _exact_feasible(p, x):
    A = np.zeros((p.m, p.n))
    for k in range(p.m):
        for q in range(int(p.row_ptr[k]), int(p.row_ptr[k + 1])):
            A[k, int(p.col[q])] = p.val[q]
    return bool(np.all(A @ x <= p.g)), A


@pytest.mark.parametrize("seed", range(6))
def test_lift_target_is_the_farthest_feasible_value(seed):
    """On integer data, the lift value of every variable is, by brute force over its integer
    values, the farthest one against the sign of its cost that keeps every row satisfied (all
    values in between stay feasible too, so the range is an interval)."""
    p = _problem(800 + seed, m=25, n=20)
    rng = np.random.default_rng(seed)
    p.c = rng.integers(-3, 4, p.n).astype(float)
    x = _feasible_start(p, rng)
    L = lm.activities(p, x)
    cols = lm._csc(p)
    for j in range(p.n):
        t = lm.lift_target(cols, p.g, L, x, p.lb, p.ub, p.is_int, p.c[j], j)
        if p.c[j] == 0:
            assert t is None
            continue
        sigma = -1 if p.c[j] > 0 else 1
        far = x[j]
        v = x[j] + sigma
        while p.lb[j] <= v <= p.ub[j]:
            x2 = x.copy()
            x2[j] = v
            if not _exact_feasible(p, x2)[0]:
                break
            far = v
            v += sigma
        assert (t is None and far == x[j]) or t == far, (j, t, far)


@pytest.mark.parametrize("seed", range(6))
def test_breakthrough_value_is_the_nearest_satisfying_integer(seed):
    """The objective row's tight move of an integer variable is, by brute force, the nearest
    integer value (clamped) at which D + c_j dx + delta <= 0."""
    rng = np.random.default_rng(seed)
    for _ in range(200):
        cj = float(rng.integers(1, 9)) * (1 if rng.random() < 0.5 else -1)
        xj = float(rng.integers(-5, 6))
        v0 = float(rng.integers(1, 30))
        t = lm.tight_value(xj, cj, v0, True)
        sgn = -1 if cj > 0 else 1
        d = 0
        while cj * (sgn * d) + v0 > 0:
            d += 1
        assert t == xj + sgn * d


@pytest.mark.parametrize("seed", range(5))
def test_incumbents_are_feasible_and_improve(seed):
    """Every incumbent satisfies every row exactly (integer data), its objective is the result's
    best objective, and over longer runs the incumbent's objective never rises."""
    p = _problem(900 + seed, m=30, n=25)
    rng = np.random.default_rng(seed)
    p.c = rng.integers(-4, 5, p.n).astype(float)
    x0 = np.clip(np.round(rng.normal(0, 3, p.n)), p.lb, p.ub)
    prev = np.inf
    found_any = False
    for it in (5, 20, 60, 150):
        x, w, best, r = lm.search_objective(p, p.lb, p.ub, x0, np.ones(p.m), it)
        if best is None:
            assert not r["found"]
            continue
        found_any = True
        assert _exact_feasible(p, best)[0]
        assert r["best_objective"] == float(p.c @ best)
        assert r["best_objective"] <= prev
        prev = r["best_objective"]
        assert r["moves"] + r["bumps"] == it
    assert found_any


def test_delta_reading():
    p = milp_from_dense([[1, 1]], [3], [0, 0], [4, 4], [1, 1])
    p.c = np.array([2.0, -1.0])
    assert lm.objective_delta(p) == 1.0
    p.c = np.array([2.5, -1.0])
    assert lm.objective_delta(p) == 1e-4
    p2 = milp_from_dense([[1, 1]], [3], [0, 0], [4, 4], [1, 0])
    p2.c = np.array([1.0, 1.0])
    assert lm.objective_delta(p2) == 1e-4
    p2.c = np.array([1.0, 0.0])
    assert lm.objective_delta(p2) == 1.0


# --- compensated activity updates and the periodic recompute ---


def test_kahan_add_compensates():
    """Ten additions of 0.1 give exactly 1.0 with the compensation (plain sums give
    0.9999999999999999); ten additions of 1.0 to 1e16 keep every unit (plain sums keep none)."""
    L, C = np.zeros(1), np.zeros(1)
    plain = 0.0
    for _ in range(10):
        lm.kahan_add(L, C, 0, 0.1)
        plain += 0.1
    assert L[0] == 1.0 and plain != 1.0
    L, C = np.array([1e16]), np.zeros(1)
    plain = 1e16
    for _ in range(10):
        lm.kahan_add(L, C, 0, 1.0)
        plain += 1.0
    assert L[0] == 1e16 + 10 and plain == 1e16


@pytest.mark.parametrize("seed", range(3))
def test_recompute_every_iteration_is_chained_single_steps(seed):
    """With recompute_period = 1 every iteration starts from activities summed afresh, which is
    what a chain of one-iteration searches does: the two agree step for step, on general data."""
    p = synth.random_milp(330 + seed, 60, 50, len_lo=2, len_hi=8, int_fraction=0.6, slack_scale=0.3)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -50.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 50.0)
    rng = np.random.default_rng(seed)
    x0 = np.clip(rng.normal(0, 10, p.n), p.lb, p.ub)
    x0[p.is_int == 1] = np.round(x0[p.is_int == 1])
    xa, wa, _ = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 30, recompute_period=1)
    xb, wb = x0, np.ones(p.m)
    for _ in range(30):
        xb, wb, _ = lm.search(p, p.lb, p.ub, xb, wb, 1)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(wa, wb)


def test_recompute_changes_nothing_on_integer_data():
    p = _problem(340)
    x0 = np.clip(np.round(np.random.default_rng(0).normal(0, 3, p.n)), p.lb, p.ub)
    a = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 40)
    b = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 40, recompute_period=7)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("objective", [False, True])
def test_moves_update_activities_through_the_compensated_add(objective, monkeypatch):
    """Every activity update of a move is a compensated add: one per nonzero of the moved
    variable's column, in both searches."""
    p = _problem(350)
    p.c = np.random.default_rng(1).integers(-3, 4, p.n).astype(float)
    x0 = np.clip(np.round(np.random.default_rng(2).normal(0, 3, p.n)), p.lb, p.ub)
    calls = []
    real = lm.kahan_add

    def counting(L, C, r, inc):
        calls.append(r)
        real(L, C, r, inc)

    monkeypatch.setattr(lm, "kahan_add", counting)
    cols = lm._csc(p)
    if objective:
        x, w, best, r = lm.search_objective(p, p.lb, p.ub, x0, np.ones(p.m), 40)
    else:
        x, w, r = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 40)
    assert r["moves"] > 0
    moved = np.flatnonzero(x != x0)
    assert len(calls) >= sum(len(cols[j]) for j in moved)
    assert set(calls) <= {k for j in range(p.n) for k, _ in cols[j]}


def test_equal_scores_on_one_variable_take_the_smaller_value():
    """x0 integer in [0, 10] at 10, rows x0 <= 8, x0 <= 7, -x0 <= -8: the first row proposes 8
    (drops 2 + 2), the second 7 (drops 2 + 3, then breaks the third by 1): both score 4, and
    the tie goes to the smaller value, 7."""
    p = milp_from_dense([[1.0], [1.0], [-1.0]], [8.0, 7.0, -8.0], [0.0], [10.0], [1])
    p.c = np.zeros(1)
    L = lm.activities(p, np.array([10.0]))
    cols = lm._csc(p)
    cands = lm.candidates(p, np.array([10.0]), L, p.lb, p.ub)
    assert [(k, t) for k, _, t in cands] == [(0, 8.0), (1, 7.0)]
    assert {lm.score(cols, p.g, np.ones(3), np.array([10.0]), L, 0, t) for _, _, t in cands} == {4.0}
    x, w, r = lm.search(p, p.lb, p.ub, [10.0], np.ones(3), 1)
    assert x[0] == 7.0 and r["moves"] == 1
