"""The local search oracle (oracle/local_mip.py: mixed tight moves, Section 2.4) against
hand-worked steps and from-scratch recomputation on random integer problems."""
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
