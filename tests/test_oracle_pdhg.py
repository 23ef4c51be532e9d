"""The approximate LP oracle (PDHG, oracle/pdhg.py) against hand-worked iterates, the LP optimum
of HiGHS (SciPy), and the fixed-point property of optimal primal-dual pairs."""
import numpy as np
import pytest

from oracle import pdhg
from paper_2510_20499_gb300 import synth
from tests.helpers import load_golden, milp_from_dense


def _case(c):
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], [0] * len(c["lb"]))
    p.c = np.array(c["c"], dtype=float)
    return p


@pytest.mark.parametrize("case", range(2))
def test_hand_worked_iterates(case):
    c = load_golden("pdhg_small.json")["cases"][case]
    p = _case(c)
    A = pdhg.matrix(p)
    x, y = np.array(c["x0"], float), np.array(c["y0"], float)
    for want_x, want_y in c["iterates"]:
        x, y = pdhg.step(A, p.c, p.g, p.lb, p.ub, x, y, c["tau"], c["sigma"])
        np.testing.assert_array_equal(x, want_x)
        np.testing.assert_array_equal(y, want_y)


def test_hand_worked_restart():
    c = load_golden("pdhg_small.json")["cases"][2]
    p = _case(c)
    # tau = sigma = 1/2: step 1/2 with primal weight 1
    x, y, r = pdhg.solve(p, p.lb, p.ub, c["x0"], c["y0"], iterations=c["iterations"], step_size=c["tau"],
                         primal_weight=1.0, restart_period=c["restart_period"])
    np.testing.assert_array_equal(x, c["final"][0])
    np.testing.assert_array_equal(y, c["final"][1])
    assert r["restarts"] == c["restarts"]


def _random_lp(seed, m, n):
    rng = np.random.default_rng(seed)
    p = synth.random_milp(seed, m, n, len_lo=2, len_hi=6, int_fraction=0.0, slack_scale=0.5)
    lb = np.where(np.isfinite(p.lb), p.lb, -10.0)
    ub = np.where(np.isfinite(p.ub), p.ub, 10.0)
    p.lb, p.ub = lb, ub
    p.c = rng.normal(0, 1, n)
    return p


def _highs(p):
    from scipy.optimize import linprog
    A = pdhg.matrix(p)
    fin = np.isfinite(p.g)
    r = linprog(p.c, A_ub=A[fin], b_ub=p.g[fin], bounds=list(zip(p.lb, p.ub)), method="highs")
    assert r.status == 0
    y = np.zeros(p.m)
    y[fin] = -r.ineqlin.marginals
    return r.x, y, r.fun


@pytest.mark.parametrize("seed", range(4))
def test_converges_to_the_lp_optimum(seed):
    pytest.importorskip("scipy")
    p = _random_lp(70 + seed, 30, 40)
    x_star, y_star, f_star = _highs(p)
    x, y, r = pdhg.solve(p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=5000, restart_period=100)
    assert abs(r["primal_obj"] - f_star) <= 1e-6 * (1 + abs(f_star)), (r, f_star)
    assert abs(r["dual_obj"] - f_star) <= 1e-6 * (1 + abs(f_star)), (r, f_star)
    assert r["primal_residual"] <= 1e-6 and r["dual_residual"] == 0.0
    np.testing.assert_allclose(p.c @ x, f_star, rtol=1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_optimal_pair_is_a_fixed_point(seed):
    pytest.importorskip("scipy")
    p = _random_lp(90 + seed, 30, 40)
    x_star, y_star, f_star = _highs(p)
    A = pdhg.matrix(p)
    eta, w = pdhg.default_step(A), pdhg.default_weight(p.c, p.g)
    x, y = pdhg.step(A, p.c, p.g, p.lb, p.ub, x_star, y_star, eta / w, eta * w)
    np.testing.assert_allclose(x, x_star, atol=1e-7)
    np.testing.assert_allclose(y, y_star, atol=1e-7)
    k = pdhg.kkt(A, p.c, p.g, p.lb, p.ub, x_star, y_star)
    assert abs(k["primal_obj"] - k["dual_obj"]) <= 1e-7 * (1 + abs(f_star))


def test_warm_start_from_the_optimum_stays():
    pytest.importorskip("scipy")
    p = _random_lp(5, 20, 25)
    x_star, y_star, f_star = _highs(p)
    x, y, r = pdhg.solve(p, p.lb, p.ub, x_star, y_star, iterations=50, restart_period=10)
    np.testing.assert_allclose(x, x_star, atol=1e-6)
    assert abs(r["primal_obj"] - f_star) <= 1e-6 * (1 + abs(f_star))


def test_default_step_bounds_the_norm():
    p = _random_lp(3, 50, 60)
    A = pdhg.matrix(p).toarray()
    assert pdhg.default_step(pdhg.matrix(p)) * np.linalg.norm(A, 2) < 1.0
