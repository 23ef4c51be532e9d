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


# --- Ruiz preconditioning ---


def test_ruiz_closed_form():
    """diag(4, 9) is equilibrated in one pass (factors 1/2 and 1/3 on both sides); for
    [[1, 4], [2, 8]] one pass gives row factors 1/sqrt(4), 1/sqrt(8) and column factors
    1/sqrt(2), 1/sqrt(8) from the same matrix."""
    import scipy.sparse as sp
    Dr, Dc = pdhg.ruiz(sp.csr_matrix(np.diag([4.0, 9.0])), 1)
    np.testing.assert_array_equal(Dr, [0.5, 1.0 / 3.0])
    np.testing.assert_array_equal(Dc, [0.5, 1.0 / 3.0])
    Dr, Dc = pdhg.ruiz(sp.csr_matrix(np.array([[1.0, 4.0], [2.0, 8.0]])), 1)
    np.testing.assert_array_equal(Dr, [1.0 / np.sqrt(4.0), 1.0 / np.sqrt(8.0)])
    np.testing.assert_array_equal(Dc, [1.0 / np.sqrt(2.0), 1.0 / np.sqrt(8.0)])
    Dr, Dc = pdhg.ruiz(sp.csr_matrix(np.array([[0.0, 0.0], [0.0, 5.0]])), 3)   # an empty row and column
    assert Dr[0] == 1.0 and Dc[0] == 1.0


def test_ruiz_equilibrates():
    """The largest scaled |a| of every nonempty row and column approaches 1 as passes
    accumulate."""
    import scipy.sparse as sp
    p = _random_lp(11, 60, 80)
    A = pdhg.matrix(p)
    A = sp.csr_matrix(sp.diags(np.random.default_rng(0).uniform(0.01, 100, p.m)) @ A)   # badly scaled rows
    prev = np.inf
    for k in (1, 4, 16):
        Dr, Dc = pdhg.ruiz(A, k)
        S = abs(sp.diags(Dr) @ A @ sp.diags(Dc))
        R, C = S.max(axis=1).toarray().ravel(), S.max(axis=0).toarray().ravel()
        dev = max(np.abs(R[R > 0] - 1).max(), np.abs(C[C > 0] - 1).max())
        assert dev < prev
        prev = dev
    assert prev < 1e-2


def _badly_scaled_lp(seed):
    """A random LP whose rows are multiplied by factors up to 1e3 and columns by factors down to
    1e-2 (bounds and costs scaled to keep the same optimum up to the column change)."""
    p = _random_lp(seed, 30, 40)
    rng = np.random.default_rng(seed)
    rs, cs = 10 ** rng.uniform(0, 3, p.m), 10 ** rng.uniform(-2, 0, p.n)
    A = pdhg.matrix(p).toarray() * rs[:, None] * cs[None, :]
    q = milp_from_dense(A, p.g * rs, p.lb / cs, p.ub / cs, np.zeros(p.n, dtype=np.uint8))
    q.c = p.c * cs
    return q


@pytest.mark.parametrize("seed", range(3))
def test_scaled_pdhg_converges_to_the_lp_optimum(seed):
    pytest.importorskip("scipy")
    p = _badly_scaled_lp(120 + seed)
    x_star, y_star, f_star = _highs(p)
    x, y, r = pdhg.solve(p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=20000, restart_period=100,
                         scaling_iterations=10)
    assert abs(r["primal_obj"] - f_star) <= 1e-6 * (1 + abs(f_star)), (r, f_star)
    assert abs(r["dual_obj"] - f_star) <= 1e-6 * (1 + abs(f_star)), (r, f_star)
    # the same budget without scaling is further from the optimum (1-20% off on these)
    _, _, r0 = pdhg.solve(p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=20000, restart_period=100)
    assert abs(r0["primal_obj"] - f_star) + abs(r0["dual_obj"] - f_star) > \
        abs(r["primal_obj"] - f_star) + abs(r["dual_obj"] - f_star)


@pytest.mark.parametrize("seed", range(2))
def test_optimum_is_a_fixed_point_of_the_scaled_step(seed):
    """(x*/D_c, y*/D_r) is a fixed point of one step on the scaled data."""
    import scipy.sparse as sp
    pytest.importorskip("scipy")
    p = _badly_scaled_lp(140 + seed)
    x_star, y_star, f_star = _highs(p)
    A0 = pdhg.matrix(p)
    Dr, Dc = pdhg.ruiz(A0, 10)
    A = sp.csr_matrix(sp.diags(Dr) @ A0 @ sp.diags(Dc))
    c, g, l, u = Dc * p.c, Dr * p.g, p.lb / Dc, p.ub / Dc
    eta, w = pdhg.default_step(A), pdhg.default_weight(c, g)
    xs, ys = x_star / Dc, y_star / Dr
    x, y = pdhg.step(A, c, g, l, u, xs, ys, eta / w, eta * w)
    np.testing.assert_allclose(x, xs, atol=1e-6 * (1 + np.abs(xs).max()))
    np.testing.assert_allclose(y, ys, atol=1e-6 * (1 + np.abs(ys).max()))


def test_zero_scaling_passes_are_the_plain_solver():
    p = _random_lp(7, 30, 40)
    a = pdhg.solve(p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=200, restart_period=50)
    b = pdhg.solve(p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=200, restart_period=50,
                   scaling_iterations=0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("seed", range(2))
def test_scaled_warm_start_from_the_optimum_stays(seed):
    """Warm-started at HiGHS's optimal pair, the scaled iteration stays there: the warm start is
    carried into the scaled space (x*/D_c, y*/D_r, a fixed point) and back."""
    pytest.importorskip("scipy")
    p = _badly_scaled_lp(160 + seed)
    x_star, y_star, f_star = _highs(p)
    x, y, r = pdhg.solve(p, p.lb, p.ub, x_star, y_star, iterations=50, restart_period=10, scaling_iterations=10)
    np.testing.assert_allclose(x, x_star, atol=1e-6 * (1 + np.abs(x_star).max()))
    np.testing.assert_allclose(y, y_star, atol=1e-6 * (1 + np.abs(y_star).max()))
    assert abs(r["primal_obj"] - f_star) <= 1e-6 * (1 + abs(f_star))


def test_default_step_and_weight_hand_example():
    """Reading R30's defaults on a hand example: A = [[1, 2], [3, 4]] has largest column |a| sum
    6 and largest row sum 7, so eta = 0.9 / sqrt(42) = 0.138873...; c = (3, 4) and g = (12, +inf)
    give omega = ||c|| / ||g over finite rows|| = 5 / 12 (the free row takes no part)."""
    import scipy.sparse as sp
    eta = pdhg.default_step(sp.csr_matrix(np.array([[1.0, 2.0], [3.0, 4.0]])))
    assert abs(eta - 0.13887301496588270) < 1e-15
    assert pdhg.default_weight(np.array([3.0, 4.0]), np.array([12.0, np.inf])) == 5.0 / 12.0
    assert pdhg.default_weight(np.array([3.0, 4.0]), np.array([np.inf, np.inf])) == 1.0
