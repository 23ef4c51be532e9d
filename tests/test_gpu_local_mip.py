"""GPU local search move scoring (local_search_mtm and local_search_objective through the C ABI)
against the oracle (oracle/local_mip.py).  Both sides apply the same operations in the same order, so points,
weights and counts must agree bit for bit."""
import numpy as np
import pytest

from oracle import local_mip as lm
from paper_2510_20499_gb300 import synth
from tests.helpers import load_golden, milp_from_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def _t(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def _gpu(pkg, p, x0, w0, iterations):
    prob = pkg.Problem(p)
    x, w = _t(x0), _t(w0)
    r = prob.local_search(_t(p.lb), _t(p.ub), x, w, iterations=iterations)
    return x.cpu().numpy(), w.cpu().numpy(), r


def _same(p, x0, w0, iterations, pkg):
    ox, ow, orr = lm.search(p, p.lb, p.ub, x0, w0, iterations)
    gx, gw, gr = _gpu(pkg, p, x0, w0, iterations)
    np.testing.assert_array_equal(gx, ox)
    np.testing.assert_array_equal(gw, ow)
    for k in ("moves", "bumps", "violated"):
        assert gr[k] == orr[k], (k, gr, orr)
    assert abs(gr["weighted_violation"] - orr["weighted_violation"]) <= 1e-9 * max(1.0, orr["weighted_violation"])
    return orr


@pytest.mark.parametrize("case", range(2))
def test_hand_worked_steps(pkg, case):
    c = load_golden("local_mip_small.json")["cases"][case]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], c["is_int"])
    p.c = np.array(c["c"], dtype=float)
    for k, (want_x, want_w) in enumerate(c["steps"]):
        x, w, r = _gpu(pkg, p, c["x0"], c["w0"], k + 1)
        np.testing.assert_array_equal(x, want_x)
        np.testing.assert_array_equal(w, want_w)
    assert r["moves"] == c["moves"] and r["bumps"] == c["bumps"]


def _integer_problem(seed, m, n):
    p = synth.random_milp(seed, m, n, len_lo=2, len_hi=8, int_fraction=1.0, slack_scale=0.3, integer_coefs=True)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -5.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 5.0)
    return p


@pytest.mark.parametrize("seed", range(5))
def test_matches_oracle_integer_data(pkg, seed):
    p = _integer_problem(500 + seed, 300, 250)
    x0 = np.clip(np.round(np.random.default_rng(seed).normal(0, 3, p.n)), p.lb, p.ub)
    r = _same(p, x0, np.ones(p.m), 60, pkg)
    assert r["moves"] > 0


@pytest.mark.parametrize("seed", range(3))
def test_matches_oracle_general_data(pkg, seed):
    """Non-integer coefficients and continuous variables: the same operation order on both sides
    still gives identical results."""
    p = synth.random_milp(600 + seed, 200, 180, len_lo=2, len_hi=8, int_fraction=0.6, slack_scale=0.3)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -50.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 50.0)
    rng = np.random.default_rng(seed)
    x0 = np.clip(rng.normal(0, 10, p.n), p.lb, p.ub)
    x0[p.is_int == 1] = np.round(x0[p.is_int == 1])
    _same(p, x0, np.ones(p.m), 40, pkg)


def test_matches_oracle_knapsack_cover(pkg):
    """A 2k x 4k, 40k-nonzero knapsack/cover instance from a random 0/1 point, 80 iterations."""
    p = synth.knapsack_cover(seed=91, m=2000, n=4000, nnz=40_000)
    x0 = (np.random.default_rng(3).random(p.n) < 0.5).astype(float)
    x0 = np.clip(x0, p.lb, p.ub)
    r = _same(p, x0, np.ones(p.m), 80, pkg)
    assert r["moves"] > 0


def test_repeatable(pkg):
    p = _integer_problem(77, 400, 300)
    x0 = np.clip(np.round(np.random.default_rng(0).normal(0, 3, p.n)), p.lb, p.ub)
    a = _gpu(pkg, p, x0, np.ones(p.m), 50)
    b = _gpu(pkg, p, x0, np.ones(p.m), 50)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


# --- objective moves (local_search_objective) ---


def _gpu_obj(pkg, p, x0, w0, iterations, obj_weight=1.0):
    import torch
    prob = pkg.Problem(p)
    x, w = _t(x0), _t(w0)
    xb = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
    r = prob.local_search_objective(_t(p.lb), _t(p.ub), x, w, xb, iterations=iterations, obj_weight=obj_weight)
    return x.cpu().numpy(), w.cpu().numpy(), xb.cpu().numpy(), r


def _same_obj(p, x0, w0, iterations, pkg):
    ox, ow, ob, orr = lm.search_objective(p, p.lb, p.ub, x0, w0, iterations)
    gx, gw, gb, gr = _gpu_obj(pkg, p, x0, w0, iterations)
    np.testing.assert_array_equal(gx, ox)
    np.testing.assert_array_equal(gw, ow)
    for k in ("moves", "bumps", "violated", "lifts", "breakthroughs", "improvements", "found", "obj_weight", "delta"):
        assert gr[k] == orr[k], (k, gr, orr)
    if orr["found"]:
        np.testing.assert_array_equal(gb, ob)
        assert abs(gr["best_objective"] - orr["best_objective"]) <= 1e-9 * max(1.0, abs(orr["best_objective"]))
    else:
        assert np.isnan(gb).all() and gr["best_objective"] == np.inf
    assert abs(gr["weighted_violation"] - orr["weighted_violation"]) <= 1e-9 * max(1.0, orr["weighted_violation"])
    return orr


@pytest.mark.parametrize("case", range(2))
def test_objective_hand_worked_steps(pkg, case):
    c = load_golden("local_mip_objective.json")["cases"][case]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], c["is_int"])
    p.c = np.array(c["c"], dtype=float)
    for k, st in enumerate(c["steps"]):
        x, w, xb, r = _gpu_obj(pkg, p, c["x0"], c["w0"], k + 1, obj_weight=c["obj_weight"])
        np.testing.assert_array_equal(x, st["x"])
        np.testing.assert_array_equal(w, st["w"])
        np.testing.assert_array_equal(xb, st["best"])
        assert r["obj_weight"] == st["w0"]
    for key in ("moves", "bumps", "lifts", "breakthroughs", "improvements", "best_objective"):
        assert r[key] == c[key], key


@pytest.mark.parametrize("seed", range(5))
def test_objective_matches_oracle_integer_data(pkg, seed):
    """Integer data and integral costs (delta = 1), started from the planted feasible point:
    lift moves first, then breakthrough moves, row and objective weight bumps."""
    p = _integer_problem(520 + seed, 80, 60)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    r = _same_obj(p, np.asarray(p.x0, dtype=float), np.ones(p.m), 300, pkg)
    assert r["lifts"] > 0 and r["improvements"] > 0 and r["breakthroughs"] > 0


@pytest.mark.parametrize("seed", range(3))
def test_objective_matches_oracle_many_blocks(pkg, seed):
    """2,500 variables (ten blocks of the per-variable passes), 3,000 rows, 40 nonzero costs
    spread over the variables: the lifts run out early and the breakthrough phase follows."""
    p = _integer_problem(580 + seed, 3000, 2500)
    rng = np.random.default_rng(seed)
    c = np.zeros(p.n)
    pick = rng.choice(p.n, 40, replace=False)
    c[pick] = rng.integers(1, 6, 40) * rng.choice([-1, 1], 40)
    p.c = c
    r = _same_obj(p, np.asarray(p.x0, dtype=float), np.ones(p.m), 300, pkg)
    assert r["lifts"] > 0 and r["breakthroughs"] > 0 and r["obj_weight"] > 1.0


@pytest.mark.parametrize("seed", range(3))
def test_objective_matches_oracle_from_infeasible_point(pkg, seed):
    p = _integer_problem(540 + seed, 300, 250)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    x0 = np.clip(np.round(np.random.default_rng(seed).normal(0, 3, p.n)), p.lb, p.ub)
    _same_obj(p, x0, np.ones(p.m), 120, pkg)


@pytest.mark.parametrize("seed", range(3))
def test_objective_matches_oracle_general_data(pkg, seed):
    """Non-integer coefficients and costs, continuous variables (delta = 1e-4): the same
    operation order on both sides still gives identical results."""
    p = synth.random_milp(620 + seed, 60, 50, len_lo=2, len_hi=8, int_fraction=0.6, slack_scale=0.3)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -50.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 50.0)
    r = _same_obj(p, np.clip(np.asarray(p.x0, dtype=float), p.lb, p.ub), np.ones(p.m), 300, pkg)
    assert r["delta"] == 1e-4 and r["lifts"] > 0


@pytest.mark.parametrize("seed", range(2))
def test_objective_zero_cost_is_local_search_mtm(pkg, seed):
    p = _integer_problem(560 + seed, 300, 250)
    p.c = np.zeros(p.n)
    x0 = np.clip(np.round(np.random.default_rng(seed).normal(0, 3, p.n)), p.lb, p.ub)
    ax, aw, ar = _gpu(pkg, p, x0, np.ones(p.m), 60)
    bx, bw, _, br = _gpu_obj(pkg, p, x0, np.ones(p.m), 60)
    np.testing.assert_array_equal(ax, bx)
    np.testing.assert_array_equal(aw, bw)
    assert ar["moves"] == br["moves"] and br["lifts"] == 0 and br["breakthroughs"] == 0


def test_objective_rejects_bad_weight(pkg):
    import torch
    p = _integer_problem(77, 40, 30)
    prob = pkg.Problem(p)
    x, w = _t(p.x0), _t(np.ones(p.m))
    xb = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        prob.local_search_objective(_t(p.lb), _t(p.ub), x, w, xb, iterations=5, obj_weight=-1.0)


def _with_dense_row(p, seed):
    """p plus one row over every variable (coefficients 1..3), its right-hand side 30% below the
    row's value at the planted point, so that the row is violated there."""
    rng = np.random.default_rng(seed)
    a = rng.integers(1, 4, p.n).astype(float)
    x0 = np.asarray(p.x0, dtype=float)
    rp = np.append(np.asarray(p.row_ptr, dtype=np.int64), int(p.row_ptr[-1]) + p.n)
    col = np.concatenate([np.asarray(p.col, dtype=np.int32), np.arange(p.n, dtype=np.int32)])
    val = np.concatenate([np.asarray(p.val, dtype=float), a])
    g = np.append(p.g, np.floor(0.7 * float(a @ x0)))
    return synth.Milp(p.m + 1, p.n, rp, col, val, g, p.lb, p.ub, p.is_int, p.c, x0=x0, name=p.name + "_dense")


def test_matches_oracle_with_a_dense_row(pkg):
    """A row over all 12,000 variables: every move's distance-2 neighbourhood holds more entries
    than the grid has warps (a thread per entry), and the dense row's cached candidates are
    scanned and recomputed by the whole grid."""
    p = _with_dense_row(_integer_problem(590, 2000, 12000), 590)
    r = _same(p, np.asarray(p.x0, dtype=float), np.ones(p.m), 25, pkg)
    assert r["moves"] > 0


# --- edge cases ---


def test_zero_iterations_leave_the_point(pkg):
    p = _integer_problem(71, 200, 150)
    x0 = np.clip(np.round(np.random.default_rng(1).normal(0, 3, p.n)), p.lb, p.ub)
    gx, gw, gr = _gpu(pkg, p, x0, np.ones(p.m), 0)
    _, _, orr = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 0)
    np.testing.assert_array_equal(gx, x0)
    np.testing.assert_array_equal(gw, np.ones(p.m))
    assert gr["moves"] == 0 and gr["bumps"] == 0 and gr["violated"] == orr["violated"]
    ox, ow, ob, ro = lm.search_objective(p, p.lb, p.ub, x0, np.ones(p.m), 0)
    bx, bw, bb, br = _gpu_obj(pkg, p, x0, np.ones(p.m), 0)
    np.testing.assert_array_equal(bx, x0)
    assert not br["found"] and np.isnan(bb).all() and br["improvements"] == ro["improvements"] == 0


def test_feasible_start_does_not_move(pkg):
    """At a point with no violated row there is no candidate and no weight to raise."""
    p = _integer_problem(72, 200, 150)
    x0 = np.asarray(p.x0, dtype=float)
    gx, gw, gr = _gpu(pkg, p, x0, np.ones(p.m), 25)
    np.testing.assert_array_equal(gx, x0)
    np.testing.assert_array_equal(gw, np.ones(p.m))
    assert gr["moves"] == 0 and gr["bumps"] == 0 and gr["violated"] == 0


# --- compensated activities with a periodic recompute ---


@pytest.mark.parametrize("seed", range(2))
def test_recompute_period_matches_oracle(pkg, seed):
    """General data (the compensation terms are nonzero) with the activities summed afresh
    every 7 iterations: points, weights and counts agree with the oracle bit for bit."""
    p = synth.random_milp(640 + seed, 200, 180, len_lo=2, len_hi=8, int_fraction=0.6, slack_scale=0.3)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -50.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 50.0)
    rng = np.random.default_rng(seed)
    x0 = np.clip(rng.normal(0, 10, p.n), p.lb, p.ub)
    x0[p.is_int == 1] = np.round(x0[p.is_int == 1])
    ox, ow, orr = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 50, recompute_period=7)
    prob = pkg.Problem(p)
    x, w = _t(x0), _t(np.ones(p.m))
    gr = prob.local_search(_t(p.lb), _t(p.ub), x, w, iterations=50, recompute_period=7)
    np.testing.assert_array_equal(x.cpu().numpy(), ox)
    np.testing.assert_array_equal(w.cpu().numpy(), ow)
    assert gr["moves"] == orr["moves"] and gr["bumps"] == orr["bumps"]


@pytest.mark.parametrize("seed", range(2))
def test_objective_recompute_period_matches_oracle(pkg, seed):
    import torch
    p = synth.random_milp(660 + seed, 60, 50, len_lo=2, len_hi=8, int_fraction=0.6, slack_scale=0.3)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -50.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 50.0)
    x0 = np.clip(np.asarray(p.x0, dtype=float), p.lb, p.ub)
    ox, ow, ob, orr = lm.search_objective(p, p.lb, p.ub, x0, np.ones(p.m), 200, recompute_period=13)
    prob = pkg.Problem(p)
    x, w = _t(x0), _t(np.ones(p.m))
    xb = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
    gr = prob.local_search_objective(_t(p.lb), _t(p.ub), x, w, xb, iterations=200, recompute_period=13)
    np.testing.assert_array_equal(x.cpu().numpy(), ox)
    np.testing.assert_array_equal(w.cpu().numpy(), ow)
    for k in ("moves", "bumps", "lifts", "breakthroughs", "improvements", "obj_weight"):
        assert gr[k] == orr[k], (k, gr, orr)
    if orr["found"]:
        np.testing.assert_array_equal(xb.cpu().numpy(), ob)
