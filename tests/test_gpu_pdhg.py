"""GPU approximate LP (pdhg_solve through the C ABI) against the PDHG oracle (oracle/pdhg.py)."""
import numpy as np
import pytest

from oracle import pdhg
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


def _gpu(pkg, p, lb, ub, x0, y0, **kw):
    prob = pkg.Problem(p)
    x, y = _t(x0), _t(y0)
    r = prob.pdhg(_t(lb), _t(ub), x, y, **kw)
    return x.cpu().numpy(), y.cpu().numpy(), r


def _close(a, b, rel=1e-9):
    np.testing.assert_allclose(a, b, rtol=rel, atol=rel * max(1.0, float(np.max(np.abs(b))) if b.size else 1.0))


@pytest.mark.parametrize("case", range(2))
def test_hand_worked_iterates(pkg, case):
    c = load_golden("pdhg_small.json")["cases"][case]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], [0] * len(c["lb"]))
    p.c = np.array(c["c"], dtype=float)
    for k, (want_x, want_y) in enumerate(c["iterates"]):
        # tau = sigma = 1/2: step 1/2, primal weight 1
        x, y, r = _gpu(pkg, p, p.lb, p.ub, c["x0"], c["y0"], iterations=k + 1, restart_period=0,
                       step=c["tau"], primal_weight=1.0)
        np.testing.assert_array_equal(x, want_x)
        np.testing.assert_array_equal(y, want_y)


def test_hand_worked_restart(pkg):
    c = load_golden("pdhg_small.json")["cases"][2]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], [0])
    p.c = np.array(c["c"], dtype=float)
    x, y, r = _gpu(pkg, p, p.lb, p.ub, c["x0"], c["y0"], iterations=c["iterations"],
                   restart_period=c["restart_period"], step=c["tau"], primal_weight=1.0)
    np.testing.assert_array_equal(x, c["final"][0])
    np.testing.assert_array_equal(y, c["final"][1])
    assert r["restarts"] == c["restarts"]


def _lp(seed, m, n, nnz, max_row):
    """The mixed power-law generator at a small size (rows up to max_row nonzeros, so the long
    rows take the piece path), its infinite bounds boxed at +-1000, objective N(0, 1)."""
    p = synth.mixed_powerlaw(seed=seed, m=m, n=n, nnz=nnz, max_row=max_row)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -1000.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 1000.0)
    p.c = np.random.default_rng(seed).normal(0, 1, n)
    return p


def _compare(p, x0, y0, **kw):
    return pdhg.solve(p, p.lb, p.ub, x0, y0, **kw)


@pytest.mark.parametrize("seed,restart", [(41, 50), (42, 0), (43, 7)])
def test_matches_oracle(pkg, seed, restart):
    p = _lp(seed, 3000, 8000, 60_000, 3000)
    rng = np.random.default_rng(seed)
    x0 = np.clip(rng.normal(0, 5, p.n), p.lb, p.ub)
    y0 = np.abs(rng.normal(0, 0.01, p.m))
    kw = dict(iterations=300, restart_period=restart)
    ox, oy, orr = _compare(p, x0, y0, **kw)
    gx, gy, gr = _gpu(pkg, p, p.lb, p.ub, x0, y0, **kw)
    assert gr["restarts"] == orr["restarts"]
    assert abs(gr["step"] - orr["step"]) <= 1e-14 * orr["step"]
    assert abs(gr["primal_weight"] - orr["primal_weight"]) <= 1e-14 * orr["primal_weight"]
    _close(gx, ox)
    _close(gy, oy)
    for k in ("primal_obj", "dual_obj", "primal_residual", "dual_residual"):
        assert abs(gr[k] - orr[k]) <= 1e-8 * max(1.0, abs(orr[k])), (k, gr[k], orr[k])


def test_full_size_matches_oracle(pkg):
    """The 200k x 500k, 5M-nonzero benchmark instance (rows up to 100k nonzeros), 40
    iterations from zero with restarts every 20, against the oracle."""
    p = synth.mixed_powerlaw()
    p.lb = np.where(np.isfinite(p.lb), p.lb, -1000.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 1000.0)
    p.c = np.random.default_rng(5).normal(0, 1, p.n)
    kw = dict(iterations=40, restart_period=20)
    ox, oy, orr = _compare(p, np.zeros(p.n), np.zeros(p.m), **kw)
    gx, gy, gr = _gpu(pkg, p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), **kw)
    _close(gx, ox)
    _close(gy, oy)
    for k in ("primal_obj", "dual_obj"):
        assert abs(gr[k] - orr[k]) <= 1e-8 * max(1.0, abs(orr[k])), (k, gr[k], orr[k])


def test_warm_start_at_the_optimum(pkg):
    pytest.importorskip("scipy")
    from scipy.optimize import linprog
    p = synth.random_milp(77, 40, 60, len_lo=2, len_hi=6, int_fraction=0.0, slack_scale=0.5)
    p.lb = np.where(np.isfinite(p.lb), p.lb, -10.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 10.0)
    p.c = np.random.default_rng(1).normal(0, 1, p.n)
    A = pdhg.matrix(p)
    fin = np.isfinite(p.g)
    r = linprog(p.c, A_ub=A[fin], b_ub=p.g[fin], bounds=list(zip(p.lb, p.ub)), method="highs")
    y = np.zeros(p.m)
    y[fin] = -r.ineqlin.marginals
    gx, gy, gr = _gpu(pkg, p, p.lb, p.ub, r.x, y, iterations=50, restart_period=10)
    np.testing.assert_allclose(gx, r.x, atol=1e-6)
    assert abs(gr["primal_obj"] - r.fun) <= 1e-6 * (1 + abs(r.fun))
    assert abs(gr["dual_obj"] - r.fun) <= 1e-6 * (1 + abs(r.fun))


def test_repeatable_and_validated(pkg):
    p = _lp(44, 1000, 3000, 20_000, 800)
    x1, y1, r1 = _gpu(pkg, p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=100)
    x2, y2, r2 = _gpu(pkg, p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=100)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2) and r1 == r2
    with pytest.raises(Exception):
        _gpu(pkg, p, p.lb, p.ub, np.zeros(p.n), np.zeros(p.m), iterations=-1)


@pytest.mark.parametrize("seed,restart", [(44, 50), (45, 0)])
def test_scaled_matches_oracle(pkg, seed, restart):
    """Ruiz preconditioning (10 passes): the scaling factors are formed in the oracle's order
    with correctly rounded square roots, the iteration runs on the scaled data; x, y, the step,
    the weight and the KKT measures of the original problem agree with the oracle."""
    p = _lp(seed, 3000, 8000, 60_000, 3000)
    rng = np.random.default_rng(seed)
    x0 = np.clip(rng.normal(0, 5, p.n), p.lb, p.ub)
    y0 = np.abs(rng.normal(0, 0.01, p.m))
    kw = dict(iterations=300, restart_period=restart, scaling_iterations=10)
    ox, oy, orr = _compare(p, x0, y0, **kw)
    gx, gy, gr = _gpu(pkg, p, p.lb, p.ub, x0, y0, **kw)
    assert abs(gr["step"] - orr["step"]) <= 1e-13 * orr["step"]
    assert abs(gr["primal_weight"] - orr["primal_weight"]) <= 1e-13 * orr["primal_weight"]
    _close(gx, ox)
    _close(gy, oy)
    for k in ("primal_obj", "dual_obj", "primal_residual", "dual_residual"):
        assert abs(gr[k] - orr[k]) <= 1e-8 * max(1.0, abs(orr[k])), (k, gr[k], orr[k])
