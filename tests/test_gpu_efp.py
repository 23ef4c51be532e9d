"""GPU extended feasibility pump (extended_fp, Algorithm 2) against the oracle composition
(oracle/efp.py) on integer data: the projections are snapped to a 2^-20 grid, so both sides
round the same points and every discrete decision agrees."""
import numpy as np
import pytest

from oracle import efp, local_mip
from paper_2510_20499_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


KW = dict(rounds=6, lp_iterations=200, ls_iterations=100)


@pytest.mark.parametrize("seed", range(5))
def test_matches_oracle(pkg, seed):
    import torch
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).normal(0, 1, p.n)
    ox, orr = efp.run(p, p.lb, p.ub, seed=seed + 1, **KW)
    prob = pkg.Problem(p)
    gx, gr = prob.extended_fp(torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda"), seed=seed + 1,
                              **KW)
    gx = gx.cpu().numpy()
    for k in ("status", "found_at", "rounds", "cycles"):
        assert gr[k] == orr[k], (k, gr, orr)
    if orr["distances"]:
        assert gr["last_distance"] == orr["distances"][-1]
    np.testing.assert_array_equal(gx, ox)
    if gr["status"] == 0:
        L = local_mip.activities(p, gx)
        fin = np.isfinite(p.g)
        assert (L[fin] <= p.g[fin]).all()


def test_loop_runs_somewhere():
    """At least one of the cases above runs the main loop with a cycle break (oracle side)."""
    seen = 0
    for seed in range(5):
        p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
        p.c = np.random.default_rng(seed).normal(0, 1, p.n)
        _, r = efp.run(p, p.lb, p.ub, seed=seed + 1, **KW)
        seen += r["rounds"] > 0 and r["cycles"] > 0
    assert seen >= 1


def _improve_case(pkg, seed, rounds):
    import torch
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    kw = dict(KW, rounds=rounds)
    ox, orr = efp.run(p, p.lb, p.ub, seed=seed + 1, improve=True, **kw)
    prob = pkg.Problem(p)
    gx, gr = prob.extended_fp(torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda"), seed=seed + 1,
                              improve=True, **kw)
    gx = gx.cpu().numpy()
    for k in ("status", "found_at", "rounds", "cycles", "improvements", "best_objective"):
        assert gr[k] == orr[k], (k, gr, orr)
    if orr["distances"]:
        assert gr["last_distance"] == orr["distances"][-1]
    np.testing.assert_array_equal(gx, ox)
    if gr["status"] == 0:
        L = local_mip.activities(p, gx)
        fin = np.isfinite(p.g)
        assert (L[fin] <= p.g[fin]).all()
        assert float(p.c @ gx) == gr["best_objective"]
    return orr


@pytest.mark.parametrize("seed", range(6))
def test_improvement_mode_matches_oracle(pkg, seed):
    """Improvement mode (the objective cut at each incumbent) with integral costs, so the cut's
    right-hand side is exact on both sides: the incumbents, rounds, cycle breaks and the final
    point agree; seeds 3 and 5 find no feasible point and run on the problem without a cut."""
    _improve_case(pkg, seed, 6)


def test_improvement_mode_cycle_after_cut(pkg):
    """Sixteen rounds: the cut tightens until a round fails and the loop breaks a cycle on the
    cut problem."""
    r = _improve_case(pkg, 0, 16)
    assert r["cycles"] >= 1 and r["improvements"] >= 10


def test_improvement_mode_with_zero_costs(pkg):
    """c = 0: the first feasible point is the only incumbent; the cut row is empty with
    right-hand side -1e-4, so the cut problem has no feasible point and every round fails."""
    import torch
    p = synth.knapsack_cover(seed=700, m=300, n=600, nnz=3000)
    p.c = np.zeros(p.n)
    ox, orr = efp.run(p, p.lb, p.ub, seed=1, improve=True, **KW)
    prob = pkg.Problem(p)
    gx, gr = prob.extended_fp(torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda"), seed=1,
                              improve=True, **KW)
    for k in ("status", "found_at", "rounds", "cycles", "improvements"):
        assert gr[k] == orr[k], (k, gr, orr)
    np.testing.assert_array_equal(gx.cpu().numpy(), ox)
    assert orr["improvements"] <= 1


@pytest.mark.parametrize("seed", [0, 2, 3])
def test_improvement_mode_polish_matches_oracle(pkg, seed):
    """Each incumbent polished by the local search's objective moves (integral costs): the
    incumbents, the polish count, the rounds and the point agree with the oracle (seed 3 finds
    no feasible point)."""
    import torch
    p = synth.knapsack_cover(seed=700 + seed, m=300, n=600, nnz=3000)
    p.c = np.random.default_rng(seed).integers(-5, 6, p.n).astype(float)
    ox, orr = efp.run(p, p.lb, p.ub, seed=seed + 1, improve=True, polish=True, **KW)
    prob = pkg.Problem(p)
    gx, gr = prob.extended_fp(torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda"), seed=seed + 1,
                              improve=True, polish=True, **KW)
    for k in ("status", "found_at", "rounds", "cycles", "improvements", "polished", "best_objective"):
        assert gr[k] == orr[k], (k, gr, orr)
    np.testing.assert_array_equal(gx.cpu().numpy(), ox)
