"""Oracle of the extended feasibility pump's orchestration (Section 2.5, Algorithm 2, generation
mode).

TEST INFRASTRUCTURE ONLY: called by the tests, never by the library.

The steps of Algorithm 2 in its order, each one an oracle already pinned on its own: the
approximate LP (oracle/pdhg.py), fix-and-propagate rounding (fp_oracle.c) and the local search
(oracle/local_mip.py).  The reading taken for what the paper leaves open:

  start     the LP relaxation (PDHG from zero, `lp_iterations`), rounded by fix-and-propagate,
            then the local search (`ls_iterations`, fresh weights); if no feasible point, the
            local search from the all-zero point (clamped to the bounds); the main loop starts
            from the end point with fewer violated rows (ties: the rounded one) and keeps its
            weights for the cycle breaks;
  project   min sum over integer variables of |x_j - s_j| with s_j at a bound: objective +1 for
            s_j at its lower bound, -1 at its upper bound, 0 otherwise (integer variables
            strictly inside their bounds and continuous ones take no term, so no columns are
            added), warm-started from the previous projection's primal and dual iterates;
  snap      the projection rounded to the nearest multiple of 2^-20 and clamped to the bounds,
            so that its distance is an exact sum and the rounding sees the same values on any
            implementation;
  distance  sum over integer variables of |x_j - s_j|;
  round     fix-and-propagate from the snapped projection (seed + round + 1), then the local
            search for ls_iterations // 5 iterations with fresh weights: a feasible point ends
            the pump;
  cycle     when at least N earlier distances exist and the distance improves on their mean by
            no more than `cycle_ratio` of that mean; a cycle is broken by the local search from
            the current point with the kept weights (ls_iterations), otherwise the next point is
            the snapped projection rounded to the nearest integers (ties up).
No objective cut (the improvement mode); the budget is a round count in place of a time limit.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import local_mip, pdhg

Q = 2.0 ** -20


def snap(x, lb, ub):
    """Nearest multiple of 2^-20 (ties to even), clamped to [lb, ub]."""
    return np.clip(np.rint(np.asarray(x, dtype=np.float64) / Q) * Q, lb, ub)


def projection_objective(is_int, s, lb, ub):
    c = np.zeros(len(s))
    ints = (np.asarray(is_int) != 0) & (lb < ub)
    c[ints & (s <= lb)] = 1.0
    c[ints & (s >= ub)] = -1.0
    return c


def distance(is_int, a, b):
    ints = np.asarray(is_int) != 0
    return float(np.sum(np.abs(np.asarray(a)[ints] - np.asarray(b)[ints])))


def cycle(history, d, window, ratio):
    if len(history) < window:
        return False
    mean = float(np.sum(history[-window:])) / window
    return mean - d <= ratio * mean


def nearest(is_int, x, lb, ub):
    out = np.array(x, dtype=np.float64)
    ints = np.asarray(is_int) != 0
    out[ints] = np.clip(np.floor(out[ints] + 0.5), lb[ints], ub[ints])
    return out


def run(p, lb, ub, rounds=20, lp_iterations=500, ls_iterations=200, cycle_window=3, cycle_ratio=0.1, seed=1):
    """Returns (x, result dict): status 0 when a feasible point was found (x is it), found_at
    -2 (start rounding), -1 (all-zero start), r >= 0 (round r) or -3 (none), rounds run, cycle
    breaks, the distances."""
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    P = oracle.Problem(p)
    zero = np.clip(np.zeros(p.n), lb, ub)
    x, y, _ = pdhg.solve(p, lb, ub, zero, np.zeros(p.m), iterations=lp_iterations, restart_period=100)
    xl = snap(x, lb, ub)
    s, _ = P.fix_and_propagate(xl, lb, ub, seed=seed)
    s1, w1, r1 = local_mip.search(p, lb, ub, s, np.ones(p.m), ls_iterations)
    res = {"status": 1, "found_at": -3, "rounds": 0, "cycles": 0, "distances": []}
    if r1["violated"] == 0:
        res.update(status=0, found_at=-2)
        return s1, res
    s2, w2, r2 = local_mip.search(p, lb, ub, zero, np.ones(p.m), ls_iterations)
    if r2["violated"] == 0:
        res.update(status=0, found_at=-1)
        return s2, res
    s, W = (s2, w2) if r2["violated"] < r1["violated"] else (s1, w1)
    hist = []
    for r in range(rounds):
        c = projection_objective(p.is_int, s, lb, ub)
        x, y, _ = pdhg.solve(p, lb, ub, x, y, iterations=lp_iterations, restart_period=100, c=c)
        xp = snap(x, lb, ub)
        d = distance(p.is_int, xp, s)
        cyc = cycle(hist, d, cycle_window, cycle_ratio)
        hist.append(d)
        res["rounds"] = r + 1
        sr, _ = P.fix_and_propagate(xp, lb, ub, seed=seed + r + 1)
        st, _, rt = local_mip.search(p, lb, ub, sr, np.ones(p.m), max(1, ls_iterations // 5))
        if rt["violated"] == 0:
            res.update(status=0, found_at=r, distances=hist)
            return st, res
        if cyc:
            s, W, _ = local_mip.search(p, lb, ub, s, W, ls_iterations)
            res["cycles"] += 1
        else:
            s = nearest(p.is_int, xp, lb, ub)
    res["distances"] = hist
    return s, res
