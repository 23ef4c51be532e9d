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
The budget is a round count in place of a time limit.

Improvement mode (`improve=True`; the paper's extension of the procedure from a generation to an
improvement heuristic, a cut perpendicular to the objective at each feasible point): the reading
taken is that a feasible point (from the start or a round) becomes the incumbent x* instead of
ending the pump; the problem then carries one more row, the cut  c x <= c x* - delta  (delta as
in the local search's objective row: 1 for an integral objective on integer variables, else
1e-4), reset at each incumbent; the loop continues from x* with an empty distance history, the
LP's dual iterate extended by 0 and the kept weights by 1 for the cut row; a point satisfying
every row of the cut problem is a better incumbent.  The round budget ends the pump, which
returns the incumbent.

Polish (`polish=True`, improvement mode; the paper also uses Local-MIP to search the
neighbourhood of an integer point): each new incumbent is first searched by the local search
with its objective moves (oracle/local_mip.py `search_objective`, ls_iterations, fresh weights,
objective weight 1) on the problem without the cut; its best point replaces the incumbent when
that search recorded a later incumbent than its start (an improvement by its own exact account
D < 0, so no separately summed objective decides).
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


class _WithCut:
    """The problem with the objective cut c x <= rhs appended as its last row."""

    def __init__(self, p, rhs):
        c = np.asarray(p.c, dtype=np.float64)
        cols = np.flatnonzero(c != 0.0).astype(np.int32)
        self.m, self.n = int(p.m) + 1, int(p.n)
        self.row_ptr = np.append(np.asarray(p.row_ptr, dtype=np.int64), int(p.row_ptr[-1]) + len(cols))
        self.col = np.concatenate([np.asarray(p.col, dtype=np.int32), cols])
        self.val = np.concatenate([np.asarray(p.val, dtype=np.float64), c[cols]])
        self.g = np.append(np.asarray(p.g, dtype=np.float64), rhs)
        self.lb, self.ub, self.is_int, self.c = p.lb, p.ub, p.is_int, c

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def with_cut(p, x_best):
    """The cut problem for incumbent x_best: rhs = c x_best - delta (plain sum in index order)."""
    c = np.asarray(p.c, dtype=np.float64)
    f = 0.0
    for j in range(p.n):
        f = f + c[j] * float(x_best[j])
    return _WithCut(p, f - local_mip.objective_delta(p))


def run(p, lb, ub, rounds=20, lp_iterations=500, ls_iterations=200, cycle_window=3, cycle_ratio=0.1, seed=1,
        improve=False, polish=False):
    """Returns (x, result dict): status 0 when a feasible point was found (x is it, or the best
    one in improvement mode), found_at -2 (start rounding), -1 (all-zero start), r >= 0 (round
    r) or -3 (none) for the first feasible point, rounds run, cycle breaks, the distances, and in
    improvement mode the incumbents recorded and the best objective."""
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    P = oracle.Problem(p)
    zero = np.clip(np.zeros(p.n), lb, ub)
    x, y, _ = pdhg.solve(p, lb, ub, zero, np.zeros(p.m), iterations=lp_iterations, restart_period=100)
    xl = snap(x, lb, ub)
    s, _ = P.fix_and_propagate(xl, lb, ub, seed=seed)
    s1, w1, r1 = local_mip.search(p, lb, ub, s, np.ones(p.m), ls_iterations)
    res = {"status": 1, "found_at": -3, "rounds": 0, "cycles": 0, "distances": [], "improvements": 0,
           "best_objective": float("inf"), "incumbents": [], "polished": 0}
    best = None
    q, Q = p, P   # the problem the loop works on (with the cut once an incumbent exists)

    def incumbent(pt, where):
        nonlocal best, q, Q, y, W
        if best is None:
            res.update(status=0, found_at=where)
            y = np.append(y, 0.0)
            W = np.append(W, 1.0)
        best = np.array(pt, dtype=np.float64)
        if polish:
            _, _, xb, rr = local_mip.search_objective(p, lb, ub, best, np.ones(p.m), ls_iterations)
            if rr["improvements"] > 1:
                best = xb
                res["polished"] += 1
        res["improvements"] += 1
        res["best_objective"] = float(np.asarray(p.c, dtype=np.float64) @ best)
        res["incumbents"].append(best.copy())
        q = with_cut(p, best)
        Q = oracle.Problem(q)

    W = None
    if r1["violated"] == 0:
        if not improve:
            res.update(status=0, found_at=-2)
            return s1, res
        s, W = s1, w1
        incumbent(s1, -2)
        s = best.copy()
    else:
        s2, w2, r2 = local_mip.search(p, lb, ub, zero, np.ones(p.m), ls_iterations)
        if r2["violated"] == 0:
            if not improve:
                res.update(status=0, found_at=-1)
                return s2, res
            s, W = s2, w2
            incumbent(s2, -1)
            s = best.copy()
        else:
            s, W = (s2, w2) if r2["violated"] < r1["violated"] else (s1, w1)
    hist = []
    for r in range(rounds):
        c = projection_objective(p.is_int, s, lb, ub)
        x, y, _ = pdhg.solve(q, lb, ub, x, y, iterations=lp_iterations, restart_period=100, c=c)
        xp = snap(x, lb, ub)
        d = distance(p.is_int, xp, s)
        cyc = cycle(hist, d, cycle_window, cycle_ratio)
        hist.append(d)
        res["rounds"] = r + 1
        sr, _ = Q.fix_and_propagate(xp, lb, ub, seed=seed + r + 1)
        st, _, rt = local_mip.search(q, lb, ub, sr, np.ones(q.m), max(1, ls_iterations // 5))
        if rt["violated"] == 0:
            if not improve:
                res.update(status=0, found_at=r, distances=hist)
                return st, res
            incumbent(st, r)
            s = best.copy()
            hist = []
            continue
        if cyc:
            s, W, _ = local_mip.search(q, lb, ub, s, W, ls_iterations)
            res["cycles"] += 1
        else:
            s = nearest(p.is_int, xp, lb, ub)
    res["distances"] = hist
    return (best if best is not None else s), res
