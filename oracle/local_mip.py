"""Oracle of the local search's move scoring (Section 2.4, GPU Local-MIP; Feasibility Jump).

TEST INFRASTRUCTURE ONLY: called by the tests, never by the library.

The paper describes its GPU Local-MIP in words (a Lagrangian-style weighted constraint violation
with penalty weights, mixed tight moves, lift and breakthrough moves, every candidate's full score
recomputed each iteration, the best selected by compaction and reduction).  The reading taken
here is the mixed-tight-move core, for A x <= g (rows with g = +inf are free), l <= x <= u:

  violation    v_k = max(0, L_k - g_k) with L_k = (A x)_k kept incrementally;
  objective    F = sum_k w_k v_k with weights w_k (1 at the first call, kept by the caller);
  candidates   for every violated row k (ascending) and every nonzero a of it (row order) on
               variable j: the value that alone makes row k satisfied,
                   t = x_j - v_k / a                 (continuous),
                   t = x_j - ceil(v_k / a)  (a > 0)  or  x_j + ceil(v_k / |a|)  (a < 0)  (integer),
               clamped to [l_j, u_j]; no candidate when t = x_j;
  score        the drop of F if x_j alone moved to t:
                   sum over the rows r of column j (ascending) of
                   w_r (v_r - max(0, L_r + a_rj (t - x_j) - g_r));
  selection    the largest score; ties: smallest variable, then smallest value;
  step         score > 0: x_j = t and L_r += a_rj (t - x_j) for the rows of column j (ascending),
               each a compensated (Kahan) sum with a per-row compensation term (the paper's
               Local-MIP keeps its row activities so); otherwise every violated row's weight
               grows by 1;
  recompute    every `recompute_period` iterations (0: never) the activities are summed afresh
               in row order and the compensation cleared, at the start of the iteration.

Lift and breakthrough moves (objective improvement) extend this core in `search_objective`
(reading at its section below).  Plain Python loops over the rows and columns, IEEE double.
"""
from __future__ import annotations

import math

import numpy as np


def _csc(p):
    """Column lists (rows ascending, with coefficients) of the CSR problem."""
    cols = [[] for _ in range(p.n)]
    for k in range(p.m):
        for q in range(int(p.row_ptr[k]), int(p.row_ptr[k + 1])):
            cols[int(p.col[q])].append((k, float(p.val[q])))
    return cols


def activities(p, x):
    """L = A x, row order (the start of the incremental activities)."""
    L = np.zeros(p.m)
    for k in range(p.m):
        s = 0.0
        for q in range(int(p.row_ptr[k]), int(p.row_ptr[k + 1])):
            s = s + float(p.val[q]) * float(x[int(p.col[q])])
        L[k] = s
    return L


def kahan_add(L, C, r, inc):
    """L[r] += inc as a compensated sum with compensation C[r] (Kahan)."""
    y = inc - C[r]
    t = L[r] + y
    C[r] = (t - L[r]) - y
    L[r] = t


def violation(L, g):
    return np.where(np.isfinite(g), np.maximum(0.0, L - g), 0.0)


def _ceil_div(e, c):
    """ceil(e / c) for e > 0, c > 0, exact when both are integers (their products are exact)."""
    d = math.ceil(e / c)
    if e == math.floor(e) and c == math.floor(c):
        while d > 1 and (d - 1) * c >= e:
            d -= 1
        while d * c < e:
            d += 1
    return float(d)


def candidates(p, x, L, lb, ub):
    """Every mixed tight move (row k, variable j, value t), in row and nonzero order."""
    g = p.g
    out = []
    for k in range(p.m):
        if not np.isfinite(g[k]):
            continue
        v = L[k] - g[k]
        if not v > 0.0:
            continue
        for q in range(int(p.row_ptr[k]), int(p.row_ptr[k + 1])):
            j, a = int(p.col[q]), float(p.val[q])
            if p.is_int[j]:
                d = _ceil_div(v, abs(a))
                t = x[j] - d if a > 0 else x[j] + d
            else:
                t = x[j] - v / a
            t = min(max(t, lb[j]), ub[j])
            if t != x[j]:
                out.append((k, j, t))
    return out


def score(cols, g, w, x, L, j, t):
    """The drop of the weighted violation if x_j alone moved to t (column rows ascending)."""
    s = 0.0
    dx = t - x[j]
    for r, a in cols[j]:
        if not np.isfinite(g[r]):
            continue
        old = max(0.0, L[r] - g[r])
        new = max(0.0, (L[r] + a * dx) - g[r])
        s = s + w[r] * (old - new)
    return s


def search(p, lb, ub, x0, w0, iterations, recompute_period=0):
    """Runs `iterations` steps from (x0, w0).  Returns (x, w, result dict)."""
    cols = _csc(p)
    x = np.array(x0, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    L = activities(p, x)
    C = np.zeros(p.m)
    moves = bumps = 0
    for it in range(int(iterations)):
        if recompute_period > 0 and it > 0 and it % recompute_period == 0:
            L = activities(p, x)
            C = np.zeros(p.m)
        best = None
        for k, j, t in candidates(p, x, L, lb, ub):
            sc = score(cols, p.g, w, x, L, j, t)
            key = (-sc, j, t)
            if best is None or key < best[0]:
                best = (key, j, t, sc)
        if best is not None and best[3] > 0.0:
            _, j, t, _ = best
            dx = t - x[j]
            for r, a in cols[j]:
                kahan_add(L, C, r, a * dx)
            x[j] = t
            moves += 1
        else:
            viol = violation(L, p.g) > 0.0
            if viol.any():
                w[viol] += 1.0
                bumps += 1
    v = violation(L, p.g)
    return x, w, {"iterations": int(iterations), "moves": moves, "bumps": bumps,
                  "violated": int((v > 0).sum()), "weighted_violation": float(w @ v),
                  "objective": float(np.asarray(p.c, dtype=np.float64) @ x)}


# ---------------------------------------------------------------------------------------------
# Objective moves (Section 2.4: Local-MIP's lift and breakthrough moves, a weighted objective).
#
# The reading taken for the moves the paper names but does not define, for min c^T x:
#
#   incumbent     at the start of an iteration, a point with no violated row whose objective is
#                 below the incumbent's (or the first such point) becomes the incumbent x*; the
#                 search keeps D = c^T x - c^T x* incrementally (D = 0 when x* is recorded, then
#                 D += c_j (t - x_j) with every move), so no absolute objective sum is needed;
#   objective row once an incumbent exists, the row  c^T x <= c^T x* - delta  joins the weighted
#                 violation with its own weight w0: its violation is v0 = max(0, D + delta);
#                 delta = 1 when every variable with a nonzero cost is integer with an integral
#                 cost (a better point is then at least 1 lower), 1e-4 otherwise;
#   lift          at a point with no violated row: for every variable with c_j != 0, the move
#                 in the direction sigma = -sign(c_j) as far as every row stays satisfied:
#                     step_r = (g_r - L_r) / |a_rj|   (continuous),  floor of it  (integer)
#                 over the rows of column j with a_rj * sigma > 0 and finite g_r, then
#                 t = x_j + sigma * min_r step_r (no such row: the bound in direction sigma),
#                 clamped to [l_j, u_j]; no move when t = x_j or t is infinite.  The largest
#                 gain -c_j (t - x_j) is applied when positive (ties: smallest variable), and
#                 ends the iteration;
#   breakthrough  while the objective row is violated: for every variable with c_j != 0
#                 (ascending), the value that alone satisfies the objective row, formed as the
#                 mixed tight move of a row with coefficients c and violation v0;
#   score         every mixed tight and breakthrough candidate: the column's weighted-violation
#                 drop (rows ascending), then plus w0 (v0 - max(0, (D + c_j dx) + delta)) when an
#                 incumbent exists; the largest score wins, ties: smallest variable, smallest
#                 value, then a mixed tight move before a breakthrough move;
#   step          a positive best score moves the variable; otherwise every violated row's
#                 weight grows by 1, or, with no violated row, w0 grows by 1.
# With c = 0 no objective move exists and the search is the mixed-tight-move core above.
# ---------------------------------------------------------------------------------------------


def objective_delta(p):
    """delta of the objective row: 1 for an integral objective on integer variables, else 1e-4."""
    c = np.asarray(p.c, dtype=np.float64)
    nz = c != 0.0
    if nz.any() and np.all(np.asarray(p.is_int)[nz] != 0) and np.all(c[nz] == np.floor(c[nz])):
        return 1.0
    return 1e-4


def _floor_div(e, c):
    """floor(e / c) for e >= 0, c > 0, exact when both are integers."""
    d = math.floor(e / c)
    if e == math.floor(e) and c == math.floor(c):
        while (d + 1) * c <= e:
            d += 1
        while d > 0 and d * c > e:
            d -= 1
    return float(d)


def lift_target(cols, g, L, x, lb, ub, is_int, cj, j):
    """The lift move's value for variable j at a point with no violated row, or None."""
    if cj == 0.0:
        return None
    sigma = -1.0 if cj > 0 else 1.0
    step = math.inf
    for r, a in cols[j]:
        if not np.isfinite(g[r]) or not a * sigma > 0:
            continue
        slack = g[r] - L[r]
        s = _floor_div(slack, abs(a)) if is_int[j] else slack / abs(a)
        step = min(step, s)
    if math.isinf(step):
        t = ub[j] if sigma > 0 else lb[j]
    else:
        t = x[j] + step if sigma > 0 else x[j] - step
        t = min(max(t, lb[j]), ub[j])
    if not math.isfinite(t) or t == x[j]:
        return None
    return t


def tight_value(xj, a, v, integer):
    """The value that alone removes violation v > 0 of a row with coefficient a on x_j."""
    if integer:
        d = _ceil_div(v, abs(a))
        return xj - d if a > 0 else xj + d
    return xj - v / a


def search_objective(p, lb, ub, x0, w0, iterations, obj_weight=1.0, recompute_period=0):
    """Local search with the objective moves, from (x0, w0, obj_weight).  Returns
    (x, w, x_best or None, result dict)."""
    cols = _csc(p)
    c = np.asarray(p.c, dtype=np.float64)
    g = p.g
    x = np.array(x0, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    delta = objective_delta(p)
    L = activities(p, x)
    C = np.zeros(p.m)
    w_obj = float(obj_weight)
    D = 0.0
    best = None
    moves = bumps = lifts = breaks = improvements = 0

    def apply(j, t):
        nonlocal D
        dx = t - x[j]
        for r, a in cols[j]:
            kahan_add(L, C, r, a * dx)
        D = D + c[j] * dx
        x[j] = t

    for it in range(int(iterations)):
        if recompute_period > 0 and it > 0 and it % recompute_period == 0:
            L[:] = activities(p, x)
            C[:] = 0.0
        nviol = int((violation(L, g) > 0.0).sum())
        if nviol == 0:
            if best is None or D < 0.0:
                best = x.copy()
                D = 0.0
                improvements += 1
            pick = None
            for j in range(p.n):
                t = lift_target(cols, g, L, x, lb, ub, p.is_int, c[j], j)
                if t is None:
                    continue
                gain = -(c[j] * (t - x[j]))
                key = (-gain, j)
                if pick is None or key < pick[0]:
                    pick = (key, j, t, gain)
            if pick is not None and pick[3] > 0.0:
                apply(pick[1], pick[2])
                moves += 1
                lifts += 1
                continue
        cands = [(j, t, 0) for _, j, t in candidates(p, x, L, lb, ub)]
        has_best = best is not None
        v0 = D + delta
        if has_best and v0 > 0.0:
            for j in range(p.n):
                if c[j] == 0.0:
                    continue
                t = min(max(tight_value(x[j], c[j], v0, p.is_int[j]), lb[j]), ub[j])
                if t != x[j]:
                    cands.append((j, t, 1))
        pick = None
        for j, t, kind in cands:
            sc = score(cols, g, w, x, L, j, t)
            if has_best:
                dx = t - x[j]
                ov0 = max(0.0, D + delta)
                nv0 = max(0.0, (D + c[j] * dx) + delta)
                sc = sc + w_obj * (ov0 - nv0)
            key = (-sc, j, t, kind)
            if pick is None or key < pick[0]:
                pick = (key, j, t, sc, kind)
        if pick is not None and pick[3] > 0.0:
            apply(pick[1], pick[2])
            moves += 1
            breaks += pick[4]
        else:
            viol = violation(L, g) > 0.0
            if viol.any():
                w[viol] += 1.0
                bumps += 1
            elif has_best:
                w_obj += 1.0
                bumps += 1
    v = violation(L, g)
    res = {"iterations": int(iterations), "moves": moves, "bumps": bumps, "lifts": lifts,
           "breakthroughs": breaks, "improvements": improvements, "found": best is not None,
           "violated": int((v > 0).sum()), "weighted_violation": float(w @ v),
           "objective": float(c @ x), "best_objective": float(c @ best) if best is not None else math.inf,
           "obj_weight": w_obj, "delta": delta}
    return x, w, best, res
