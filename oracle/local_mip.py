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
  step         score > 0: x_j = t and L_r += a_rj (t - x_j) for the rows of column j (ascending);
               otherwise every violated row's weight grows by 1.

Lift and breakthrough moves (objective improvement) are not part of this core.  Plain Python
loops over the rows and columns, IEEE double.
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


def search(p, lb, ub, x0, w0, iterations):
    """Runs `iterations` steps from (x0, w0).  Returns (x, w, result dict)."""
    cols = _csc(p)
    x = np.array(x0, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    L = activities(p, x)
    moves = bumps = 0
    for _ in range(int(iterations)):
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
                L[r] = L[r] + a * dx
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
