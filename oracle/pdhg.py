"""Oracle of the approximate LP: warm-started primal-dual hybrid gradient (PDHG).

TEST INFRASTRUCTURE ONLY: called by the tests and the benchmark's CPU leg, never by the library.

The paper uses a GPU PDLP as an approximate LP solver, warm-started from the previous primal and
dual solutions, for the LP relaxation and for the feasibility pump's projections (Sections 1 and
2.5; the method is that of Applegate et al., "Practical large-scale linear programming using
primal-dual hybrid gradient", NeurIPS 2021).  The paper gives no formulas; the reading taken
here is the core iteration for

    min c^T x   subject to   A x <= g,   l <= x <= u        (rows with g = +inf are free)

with duals y >= 0 of the rows, step sizes tau = eta / omega and sigma = eta * omega
(eta * ||A||_2 < 1 keeps the iteration convergent; omega is the primal weight):

    x+ = proj_[l, u](x - tau (c + A^T y))
    y+ = max(0, y + sigma (A (2 x+ - x) - g))

and, with a restart period R > 0, every R iterations the iterate is replaced by the average of
the R iterates since the previous restart (PDLP restarts to the average adaptively; a fixed
period keeps every step a plain function of the inputs).  The default step is
eta = 0.9 / sqrt(||A||_1 ||A||_inf) (largest column and row sums of |a|; their geometric mean
bounds ||A||_2), and the default primal weight PDLP's initial one, omega = ||c||_2 / ||g||_2
(finite rows; 1 when either is zero).

Preconditioning (PDLP's diagonal rescaling; `scaling_iterations` K > 0): K passes of Ruiz
equilibration, each computing the row and column maxima of the current scaled |a| (both from the
same matrix) and dividing the row factors D_r and column factors D_c by their square roots
(factor 1 where the maximum is 0).  The iteration then runs on the scaled problem
D_r A D_c, c~ = D_c c, g~ = D_r g, bounds l / D_c, u / D_c, from the scaled warm start
x0 / D_c, y0 / D_r (the default step and weight taken on the scaled data), and returns
x = D_c x~, y = D_r y~; the KKT measures are those of the original problem.

Every step is a library matrix-vector product or an elementwise numpy operation in float64, in
the order written above.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def matrix(p) -> sp.csr_matrix:
    return sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))


def default_step(A: sp.csr_matrix) -> float:
    """eta = 0.9 / sqrt(max column |a| sum * max row |a| sum)."""
    absA = abs(A)
    n1 = float(absA.sum(axis=0).max()) if A.nnz else 0.0
    ninf = float(absA.sum(axis=1).max()) if A.nnz else 0.0
    return 0.9 / np.sqrt(n1 * ninf) if n1 > 0 and ninf > 0 else 1.0


def default_weight(c, g) -> float:
    """omega = ||c||_2 / ||g||_2 over the finite rows, 1 when either norm is zero."""
    gf = g[np.isfinite(g)]
    nc, ng = float(np.linalg.norm(c)), float(np.linalg.norm(gf))
    return nc / ng if nc > 0 and ng > 0 else 1.0


def ruiz(A: sp.csr_matrix, iterations: int):
    """Row and column factors of `iterations` Ruiz passes (the scaled entries formed as
    (D_r a) D_c)."""
    m, n = A.shape
    Dr, Dc = np.ones(m), np.ones(n)
    absA = abs(A)
    for _ in range(int(iterations)):
        S = sp.diags(Dr) @ absA @ sp.diags(Dc)
        R = np.asarray(S.max(axis=1).todense()).ravel()
        C = np.asarray(S.max(axis=0).todense()).ravel()
        Dr = np.where(R > 0, Dr / np.sqrt(np.where(R > 0, R, 1.0)), Dr)
        Dc = np.where(C > 0, Dc / np.sqrt(np.where(C > 0, C, 1.0)), Dc)
    return Dr, Dc


def step(A, c, g, l, u, x, y, tau, sigma):
    """One PDHG iteration; returns (x+, y+)."""
    xn = np.clip(x - tau * (c + A.T @ y), l, u)
    xe = 2.0 * xn - x
    yn = np.maximum(0.0, y + sigma * (A @ xe - g))
    return xn, yn


def kkt(A, c, g, l, u, x, y):
    """Primal residual ||max(Ax - g, 0)||_2 over finite rows; dual residual: the reduced costs
    r = c + A^T y that push a variable toward an infinite bound (r_j > 0 with l_j = -inf, or
    r_j < 0 with u_j = +inf); primal objective c^T x; dual objective -g^T y + sum_j min over
    [l_j, u_j] of r_j x_j (finite parts only)."""
    ax = A @ x
    fin = np.isfinite(g)
    pres = float(np.linalg.norm(np.maximum(ax[fin] - g[fin], 0.0)))
    r = c + A.T @ y
    bad = np.where((r > 0) & ~np.isfinite(l), r, 0.0) + np.where((r < 0) & ~np.isfinite(u), -r, 0.0)
    dres = float(np.linalg.norm(bad))
    term = np.where(r > 0, r * np.where(np.isfinite(l), l, 0.0), r * np.where(np.isfinite(u), u, 0.0))
    dobj = float(-(g[fin] @ y[fin]) + term.sum())
    return {"primal_residual": pres, "dual_residual": dres, "primal_obj": float(c @ x), "dual_obj": dobj}


def solve(p, lb, ub, x0, y0, iterations=1000, step_size=0.0, primal_weight=0.0, restart_period=100, c=None,
          scaling_iterations=0):
    """Runs `iterations` PDHG iterations from the warm start (x0, y0), on the Ruiz-scaled problem
    when scaling_iterations > 0.  step_size 0 and primal_weight 0 take the defaults.  Returns
    (x, y, result dict)."""
    A0 = matrix(p)
    c0 = np.asarray(p.c if c is None else c, dtype=np.float64)
    g0 = np.asarray(p.g, dtype=np.float64)
    l0 = np.asarray(lb, dtype=np.float64)
    u0 = np.asarray(ub, dtype=np.float64)
    Dr, Dc = ruiz(A0, scaling_iterations)
    if scaling_iterations > 0:
        A = sp.csr_matrix(sp.diags(Dr) @ A0 @ sp.diags(Dc))
        c, g, l, u = Dc * c0, Dr * g0, l0 / Dc, u0 / Dc
        x = np.asarray(x0, dtype=np.float64) / Dc
        y = np.asarray(y0, dtype=np.float64) / Dr
    else:
        A, c, g, l, u = A0, c0, g0, l0, u0
        x = np.array(x0, dtype=np.float64)
        y = np.array(y0, dtype=np.float64)
    eta = step_size if step_size > 0 else default_step(A)
    omega = primal_weight if primal_weight > 0 else default_weight(c, g)
    tau, sigma = eta / omega, eta * omega
    xs, ys, cnt, restarts = np.zeros_like(x), np.zeros_like(y), 0, 0
    for _ in range(int(iterations)):
        x, y = step(A, c, g, l, u, x, y, tau, sigma)
        if restart_period > 0:
            xs += x
            ys += y
            cnt += 1
            if cnt == restart_period:
                x, y = xs / restart_period, ys / restart_period
                xs, ys, cnt = np.zeros_like(x), np.zeros_like(y), 0
                restarts += 1
    if scaling_iterations > 0:
        x, y = Dc * x, Dr * y
    res = kkt(A0, c0, g0, l0, u0, x, y)
    res.update(iterations=int(iterations), restarts=restarts, step=eta, primal_weight=omega)
    return x, y, res
