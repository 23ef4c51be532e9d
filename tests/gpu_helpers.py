"""Comparison of GPU propagation results with the oracle (used by the gpu tests)."""
import numpy as np

import oracle

REL_CONT = 1e-9   # continuous bounds: relative agreement required with the oracle


def run_gpu(prob, lb, ub, **kw):
    import torch
    gl = torch.tensor(np.asarray(lb, dtype=np.float64), device="cuda")
    gu = torch.tensor(np.asarray(ub, dtype=np.float64), device="cuda")
    r = prob.propagate(gl, gu, **kw)
    return gl.cpu().numpy(), gu.cpu().numpy(), r


def assert_bounds_match(p, gl, gu, ol, ou):
    ints = p.is_int == 1
    np.testing.assert_array_equal(gl[ints], ol[ints], err_msg="integer lower bounds")
    np.testing.assert_array_equal(gu[ints], ou[ints], err_msg="integer upper bounds")
    for g, o, what in ((gl, ol, "lower"), (gu, ou, "upper")):
        c = ~ints
        inf = ~np.isfinite(o[c])
        np.testing.assert_array_equal(g[c][inf], o[c][inf], err_msg=f"infinite continuous {what} bounds")
        fin = ~inf
        d = np.abs(g[c][fin] - o[c][fin])
        tol = REL_CONT * np.maximum(1.0, np.abs(o[c][fin]))
        bad = np.flatnonzero(d > tol)
        assert len(bad) == 0, f"continuous {what} bounds differ beyond 1e-9 rel at {len(bad)} vars, max {d.max()}"


def compare(p, gl, gu, gr, ol, ou, orr, exact_counts=True, planted=None):
    """The GPU must match the oracle: status, rounds, work count, first infeasible indices
    and integer bounds exactly, continuous bounds within 1e-9 relative.  When the oracle saw a
    fragile decision (one that summation order may flip) the two may legitimately differ: the
    function then returns False (the caller skips the exact comparison), after checking what
    still holds, if the caller gives `planted`, a point satisfying every row inside the start
    bounds: propagation never cuts off a feasible point, so the GPU must not report
    infeasibility and its bounds must contain the point (integers exactly, continuous values
    within 1e-6 relative)."""
    assert gr["error"] == 0, gr
    if orr["fragile"]:
        if planted is not None:
            assert gr["status"] != oracle.INFEASIBLE, gr
            ints = p.is_int == 1
            slack = np.where(ints, 0.0, 1e-6 * np.maximum(1.0, np.abs(planted)))
            assert (gl <= planted + slack).all() and (gu >= planted - slack).all()
        return False
    for key in ("status", "rounds", "first_infeasible_row", "first_infeasible_var"):
        assert gr[key] == orr[key], (key, gr[key], orr[key])
    if exact_counts:
        assert gr["nnz_updates"] == orr["nnz_updates"], (gr["nnz_updates"], orr["nnz_updates"])
        assert gr["n_changed"] == orr["n_changed"], (gr["n_changed"], orr["n_changed"])
    assert_bounds_match(p, gl, gu, ol, ou)
    return True


def verified_feasible(p, P, xo):
    """The oracle's verdict on a FEASIBLE result: integer values integral, propagation from the
    original bounds with the integer variables fixed not infeasible, and (with SciPy) a
    continuous completion within 1e-6 of every row (HiGHS on the remaining linear system)."""
    ints = p.is_int == 1
    if not (xo[ints] == np.round(xo[ints])).all():
        return False
    lo, hi = p.lb.copy(), p.ub.copy()
    lo[ints] = hi[ints] = xo[ints]
    _, _, rb, _ = P.bp(lo, hi)
    if rb["status"] == oracle.INFEASIBLE:
        return False
    try:
        import scipy.sparse as sp
        from scipy.optimize import linprog
    except ImportError:
        return True
    A = sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))
    cont = np.flatnonzero(~ints)
    rhs = p.g - A[:, np.flatnonzero(ints)] @ xo[ints] + 1e-6
    r = linprog(np.zeros(len(cont)), A_ub=A[:, cont], b_ub=rhs, bounds=list(zip(p.lb[cont], p.ub[cont])),
                method="highs")
    return r.status == 0
