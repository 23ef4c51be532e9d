"""Small helpers shared by the tests (no propagation arithmetic here)."""
import itertools
import json
import os

import numpy as np

from paper_2510_20499_gb300.synth import Milp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fnum(x):
    if isinstance(x, str):
        return float(x)  # "inf", "-inf"
    return float(x)


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_problem(d, case=None):
    g = case.get("g", d["g"]) if case else d["g"]
    return Milp(d["m"], d["n"], np.array(d["row_ptr"], dtype=np.int64), np.array(d["col"], dtype=np.int32),
                np.array(d["val"], dtype=np.float64), np.array([fnum(x) for x in g]),
                np.zeros(d["n"]), np.ones(d["n"]), np.array(d["is_int"], dtype=np.uint8), np.zeros(d["n"]))


def milp_from_dense(A, g, lb, ub, is_int):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    row_ptr = [0]
    col, val = [], []
    for k in range(m):
        nz = np.flatnonzero(A[k])
        col.extend(nz.tolist())
        val.extend(A[k, nz].tolist())
        row_ptr.append(len(col))
    return Milp(m, n, np.array(row_ptr, dtype=np.int64), np.array(col, dtype=np.int32),
                np.array(val, dtype=np.float64), np.asarray(g, dtype=np.float64),
                np.asarray(lb, dtype=np.float64), np.asarray(ub, dtype=np.float64),
                np.asarray(is_int, dtype=np.uint8), np.zeros(n))


def dense(p):
    A = np.zeros((p.m, p.n))
    for k in range(p.m):
        for q in range(p.row_ptr[k], p.row_ptr[k + 1]):
            A[k, p.col[q]] = p.val[q]
    return A


def feasible_points(p, lb, ub):
    """All integer points of a tiny pure-integer problem inside [lb, ub] with A x <= g + 1e-9."""
    A = dense(p)
    doms = [np.arange(int(np.ceil(lb[j])), int(np.floor(ub[j])) + 1) for j in range(p.n)]
    if any(len(d) == 0 for d in doms):
        return np.zeros((0, p.n))
    pts = np.array(list(itertools.product(*doms)), dtype=np.float64)
    if p.m:
        ok = (pts @ A.T <= p.g[None, :] + 1e-9).all(axis=1)
        pts = pts[ok]
    return pts
