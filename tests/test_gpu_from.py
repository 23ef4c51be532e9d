"""bp_propagate_from (round 0 = rows of given variables) against the oracle started from the
same rows, and against the batched probing cache."""
import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.gpu_helpers import assert_bounds_match, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def rows_of(p, vars_):
    row_of = np.repeat(np.arange(p.m, dtype=np.int32), np.diff(p.row_ptr))
    return np.unique(row_of[np.isin(p.col, vars_)]).astype(np.int32)


def run_from(pkg, prob, lb, ub, vars_, **kw):
    import torch
    gl = torch.tensor(lb, device="cuda")
    gu = torch.tensor(ub, device="cuda")
    vt = torch.tensor(np.asarray(vars_, dtype=np.int32), device="cuda")
    r = prob.propagate_from(gl, gu, vt, **kw)
    return gl.cpu().numpy(), gu.cpu().numpy(), r


@pytest.mark.parametrize("seed,m,n,lo,hi,kw", [
    (21, 300, 400, 1, 30, dict()),
    (22, 200, 300, 2, 12, dict(integer_coefs=True, int_fraction=1.0)),
    (23, 120, 2000, 200, 1500, dict()),
    (24, 500, 400, 1, 60, dict(eq_fraction=0.3, inf_fraction=0.1)),
])
@pytest.mark.parametrize("nfix", [1, 7, 40])
def test_from_fixed_variables(pkg, seed, m, n, lo, hi, kw, nfix):
    """Fix some integer variables of the root fixpoint, then propagate from their rows."""
    p = synth.random_milp(seed, m, n, len_lo=lo, len_hi=hi, **kw)
    O = oracle.Problem(p)
    rl, ru, rr, _ = O.bp(p.lb, p.ub)
    if rr["status"] != 0 or rr["fragile"]:
        pytest.skip("root not a clean fixpoint")
    rng = np.random.default_rng(seed * 100 + nfix)
    free = np.flatnonzero((p.is_int == 1) & (rl < ru) & np.isfinite(rl))
    vs = rng.choice(free, size=min(nfix, len(free)), replace=False).astype(np.int32)
    lb, ub = rl.copy(), ru.copy()
    ub[vs] = lb[vs]                                   # fix at the lower bound
    ol, ou, orr, _ = O.bp(lb, ub, w0=rows_of(p, vs))
    dup = np.concatenate([vs, vs[::-1]])              # duplicates are allowed
    gl, gu, gr = run_from(pkg, pkg.Problem(p), lb, ub, dup)
    if not compare(p, gl, gu, gr, ol, ou, orr):
        pytest.skip("fragile decision in the oracle")


def test_from_matches_probe_cache(pkg):
    """One launch per branch reproduces the implied bounds the batched probe engine caches."""
    import torch
    p = synth.binary_knapsack()
    prob = pkg.Problem(p)
    O = oracle.Problem(p)
    rl, ru, rr, _ = O.bp(p.lb, p.ub)
    free = np.flatnonzero(rl < ru)[:24].astype(np.int32)
    boxes = np.stack([rl[free], rl[free], ru[free], ru[free]], axis=1)
    c = prob.probe_batch(torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda"),
                         torch.tensor(free, device="cuda"), torch.tensor(boxes, device="cuda"))
    st = c["status"].cpu().numpy()
    off = c["offsets"].cpu().numpy()
    ev, el, eu = c["var"].cpu().numpy(), c["l"].cpu().numpy(), c["u"].cpu().numpy()
    nnzu = c["nnz_updates"].cpu().numpy()
    for i, v in enumerate(free):
        for b in range(2):
            lb, ub = rl.copy(), ru.copy()
            lb[v], ub[v] = boxes[i, 2 * b], boxes[i, 2 * b + 1]
            gl, gu, gr = run_from(pkg, prob, lb, ub, [v])
            k = 2 * i + b
            assert gr["error"] == 0 and gr["status"] == st[k], (v, b, gr, st[k])
            assert gr["nnz_updates"] == nnzu[k]
            if st[k] != 0:
                continue
            chg = np.flatnonzero((gl != rl) | (gu != ru))
            ent = ev[off[k]:off[k + 1]]
            np.testing.assert_array_equal(np.sort(chg), np.sort(ent))
            o = np.argsort(ent)
            np.testing.assert_array_equal(gl[ent[o]], el[off[k]:off[k + 1]][o])
            np.testing.assert_array_equal(gu[ent[o]], eu[off[k]:off[k + 1]][o])


def test_from_empty_and_invalid(pkg):
    p = synth.random_milp(25, 100, 80, len_lo=1, len_hi=8)
    prob = pkg.Problem(p)
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub, w0=np.zeros(0, dtype=np.int32))
    gl, gu, gr = run_from(pkg, prob, p.lb, p.ub, np.zeros(0, dtype=np.int32))
    assert gr["status"] == 0 and gr["rounds"] == 0 and gr["nnz_updates"] == 0 and gr["error"] == 0
    assert_bounds_match(p, gl, gu, ol, ou)
    # an index out of range is reported, not dereferenced; the handle stays usable
    _, _, bad = run_from(pkg, prob, p.lb, p.ub, [3, p.n + 5])
    assert bad["error"] == pkg.BP_ERR_INVALID
    _, _, bad = run_from(pkg, prob, p.lb, p.ub, [-1])
    assert bad["error"] == pkg.BP_ERR_INVALID
    allv = np.arange(p.n, dtype=np.int32)
    rl, ru, rr, _ = oracle.Problem(p).bp(p.lb, p.ub, w0=rows_of(p, allv))
    gl, gu, gr = run_from(pkg, prob, p.lb, p.ub, allv)
    assert compare(p, gl, gu, gr, rl, ru, rr) or rr["fragile"]
