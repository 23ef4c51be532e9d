"""Pins of the oracle's probing (Section 2.2): probe split, cache contents, brute-force
soundness of cached implications, and the probe priority keys."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.helpers import dense, feasible_points, golden_problem, load_golden, milp_from_dense


def test_probe_split_cases():
    assert oracle.probe_split(1, 0, 1) == (0, 0, 1, 1)
    assert oracle.probe_split(1, 0, 100) == (0, 49, 50, 100)    # x < 50 | x >= 50
    assert oracle.probe_split(1, 0, 3) == (0, 1, 2, 3)          # x < 1.5 | x >= 1.5
    assert oracle.probe_split(1, -3, 2) == (-3, -1, 0, 2)       # (l+u)/2 = -0.5
    assert oracle.probe_split(1, 4, np.inf) == (4, 4, 5, np.inf)
    assert oracle.probe_split(1, -np.inf, 7) == (7, 7, -np.inf, 6)
    assert oracle.probe_split(0, 0, 1) is None                   # continuous
    assert oracle.probe_split(1, 2, 2) is None                   # fixed
    assert oracle.probe_split(1, -np.inf, np.inf) is None        # free


def test_probe_cache_golden():
    d = load_golden("probe_knapsack.json")
    p = golden_problem(d)
    P = oracle.Problem(p)
    res = P.probe_batch(np.array(d["root_lb"], float), np.array(d["root_ub"], float), d["var"], d["boxes"])
    for e, want in enumerate(d["expect"]):
        assert res["status"][e] == want["status"], want["note"]
        a, b = res["offsets"][e], res["offsets"][e + 1]
        got = [[int(res["var"][q]), float(res["l"][q]), float(res["u"][q])] for q in range(a, b)]
        assert got == [[int(x[0]), float(x[1]), float(x[2])] for x in want["entries"]], want["note"]


@pytest.mark.parametrize("seed", range(15))
def test_probe_brute_force(seed):
    """A branch marked infeasible has no feasible point; every cached bound holds for every
    feasible point of its branch; a branch's cache equals the plain propagation of root ∩ box
    whose first round holds the rows of the probed variable."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 7))
    m = int(rng.integers(2, 6))
    A = rng.integers(-3, 4, size=(m, n)).astype(float)
    A[rng.uniform(size=(m, n)) < 0.35] = 0.0
    for k in range(m):
        if not A[k].any():
            A[k, rng.integers(0, n)] = 1.0
    ub = rng.integers(1, 4, size=n).astype(float)
    lb = np.zeros(n)
    g = rng.integers(0, 7, size=m).astype(float)
    p = milp_from_dense(A, g, lb, ub, np.ones(n))
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(lb, ub)
    if r["status"] != oracle.FIXPOINT:
        return
    var, boxes = [], []
    for j in range(n):
        s = oracle.probe_split(1, rl[j], ru[j])
        if s:
            var.append(j)
            boxes.append(s)
    if not var:
        return
    res = P.probe_batch(rl, ru, var, boxes)
    pts = feasible_points(p, rl, ru)
    for i, v in enumerate(var):
        for b in range(2):
            e = 2 * i + b
            lo, hi = boxes[i][2 * b], boxes[i][2 * b + 1]
            inb = pts[(pts[:, v] >= lo) & (pts[:, v] <= hi)] if len(pts) else pts
            if res["status"][e] == oracle.INFEASIBLE:
                assert len(inb) == 0
                continue
            l2, u2 = rl.copy(), ru.copy()
            for q in range(res["offsets"][e], res["offsets"][e + 1]):
                l2[res["var"][q]] = res["l"][q]
                u2[res["var"][q]] = res["u"][q]
            if len(inb):
                assert (inb >= l2).all() and (inb <= u2).all()
            # composition: the same as one propagation from root ∩ box, round 0 = rows of v
            sl, su = rl.copy(), ru.copy()
            sl[v], su[v] = max(sl[v], lo), min(su[v], hi)
            rows_v = [k for k in range(m) if A[k, v] != 0]
            cl, cu, cr, _ = P.bp(sl, su, w0=rows_v)
            np.testing.assert_array_equal(cl, l2)
            np.testing.assert_array_equal(cu, u2)
            assert cr["rounds"] == res["rounds"][e]


def test_priority_golden():
    d = load_golden("priority_small.json")
    p = golden_problem(d)
    P = oracle.Problem(p)
    k1, k2, k3 = P.probe_priority(np.array(d["lb"], float), np.array(d["ub"], float))
    np.testing.assert_array_equal(k1, d["key1"])
    np.testing.assert_array_equal(k2, d["key2"])
    np.testing.assert_array_equal(k3, d["key3"])
    np.testing.assert_array_equal(oracle.priority_order(k1, k2, k3), d["order"])


@pytest.mark.parametrize("seed", range(10))
def test_priority_flip_counts_by_enumeration(seed):
    """key1 counts the rows whose smallest activity over the box, with the variable pinned to
    the bound that maximises its own term, exceeds g + tol; key3 is the smallest
    (g - min activity) / |a|.  The minima come from enumerating the box's integer points."""
    rng = np.random.default_rng(200 + seed)
    n, m = 5, 4
    A = rng.integers(-4, 5, size=(m, n)).astype(float)
    A[rng.uniform(size=(m, n)) < 0.3] = 0.0
    lb = np.zeros(n)
    ub = rng.integers(1, 3, size=n).astype(float)
    g = rng.integers(-2, 6, size=m).astype(float)
    p = milp_from_dense(A, g, lb, ub, np.ones(n))
    k1, k2, k3 = oracle.Problem(p).probe_priority(lb, ub)
    pts = np.array(list(itertools.product(*[np.arange(0, int(u) + 1) for u in ub])), dtype=float)
    act = pts @ A.T
    for j in range(n):
        rows = [k for k in range(m) if A[k, j] != 0]
        mixed = any(A[k, j] > 0 for k in rows) and any(A[k, j] < 0 for k in rows)
        cnt, exc, unit = 0, 0.0, np.inf
        for k in rows:
            lmin = act[:, k].min()
            unit = min(unit, (g[k] - lmin) / abs(A[k, j]))
            if mixed:
                pin = ub[j] if A[k, j] > 0 else lb[j]
                fl = act[pts[:, j] == pin, k].min()
                if fl > g[k] + 1e-6:
                    cnt += 1
                    exc = max(exc, fl - g[k])
        if not rows:
            unit = np.inf
        assert k1[j] == cnt
        assert k2[j] == exc
        assert k3[j] == unit


def test_priority_order_on_probing_instance():
    p = synth.knapsack_cover(seed=5, m=500, n=1000, nnz=10_000)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    assert r["status"] == oracle.FIXPOINT
    k1, k2, k3 = P.probe_priority(rl, ru)
    order = oracle.priority_order(k1, k2, k3)
    assert len(order) == int(((k1 >= 0)).sum())
    keys = [(-k1[j], -k2[j], k3[j], j) for j in order]
    assert keys == sorted(keys)



def _apply_case(c):
    p = milp_from_dense(np.array(c["A"], float), c["g"], np.array(c["lb"], float), np.array(c["ub"], float),
                        np.array(c["is_int"]))
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    var = np.array(c["probe"], dtype=np.int32)
    boxes = np.array([oracle.probe_split(p.is_int[j], rl[j], ru[j]) for j in var], dtype=float).reshape(-1, 4)
    return p, P, rl, ru, P.probe_batch(rl, ru, var, boxes)


@pytest.mark.parametrize("case", range(4))
def test_probe_cache_apply_golden(case):
    """Hand-worked global bounds from the probing cache (Section 2.2): a branch proven
    infeasible fixes its variable, an implication of both branches holds everywhere, two
    infeasible branches prove the problem infeasible."""
    c = load_golden("probe_apply.json")["cases"][case]
    p, P, rl, ru, cache = _apply_case(c)
    l, u, r = P.probe_cache_apply(rl, ru, cache)
    for k in ("status", "first_infeasible_pair", "first_infeasible_var", "fixed_pairs"):
        assert r[k] == c[k], (k, r, c["note"])
    if "out_lb" in c:
        np.testing.assert_array_equal(l, c["out_lb"])
        np.testing.assert_array_equal(u, c["out_ub"])
        assert r["tightened"] == c["tightened"]


@pytest.mark.parametrize("seed", range(40))
def test_probe_cache_apply_brute_force(seed):
    """Tiny general-integer problems: every integer point satisfying all rows lies inside the
    bounds derived from the cache of every probeable variable, and INFEASIBLE is reported only
    when there is no such point; the derived bounds never loosen the root's."""
    rng = np.random.default_rng(500 + seed)
    n, m = int(rng.integers(3, 7)), int(rng.integers(2, 6))
    A = rng.integers(-4, 5, size=(m, n)).astype(float)
    A[rng.uniform(size=(m, n)) < 0.3] = 0.0
    for k in range(m):
        if not A[k].any():
            A[k, rng.integers(0, n)] = 1.0
    ub = rng.integers(1, 4, size=n).astype(float)
    g = rng.integers(-3, 8, size=m).astype(float)
    p = milp_from_dense(A, g, np.zeros(n), ub, np.ones(n))
    P = oracle.Problem(p)
    rl, ru, r0, _ = P.bp(p.lb, p.ub)
    if r0["status"] == oracle.INFEASIBLE:
        return
    var = np.array([j for j in range(n) if rl[j] < ru[j]], dtype=np.int32)
    if len(var) == 0:
        return
    boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=float).reshape(-1, 4)
    cache = P.probe_batch(rl, ru, var, boxes)
    l, u, r = P.probe_cache_apply(rl, ru, cache)
    assert (l >= rl).all() and (u <= ru).all()
    pts = feasible_points(p, p.lb, p.ub)
    if r["status"] == oracle.INFEASIBLE:
        assert len(pts) == 0
    else:
        assert ((pts >= l) & (pts <= u)).all()


def test_priority_flip_uses_the_tolerance():
    """Key 1 counts rows whose flipped activity L_min + |a| (u - l) exceeds g + 1e-6 (reading
    R11 with Section 3's tolerance): x0 in {0, 1} with rows x0 <= 1 - 5e-7 and -x0 <= 0 (both
    signs): the first flips to 1, within the tolerance of g, so neither row counts."""
    A = np.array([[1.0, 0.0], [-1.0, 0.0]])
    lb, ub = np.array([0.0, 0.0]), np.array([1.0, 1.0])
    p = milp_from_dense(A, [1.0 - 5e-7, 0.0], lb, ub, [1, 0])
    k1, k2, k3 = oracle.Problem(p).probe_priority(lb, ub)
    assert k1[0] == 0 and k2[0] == 0.0
    p = milp_from_dense(A, [1.0 - 2e-6, 0.0], lb, ub, [1, 0])   # beyond the tolerance: counted
    k1, k2, k3 = oracle.Problem(p).probe_priority(lb, ub)
    assert k1[0] == 1 and abs(k2[0] - 2e-6) < 1e-15


def test_priority_ignores_rows_with_an_infinite_minimal_activity():
    """x0 in [0, 3] integer, y unbounded below, x0 + y <= 4: the row's L_min is -inf, so it takes
    no part and x0's smallest unit slack stays +inf (counted, it would be 4)."""
    lb, ub = np.array([0.0, -np.inf]), np.array([3.0, 5.0])
    p = milp_from_dense(np.array([[1.0, 1.0]]), [4.0], lb, ub, [1, 0])
    k1, k2, k3 = oracle.Problem(p).probe_priority(lb, ub)
    assert k1[0] == 0 and k3[0] == np.inf
    assert k1[1] == -1   # continuous: not probeable


def test_branch_starts_from_root_intersected_with_its_box():
    """A branch runs from root ∩ box (reading of Section 2.2's double probe): x0 integer with
    root [1, 3] and a down box [0, 1] starts the branch at [1, 1], so the cache lists x0 with
    l = 1 (unchanged) and u = 1, never the box's l = 0."""
    lb, ub = np.array([1.0, 0.0]), np.array([3.0, 5.0])
    p = milp_from_dense(np.array([[1.0, 1.0]]), [6.0], lb, ub, [1, 1])
    c = oracle.Problem(p).probe_batch(lb, ub, np.array([0], dtype=np.int32), np.array([[0.0, 1.0, 2.0, 3.0]]))
    b = slice(int(c["offsets"][0]), int(c["offsets"][1]))
    ents = {int(v): (l, u) for v, l, u in zip(c["var"][b], c["l"][b], c["u"][b])}
    assert c["status"][0] == oracle.FIXPOINT and ents[0] == (1.0, 1.0)


def test_infeasible_branch_lists_nothing():
    """x0 + x1 <= 1 with x1 fixed at 1: the up branch of x0 ([1, 1]) is infeasible and lists no
    implied bounds; the down branch is feasible and lists x0 = 0."""
    lb, ub = np.array([0.0, 1.0]), np.array([1.0, 1.0])
    p = milp_from_dense(np.array([[1.0, 1.0]]), [1.0], lb, ub, [1, 1])
    c = oracle.Problem(p).probe_batch(lb, ub, np.array([0], dtype=np.int32), np.array([[0.0, 0.0, 1.0, 1.0]]))
    assert c["status"][1] == oracle.INFEASIBLE and c["offsets"][2] == c["offsets"][1]
    assert c["status"][0] == oracle.FIXPOINT and list(c["var"][:c["offsets"][1]]) == [0]
