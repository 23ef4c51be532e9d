"""Pins of the CPU oracle's bound propagation (no GPU).

The oracle is checked against things other than itself: hand-worked examples (golden
fixtures), a closed form (chain of implications), exact rational arithmetic, brute-force
enumeration of tiny integer problems, and invariants (bounds only tighten, a fixpoint is
idempotent, worklist == full sweep, Jacobi == Gauss-Seidel on integer problems,
permutation invariance).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.helpers import dense, feasible_points, fnum, golden_problem, load_golden, milp_from_dense

GOLDEN_FILES = ["knapsack_3var.json", "continuous_2var.json", "infinite_bounds.json",
                "cover_infeasible.json"]


@pytest.mark.parametrize("fname", GOLDEN_FILES)
def test_golden_examples(fname):
    d = load_golden(fname)
    for case in d["cases"]:
        p = golden_problem(d, case)
        P = oracle.Problem(p)
        lb = np.array([fnum(x) for x in case["lb"]])
        ub = np.array([fnum(x) for x in case["ub"]])
        ol, ou, r, _ = P.bp(lb, ub)
        assert r["status"] == case["status"], case["note"]
        assert r["rounds"] == case["rounds"], case["note"]
        assert r["nnz_updates"] == case["nnz_updates"], case["note"]
        if "n_changed" in case:
            assert r["n_changed"] == case["n_changed"], case["note"]
        if "first_infeasible_row" in case:
            assert r["first_infeasible_row"] == case["first_infeasible_row"]
        np.testing.assert_array_equal(ol, [fnum(x) for x in case["out_lb"]], err_msg=case["note"])
        np.testing.assert_array_equal(ou, [fnum(x) for x in case["out_ub"]], err_msg=case["note"])
        assert r["fragile"] == 0


@pytest.mark.parametrize("k", [2, 3, 5, 17])
def test_chain_round_count_closed_form(k):
    """x_i - x_{i+1} <= 0 (i = 1..k-1), x_k fixed to 0, x integer in [0, 10]: round j
    (j = 0..k-2) fixes u of x_{k-1-j} to 0, round k-1 finds nothing, so exactly k rounds and
    2(k-1) + 4(k-2) + 2 = 6k - 8 row nonzeros are processed."""
    A = np.zeros((k - 1, k))
    for i in range(k - 1):
        A[i, i], A[i, i + 1] = 1.0, -1.0
    lb = np.zeros(k)
    ub = np.full(k, 10.0)
    ub[-1] = 0.0
    p = milp_from_dense(A, np.zeros(k - 1), lb, ub, np.ones(k))
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    assert r["status"] == oracle.FIXPOINT
    assert r["rounds"] == k
    assert r["nnz_updates"] == 6 * k - 8
    np.testing.assert_array_equal(ou, np.zeros(k))
    np.testing.assert_array_equal(ol, np.zeros(k))
    # the round limit stops one round short
    _, ou2, r2, _ = oracle.Problem(p).bp(lb, ub, max_rounds=k - 1)
    assert r2["status"] == oracle.ROUND_LIMIT and r2["rounds"] == k - 1


def _exact_round(p, lb, ub, theta=1e-3, tol=1e-6):
    """One Jacobi round of Section 2.1 in exact rational arithmetic on the double inputs."""
    tolq = Fraction(tol)
    nl = [Fraction(x) if math.isfinite(x) else x for x in lb]
    nu = [Fraction(x) if math.isfinite(x) else x for x in ub]
    decisions = []
    for k in range(p.m):
        terms, ninf, infj = [], 0, -1
        for q in range(p.row_ptr[k], p.row_ptr[k + 1]):
            a, j = Fraction(p.val[q]), int(p.col[q])
            b = lb[j] if a > 0 else ub[j]
            if math.isinf(b):
                ninf += 1
                infj = j
            else:
                terms.append((q, a * Fraction(b)))
        lmin = sum(t for _, t in terms)
        g = Fraction(p.g[k])
        if ninf == 0 and lmin > g + tolq:
            decisions.append(("rowinf", k))
            continue
        if ninf >= 2:
            continue
        tmap = dict(terms)
        for q in range(p.row_ptr[k], p.row_ptr[k + 1]):
            a, j = Fraction(p.val[q]), int(p.col[q])
            if ninf == 1 and j != infj:
                continue
            resid = lmin - tmap.get(q, 0) if ninf == 0 else lmin
            cand = (g - resid) / a
            if a > 0:
                if p.is_int[j]:
                    c = Fraction(math.floor(cand + tolq))
                    if math.isinf(ub[j]) or c < Fraction(ub[j]):
                        nu[j] = c if (math.isinf(nu[j]) or c < nu[j]) else nu[j]
                elif math.isinf(ub[j]) or Fraction(ub[j]) - cand > Fraction(theta) * max(1, abs(Fraction(ub[j]))):
                    nu[j] = cand if (math.isinf(nu[j]) or cand < nu[j]) else nu[j]
            else:
                if p.is_int[j]:
                    c = Fraction(math.ceil(cand - tolq))
                    if math.isinf(lb[j]) or c > Fraction(lb[j]):
                        nl[j] = c if (math.isinf(nl[j]) or c > nl[j]) else nl[j]
                elif math.isinf(lb[j]) or cand - Fraction(lb[j]) > Fraction(theta) * max(1, abs(Fraction(lb[j]))):
                    nl[j] = cand if (math.isinf(nl[j]) or cand > nl[j]) else nl[j]
    return nl, nu, decisions


@pytest.mark.parametrize("seed", range(12))
def test_one_round_matches_exact_rationals(seed):
    """After one round, integer bounds equal the exact-arithmetic result unless the oracle
    flags a fragile decision, and continuous bounds are within the oracle's own reported
    uncertainty of the exact values."""
    p = synth.random_milp(1000 + seed, m=6, n=10, len_lo=1, len_hi=6, inf_fraction=0.2, slack_scale=0.02)
    lb, ub = synth.tighten_random(seed, p, 3, planted=(seed % 2 == 0))
    P = oracle.Problem(p)
    lb, ub = P.normalize(lb, ub)
    ol, ou, r, (dl, du) = P.bp(lb, ub, max_rounds=1)
    nl, nu, dec = _exact_round(p, lb, ub)
    assert (r["status"] == oracle.INFEASIBLE) == (any(d[0] == "rowinf" for d in dec) or
                                                  any(not math.isinf(nl[j]) and not math.isinf(nu[j]) and
                                                      (nl[j] > nu[j] if p.is_int[j] else nl[j] > nu[j] + Fraction(1e-6))
                                                      for j in range(p.n))) or r["fragile"] > 0
    if r["fragile"]:
        return
    for j in range(p.n):
        for got, want, d in ((ol[j], nl[j], dl[j]), (ou[j], nu[j], du[j])):
            if isinstance(want, float) and math.isinf(want):
                assert got == want
            elif p.is_int[j]:
                assert Fraction(got) == want
            else:
                assert abs(Fraction(got) - want) <= Fraction(d) + Fraction(abs(got)) * Fraction(2.0 ** -52)


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_soundness(seed):
    """BP never cuts off an integer-feasible point; INFEASIBLE only without feasible points."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 8))
    m = int(rng.integers(1, 6))
    A = rng.integers(-4, 5, size=(m, n)).astype(float)
    A[rng.uniform(size=(m, n)) < 0.3] = 0.0
    for k in range(m):
        if not A[k].any():
            A[k, rng.integers(0, n)] = 1.0
    ub = rng.integers(1, 4, size=n).astype(float)
    lb = np.zeros(n)
    g = rng.integers(-3, 8, size=m).astype(float)
    p = milp_from_dense(A, g, lb, ub, np.ones(n))
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    pts = feasible_points(p, lb, ub)
    if r["status"] == oracle.INFEASIBLE:
        assert len(pts) == 0
    else:
        assert r["status"] == oracle.FIXPOINT
        if len(pts):
            assert (pts >= ol[None, :]).all() and (pts <= ou[None, :]).all()
    assert r["fragile"] == 0


def _inv_case(seed):
    return synth.random_milp(seed, m=60, n=80, len_lo=1, len_hi=9, integer_coefs=True,
                             int_fraction=1.0, bin_fraction=0.4, slack_scale=0.1)


@pytest.mark.parametrize("seed", range(8))
def test_invariants(seed):
    p = _inv_case(50 + seed)
    P = oracle.Problem(p)
    lb, ub = synth.tighten_random(seed, p, 8)
    lb, ub = P.normalize(lb, ub)
    ol, ou, r, _ = P.bp(lb, ub)
    # bounds only tighten
    assert (ol >= lb).all() and (ou <= ub).all()
    if r["status"] != oracle.FIXPOINT:
        return
    # idempotent
    ol2, ou2, r2, _ = P.bp(ol, ou)
    np.testing.assert_array_equal(ol2, ol)
    np.testing.assert_array_equal(ou2, ou)
    assert r2["n_changed"] == 0 and r2["rounds"] == 1
    # full sweep: same bounds and rounds, at least as much work
    ol3, ou3, r3, _ = P.bp(lb, ub, mode=1)
    np.testing.assert_array_equal(ol3, ol)
    np.testing.assert_array_equal(ou3, ou)
    assert r3["rounds"] == r["rounds"] and r3["nnz_updates"] >= r["nnz_updates"]
    # Gauss-Seidel reaches the same fixpoint on a bounded integer problem
    ol4, ou4, r4, _ = P.bp(lb, ub, mode=2)
    assert r4["status"] == oracle.FIXPOINT
    np.testing.assert_array_equal(ol4, ol)
    np.testing.assert_array_equal(ou4, ou)


@pytest.mark.parametrize("seed", range(5))
def test_permutation_invariance_exact(seed):
    """Integer data: permuting rows and variables permutes the result, rounds unchanged."""
    p = _inv_case(90 + seed)
    lb, ub = synth.tighten_random(seed, p, 6)
    rng = np.random.default_rng(seed)
    rp = rng.permutation(p.m)
    cp = rng.permutation(p.n)
    A = dense(p)
    q = milp_from_dense(A[rp][:, cp], p.g[rp], lb[cp], ub[cp], p.is_int[cp])
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    ql, qu, s, _ = oracle.Problem(q).bp(lb[cp], ub[cp])
    assert r["status"] == s["status"] and r["rounds"] == s["rounds"]
    assert r["nnz_updates"] == s["nnz_updates"]
    np.testing.assert_array_equal(ql, ol[cp])
    np.testing.assert_array_equal(qu, ou[cp])


@pytest.mark.parametrize("seed", range(8))
def test_error_window_covers_summation_order(seed):
    """Non-integer data: relabelling variables changes every row's summation order.  Both
    runs must agree on integer bounds and status when neither saw a fragile decision, and
    on continuous bounds within the sum of their reported uncertainties."""
    p = synth.random_milp(300 + seed, m=400, n=300, len_lo=2, len_hi=30, slack_scale=0.03)
    lb, ub = synth.tighten_random(seed, p, 40, planted=(seed % 2 == 0))
    cp = np.random.default_rng(seed).permutation(p.n)
    A = dense(p)
    q = milp_from_dense(A[:, cp], p.g, lb[cp], ub[cp], p.is_int[cp])
    ol, ou, r, (dl, du) = oracle.Problem(p).bp(lb, ub)
    ql, qu, s, (el, eu) = oracle.Problem(q).bp(lb[cp], ub[cp])
    if r["fragile"] or s["fragile"]:
        pytest.skip("fragile decision in this seed")
    assert r["status"] == s["status"] and r["rounds"] == s["rounds"]
    ints = p.is_int[cp] == 1
    np.testing.assert_array_equal(ql[ints], ol[cp][ints])
    np.testing.assert_array_equal(qu[ints], ou[cp][ints])
    fin = np.isfinite(ol[cp])
    assert (np.abs(ql[fin] - ol[cp][fin]) <= el[fin] + dl[cp][fin] + 1e-300).all()
    fin = np.isfinite(ou[cp])
    assert (np.abs(qu[fin] - ou[cp][fin]) <= eu[fin] + du[cp][fin] + 1e-300).all()


def test_normalisation():
    p = milp_from_dense(np.ones((1, 4)), [10.0], np.zeros(4), np.ones(4), [1, 1, 0, 0])
    P = oracle.Problem(p)
    lb, ub = P.normalize([0.3, -1e21, -2e20, 0.5], [2.9999999, 7.0000001, 1e20, 3.0])
    np.testing.assert_array_equal(lb, [1.0, -np.inf, -np.inf, 0.5])
    np.testing.assert_array_equal(ub, [3.0, 7.0, np.inf, 3.0])


def test_entry_crossing_and_empty_row():
    # an empty row with g < 0 is infeasible in round 0 (0 > g + tol)
    p = milp_from_dense(np.zeros((1, 2)), [-1.0], np.zeros(2), np.ones(2), [1, 1])
    _, _, r, _ = oracle.Problem(p).bp(np.zeros(2), np.ones(2))
    assert r["status"] == oracle.INFEASIBLE and r["rounds"] == 1 and r["first_infeasible_row"] == 0
    # bounds that already cross: infeasible before any round
    p = milp_from_dense(np.ones((1, 2)), [5.0], np.zeros(2), np.ones(2), [1, 0])
    _, _, r, _ = oracle.Problem(p).bp([0.0, 2.0], [1.0, 1.0])
    assert r["status"] == oracle.INFEASIBLE and r["rounds"] == 0 and r["first_infeasible_var"] == 1
    # a continuous crossing within the tolerance is not infeasible
    _, _, r, _ = oracle.Problem(p).bp([0.0, 1.0 + 5e-7], [1.0, 1.0])
    assert r["status"] == oracle.FIXPOINT


def test_rejects_malformed():
    from paper_2510_20499_gb300.synth import Milp
    base = dict(m=1, n=2, g=np.array([1.0]), lb=np.zeros(2), ub=np.ones(2),
                is_int=np.ones(2, dtype=np.uint8), c=np.zeros(2))
    bad = [
        (np.array([0, 2]), np.array([1, 0]), np.array([1.0, 1.0])),      # columns not increasing
        (np.array([0, 2]), np.array([0, 2]), np.array([1.0, 1.0])),      # column out of range
        (np.array([0, 2]), np.array([0, 1]), np.array([1.0, 0.0])),      # zero coefficient
        (np.array([0, 2]), np.array([0, 1]), np.array([1.0, np.nan])),   # NaN
    ]
    for rp, cl, vl in bad:
        q = Milp(row_ptr=rp.astype(np.int64), col=cl.astype(np.int32), val=vl, **base)
        with pytest.raises(ValueError):
            oracle.Problem(q)


def test_mixed_instance_small_runs_clean():
    """A scaled-down mixed power-law instance runs to a fixpoint with no fragile decision."""
    p = synth.mixed_powerlaw(seed=7, m=2000, n=5000, nnz=50_000, max_row=1000)
    ol, ou, r, _ = oracle.Problem(p).bp(p.lb, p.ub)
    assert r["status"] == oracle.FIXPOINT
    assert r["fragile"] == 0
    # the planted point stays inside the bounds (soundness on a known feasible point)
    assert (p.x0 >= ol - 1e-6).all() and (p.x0 <= ou + 1e-6).all()


def _rows_of(p, vars_):
    """Rows holding any of the given variables (ascending)."""
    col = np.asarray(p.col)
    row_of = np.repeat(np.arange(p.m), np.diff(p.row_ptr))
    return np.unique(row_of[np.isin(col, vars_)]).astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_block_diagonal_pair_propagates_each_copy_alone(seed):
    """Two copies of one problem side by side (rows k and m + k, variables j and n + j), each
    started from its own fixings: propagated together from the union of their start rows, every
    copy ends with the bounds of its own propagation, the nonzeros add up and the rounds are the
    larger of the two. Jacobi rounds never couple disjoint blocks; this is what lets the two
    candidate vectors of a fix-and-propagate bulk share one propagation."""
    p = synth.random_milp(900 + seed, m=250, n=320, len_lo=1, len_hi=12, int_fraction=0.8, integer_coefs=True)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    if r["status"] != oracle.FIXPOINT:
        pytest.skip("root not at a fixpoint")
    rng = np.random.default_rng(seed)
    free = np.flatnonzero((rl < ru) & (p.is_int == 1))
    starts = []
    for c in range(2):
        fix = rng.choice(free, size=min(6, len(free)), replace=False)
        l, u = rl.copy(), ru.copy()
        for j in fix:   # round the variable to one of its bounds, as a rounding bulk does
            v = l[j] if rng.uniform() < 0.5 else u[j]
            if not np.isfinite(v):
                v = l[j] if np.isfinite(l[j]) else u[j]
            l[j] = u[j] = v
        starts.append((l, u, _rows_of(p, fix)))
    alone = [P.bp(l, u, w0=w) for l, u, w in starts]
    if any(a[2]["status"] == oracle.INFEASIBLE for a in alone):
        pytest.skip("a copy is infeasible: the pair would stop with it")
    pair, ro, co = synth.block_diagonal([p, p])
    PP = oracle.Problem(pair)
    w0 = np.concatenate([starts[0][2], starts[1][2] + p.m]).astype(np.int32)
    L, U, R, _ = PP.bp(np.concatenate([starts[0][0], starts[1][0]]), np.concatenate([starts[0][1], starts[1][1]]), w0=w0)
    for c in range(2):
        np.testing.assert_array_equal(L[c * p.n:(c + 1) * p.n], alone[c][0])
        np.testing.assert_array_equal(U[c * p.n:(c + 1) * p.n], alone[c][1])
    assert R["status"] == oracle.FIXPOINT
    assert R["nnz_updates"] == alone[0][2]["nnz_updates"] + alone[1][2]["nnz_updates"]
    assert R["rounds"] == max(alone[0][2]["rounds"], alone[1][2]["rounds"])


# --- hand-worked readings at the edges of the tolerances and of the infinity counts ---


def test_row_violation_within_the_tolerance_is_feasible():
    """Row infeasibility is L_min > g + 1e-6 (Section 3's tolerance): x0 <= -5e-7 with x0 in
    [0, 1] has L_min = 0, within the tolerance of g, so it is not infeasible; x0 <= -2e-6 is."""
    lb, ub = np.array([0.0]), np.array([1.0])
    p = milp_from_dense([[1.0]], [-5e-7], lb, ub, [0])
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    assert r["status"] == oracle.FIXPOINT
    p = milp_from_dense([[1.0]], [-2e-6], lb, ub, [0])
    _, _, r, _ = oracle.Problem(p).bp(lb, ub)
    assert r["status"] == oracle.INFEASIBLE and r["first_infeasible_row"] == 0


def test_two_infinite_contributions_propose_no_bound():
    """x0 + x1 + x2 <= 5 with x0, x1 unbounded below: L_min has two infinite contributions, so no
    residual is finite and x2 in [0, 10] keeps its bounds (with one, x2 would get u = 5 - ...)."""
    lb = np.array([-np.inf, -np.inf, 0.0])
    ub = np.array([10.0, 10.0, 10.0])
    p = milp_from_dense([[1.0, 1.0, 1.0]], [5.0], lb, ub, [0, 0, 0])
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    np.testing.assert_array_equal(ol, lb)
    np.testing.assert_array_equal(ou, ub)
    assert r["rounds"] == 1 and r["n_changed"] == 0
    # one infinite contribution: only the infinite variable gets a bound, 5 - L_min(others)
    lb1 = np.array([-np.inf, 0.0, 0.0])
    p = milp_from_dense([[1.0, 1.0, 1.0]], [5.0], lb1, ub, [0, 0, 0])
    ol, ou, r, _ = oracle.Problem(p).bp(lb1, ub)
    np.testing.assert_array_equal(ou, [5.0, 10.0, 10.0])


def test_continuous_threshold_uses_at_least_one():
    """A continuous bound moves only when the improvement exceeds theta * max(1, |bound|):
    x0 <= 0.4993 with x0 in [0, 0.5] improves u by 7e-4 < 1e-3 * max(1, 0.5), so nothing moves
    (theta * |u| = 5e-4 would have accepted it); x0 <= 0.4985 (1.5e-3) moves u."""
    lb, ub = np.array([0.0]), np.array([0.5])
    p = milp_from_dense([[1.0]], [0.4993], lb, ub, [0])
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    assert ou[0] == 0.5 and r["n_changed"] == 0
    p = milp_from_dense([[1.0]], [0.4985], lb, ub, [0])
    ol, ou, r, _ = oracle.Problem(p).bp(lb, ub)
    assert ou[0] == 0.4985


def test_first_infeasible_indices_are_the_smallest():
    """When several variables cross (or rows are infeasible) in the same round, the result
    reports the smallest index.  Variables: x0, x1 integer in [0, 1], z, w continuous in [0, 1];
    rows -x - z <= -2 give x >= 1 and x + w <= 0.5 give x <= 0 for both x0 and x1 in round 0,
    with every row feasible: both cross, the first infeasible variable is 0.  Rows -x1 <= -2 and
    -x0 <= -2 (x0, x1 in [0, 1]) are both infeasible in round 0: the first infeasible row is 0."""
    A = [[-1, 0, -1, 0], [1, 0, 0, 1], [0, -1, -1, 0], [0, 1, 0, 1]]
    lb, ub = np.zeros(4), np.ones(4)
    p = milp_from_dense(A, [-2, 0.5, -2, 0.5], lb, ub, [1, 1, 0, 0])
    _, _, r, _ = oracle.Problem(p).bp(lb, ub)
    assert (r["status"], r["rounds"], r["first_infeasible_var"], r["first_infeasible_row"]) == (oracle.INFEASIBLE, 1, 0, -1)
    p = milp_from_dense([[0, -1], [-1, 0]], [-2, -2], np.zeros(2), np.ones(2), [1, 1])
    _, _, r, _ = oracle.Problem(p).bp(np.zeros(2), np.ones(2))
    assert (r["status"], r["first_infeasible_row"], r["first_infeasible_var"]) == (oracle.INFEASIBLE, 0, -1)
