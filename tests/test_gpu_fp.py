"""GPU fix-and-propagate (fix_and_propagate through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.helpers import dense, load_golden

pytestmark = pytest.mark.gpu

KEYS = ("status", "bulks", "bp_runs", "recoveries", "fixed_by_choice", "refuted", "nnz_updates")


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def _t(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), device="cuda", dtype=dtype)


def _gpu_fp(pkg, p, x, cache=None, **kw):
    import torch
    prob = pkg.Problem(p)
    gc = None
    if cache is not None:
        gc = {k: _t(cache[k]) for k in ("status", "offsets", "var", "l", "u")}
        gc["pairs"] = _t(cache["pairs"], torch.int32)
        gc["boxes"] = _t(cache["boxes"], torch.float64)
        gc["status"] = gc["status"].to(torch.int32)
        gc["offsets"] = gc["offsets"].to(torch.int64)
        gc["var"] = gc["var"].to(torch.int32)
    kw2 = dict(kw)
    for k in ("order_score", "up_prob"):
        if kw2.get(k) is not None:
            kw2[k] = _t(kw2[k], torch.float64)
    out, r = prob.fix_and_propagate(_t(x, torch.float64), _t(p.lb, torch.float64), _t(p.ub, torch.float64),
                                    cache=gc, **kw2)
    return out.cpu().numpy(), r


def _check(p, x, cache=None, **kw):
    import paper_2510_20499_gb300 as pkg
    ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, cache=cache, **kw)
    gx, gr = _gpu_fp(pkg, p, x, cache=cache, **kw)
    for k in KEYS:
        assert gr[k] == orr[k], (k, gr, orr)
    np.testing.assert_array_equal(gx, ox)
    return gr


@pytest.mark.parametrize("case", range(5))
def test_golden(pkg, case):
    c = load_golden("fp_small.json")["cases"][case]
    p = synth.Milp(c["m"], c["n"], np.array(c["row_ptr"], dtype=np.int64), np.array(c["col"], dtype=np.int32),
                   np.array(c["val"], float), np.array(c["g"], float), np.array(c["lb"], float),
                   np.array(c["ub"], float), np.array(c["is_int"], dtype=np.uint8), np.zeros(c["n"]))
    gx, gr = _gpu_fp(pkg, p, np.array(c["x"], float))
    assert gr["status"] == c["status"] and gr["bulks"] == c["bulks"] and gr["bp_runs"] == c["bp_runs"]
    np.testing.assert_array_equal(gx, c["x_out"])


@pytest.mark.parametrize("seed", range(4))
def test_knapsack_cover_exact(pkg, seed):
    p = synth.knapsack_cover(seed=80 + seed, m=3000, n=6000, nnz=60_000)
    x = np.random.default_rng(seed).uniform(0, 1, p.n)
    _check(p, x, seed=seed)


@pytest.mark.parametrize("seed", range(3))
def test_general_integer_exact(pkg, seed):
    p = synth.random_milp(900 + seed, 2000, 3000, len_lo=2, len_hi=40, integer_coefs=True, int_fraction=1.0,
                          slack_scale=0.2, neg_fraction=0.4)
    x = np.random.default_rng(seed).uniform(0, 20, p.n)
    _check(p, x, seed=seed + 10)
    _check(p, x, seed=seed + 20, bulk_rule=1, fraction=0.02, last_single=10)


def test_with_probing_cache(pkg):
    import torch
    p = synth.knapsack_cover(seed=7, m=2000, n=4000, nnz=40_000)
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    k1, k2, k3 = P.probe_priority(rl, ru)
    var = oracle.priority_order(k1, k2, k3)[:800].astype(np.int32)
    boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=np.float64).reshape(-1, 4)
    cache = P.probe_batch(rl, ru, var, boxes)
    cache["pairs"], cache["boxes"] = var, boxes
    for seed in range(3):
        x = np.random.default_rng(seed).uniform(0, 1, p.n)
        _check(p, x, cache=cache, seed=seed)


def test_hooks(pkg):
    p = synth.random_milp(31, 1500, 2500, len_lo=2, len_hi=20, integer_coefs=True, int_fraction=1.0, slack_scale=0.3)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 20, p.n)
    _check(p, x, order_score=rng.standard_normal(p.n), up_prob=rng.uniform(0, 1, p.n))


def test_general_data_soundness(pkg):
    """Non-integer coefficients: every FEASIBLE result is verified row by row by the oracle's
    side (integer values integral, a propagation from the start bounds with them fixed not
    infeasible, and a continuous completion found by HiGHS within 1e-6 of every row)."""
    pytest.importorskip("scipy")
    from tests.gpu_helpers import verified_feasible
    feasible = 0
    for inst in range(3):
        p = synth.random_milp(55 + inst, 1500, 2000, len_lo=2, len_hi=30, int_fraction=0.7, slack_scale=0.2)
        P = oracle.Problem(p)
        for seed in range(3):
            x = np.clip(p.x0 + np.random.default_rng(seed).normal(0, 0.5, p.n), p.lb, p.ub)
            gx, gr = _gpu_fp(pkg, p, x, seed=seed)
            if gr["status"] == 0:
                feasible += 1
                assert verified_feasible(p, P, gx), (inst, seed)
    assert feasible >= 3


MIXED = [(55, 0, {}), (56, 1, {}), (57, 2, dict(bulk_rule=1, fraction=0.02, last_single=10)),
         (58, 0, dict(bulk_rule=1, fraction=0.05)), (59, 1, {})]


@pytest.mark.parametrize("inst,seed,kw", MIXED, ids=[f"i{m[0]}-s{m[1]}" for m in MIXED])
def test_mixed_data_parity(pkg, inst, seed, kw):
    """Mixed integer/continuous problems with non-integer coefficients (power-of-ten decimals):
    the oracle reports no fragile decision (propagations and implied-slack bulk boundaries), so
    the GPU must take every decision the oracle takes: the same status, bulks, propagations,
    recoveries, kept fixings and work, the same integer values, and continuous values within
    1e-9 relative."""
    p = synth.random_milp(inst, 1500, 2000, len_lo=2, len_hi=30, int_fraction=0.7, slack_scale=0.2)
    x = np.clip(p.x0 + np.random.default_rng(seed).normal(0, 0.5, p.n), p.lb, p.ub)
    ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, seed=seed, **kw)
    assert orr["fragile"] == 0, orr
    gx, gr = _gpu_fp(pkg, p, x, seed=seed, **kw)
    for k in KEYS:
        assert gr[k] == orr[k], (k, gr, orr)
    ints = p.is_int == 1
    np.testing.assert_array_equal(gx[ints], ox[ints])
    np.testing.assert_allclose(gx[~ints], ox[~ints], rtol=1e-9, atol=1e-9)


def test_order_score_replaces_implied_slack_order(pkg):
    """The hand-worked case of the oracle's pin: with the score, one bulk and no recovery."""
    from tests.helpers import milp_from_dense
    A = np.array([[10.0, 10.0, 0.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
    p = milp_from_dense(A, [10.0, 1.5], np.zeros(4), np.ones(4), np.ones(4))
    x = np.full(4, 0.8)
    r = _check(p, x, last_single=0)
    assert (r["bulks"], r["recoveries"]) == (4, 2)
    r = _check(p, x, last_single=0, order_score=np.array([3.0, 0.0, 2.0, 1.0]))
    assert (r["bulks"], r["recoveries"]) == (1, 0)


@pytest.mark.parametrize("seed", range(2))
def test_hooks_fraction_rule(pkg, seed):
    """Score order (no implied-slack sort) and up probabilities under the 1% bulk rule."""
    p = synth.random_milp(61 + seed, 3000, 5000, len_lo=2, len_hi=30, integer_coefs=True, int_fraction=1.0,
                          slack_scale=0.3)
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 20, p.n)
    _check(p, x, seed=seed, bulk_rule=1, fraction=0.01, order_score=rng.standard_normal(p.n),
           up_prob=rng.uniform(0, 1, p.n))


def test_implied_slack_order_golden(pkg):
    """The hand-worked implied-slack case (Section 2.3, Algorithm 1) on the GPU: the same first
    bulk and result as the fixture."""
    c = load_golden("fp_slack_order.json")
    p = synth.Milp(c["m"], c["n"], np.array(c["row_ptr"], dtype=np.int64), np.array(c["col"], dtype=np.int32),
                   np.array(c["val"], float), np.array(c["g"], float), np.array(c["lb"], float),
                   np.array(c["ub"], float), np.array(c["is_int"], dtype=np.uint8), np.zeros(c["n"]))
    for seed in (1, 2):
        gx, gr = _gpu_fp(pkg, p, np.array(c["x"], float), seed=seed, last_single=c["last_single"])
        np.testing.assert_array_equal(gx, c["x_out"])
        assert (gr["status"], gr["bulks"], gr["bp_runs"], gr["recoveries"]) == \
            (c["status"], c["bulks"], c["bp_runs"], c["recoveries"])


def test_final_check_refutes_an_incremental_verdict(pkg):
    """The hand-worked case of the oracle's pin: every incremental propagation is feasible, the
    final check from the caller's bounds is not (refuted, INFEASIBLE), as in the oracle."""
    from tests.helpers import milp_from_dense
    A = np.array([[50.0, 0, 1, 0], [0, 0.02, 1, 0], [0, 0, -1, 0], [0, 0, -1, 1], [0, 0, 0, -1]])
    p = milp_from_dense(A, [100, 50.01, -49.985, -49.985, -0.01], np.zeros(4), np.array([1, 1, 100, 10.0]),
                        np.array([1, 1, 0, 0]))
    r = _check(p, np.array([0.8, 0.8, 50.0, 0.02]), seed=1)
    assert (r["status"], r["refuted"], r["bulks"], r["bp_runs"]) == (1, 1, 2, 5)


RECOVERY = [(3000, 1, False), (3001, 1, True), (3004, 2, False), (3005, 1, True)]


@pytest.mark.parametrize("inst,seed,learned", RECOVERY, ids=[f"i{r[0]}-s{r[1]}-{'up' if r[2] else 'plain'}"
                                                             for r in RECOVERY])
def test_recovery_on_device_parity(pkg, inst, seed, learned):
    """Runs with several failed bulks (Algorithm 1's recovery: the failed bulk's variables one at
    a time, each with the drawn value and the other rounding) on 100k-nonzero rounding
    instances; without a probing cache the one-variable bulks run in one device-driven launch
    per recovery.  With and without given up-probabilities (which replace the draw's band), the
    result must equal the oracle's: every count, the integer values, and the continuous values
    within 1e-9 relative (the oracle reports no fragile decision)."""
    p, x = synth.rounding_instance(inst, 100_000, eq_fraction=0.01)
    kw = dict(seed=seed, bulk_rule=1, fraction=0.01)
    if learned:
        kw["up_prob"] = np.random.default_rng((inst - 3000) * 10 + seed).uniform(0, 1, p.n)
    ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, **kw)
    assert orr["fragile"] == 0 and orr["recoveries"] > 0, orr
    gx, gr = _gpu_fp(pkg, p, x, **kw)
    for k in KEYS:
        assert gr[k] == orr[k], (k, gr, orr)
    ints = p.is_int == 1
    np.testing.assert_array_equal(gx[ints], ox[ints])
    np.testing.assert_allclose(gx[~ints], ox[~ints], rtol=1e-9, atol=1e-9)


def test_recovery_ending_infeasible_parity(pkg):
    """A run whose recovery meets a variable with both values infeasible (the rounding fails,
    status 1):
    20% equality pairs at 100k nonzeros.  Same counts and output as the oracle."""
    for inst in range(1000, 1012):
        p, x = synth.rounding_instance(inst, 100_000)
        ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, seed=1, bulk_rule=1, fraction=0.01)
        if orr["status"] == 1 and orr["recoveries"] > 0 and orr["refuted"] == 0 \
                and orr["fragile"] == 0:
            break
    else:
        pytest.fail("no instance of the set ends infeasible in a recovery")
    gx, gr = _gpu_fp(pkg, p, x, seed=1, bulk_rule=1, fraction=0.01)
    for k in KEYS:
        assert gr[k] == orr[k], (k, gr, orr)
    ints = p.is_int == 1
    np.testing.assert_array_equal(gx[ints], ox[ints])
    np.testing.assert_allclose(gx[~ints], ox[~ints], rtol=1e-9, atol=1e-9)


RKEYS = KEYS + ("repairs", "repair_runs")


@pytest.mark.parametrize("which", ["case", "with_implied"])
@pytest.mark.parametrize("seed", range(1, 7))
def test_repair_golden(pkg, which, seed):
    """The hand-worked repair cases (Section 2.3, the repair branch of Algorithm 1) on the GPU."""
    from tests.helpers import milp_from_dense
    d = load_golden("fp_repair.json")
    c = d if which == "case" else d["with_implied"]
    p = milp_from_dense(c["A"], c["g"], c["lb"], c["ub"], [1] * len(c["lb"]))
    x = np.array(c["x"])
    up = oracle.uniform(seed, 1, 1, 0) < d["p_up_x1"]
    want = c["with_repair"]["x1_drawn_up" if up else "x1_drawn_down"]
    gx, gr = _gpu_fp(pkg, p, x, seed=seed, repair_max=4)
    for k in ("status", "bulks", "fixed_by_choice", "repairs", "repair_runs", "bp_runs"):
        assert gr[k] == want[k], (k, gr, want)
    np.testing.assert_array_equal(gx, want["x_out"])
    gx, gr = _gpu_fp(pkg, p, x, seed=seed)
    assert gr["status"] == c["without_repair"]["status"] and gr["repairs"] == 0
    np.testing.assert_array_equal(gx, c["without_repair"]["x_out"])


def test_repair_tiny_planted_parity(pkg):
    """Tiny planted problems rounded from the opposite corner (one-variable bulks driven by the
    host): with repair the GPU takes the oracle's every decision."""
    from tests.test_oracle_repair import _tiny_planted
    rng = np.random.default_rng(11)
    repaired = 0
    for _ in range(200):
        n = int(rng.integers(4, 9))
        p, A, g, ub, x = _tiny_planted(rng, n, int(rng.integers(3, 7)), 0.3, 2)
        seed = int(rng.integers(1, 1000))
        ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, seed=seed, repair_max=6)
        gx, gr = _gpu_fp(pkg, p, x, seed=seed, repair_max=6)
        for k in RKEYS:
            assert gr[k] == orr[k], (k, gr, orr)
        np.testing.assert_array_equal(gx, ox)
        repaired += orr["repair_runs"] > 0
    assert repaired >= 5


@pytest.mark.parametrize("inst", [1001, 1002, 1003])
def test_repair_parity_rounding_instances(pkg, inst):
    """100k-nonzero rounding instances (20% equality pairs, 1% bulks) whose retries of a failed
    bulk run into a variable failing both ways: the repair starts from the device-driven retry
    launch, which resumes behind the repaired variable.  1001: the repair fails; 1002: it
    succeeds and the rounding ends feasible; 1003: one success, then a failure."""
    p, x = synth.rounding_instance(inst, 100_000)
    kw = dict(seed=1, bulk_rule=1, fraction=0.01, repair_max=4)
    ox, orr = oracle.Problem(p).fix_and_propagate(x, p.lb, p.ub, **kw)
    assert orr["fragile"] == 0 and orr["repair_runs"] > 0, orr
    gx, gr = _gpu_fp(pkg, p, x, **kw)
    for k in RKEYS:
        assert gr[k] == orr[k], (k, gr, orr)
    ints = p.is_int == 1
    np.testing.assert_array_equal(gx[ints], ox[ints])
    np.testing.assert_allclose(gx[~ints], ox[~ints], rtol=1e-9, atol=1e-9)


def test_repair_rejects_a_cache(pkg):
    d = load_golden("fp_repair.json")
    from tests.helpers import milp_from_dense
    p = milp_from_dense(d["A"], d["g"], d["lb"], d["ub"], [1] * 3)
    cache = {"pairs": np.array([0], np.int32), "boxes": np.array([[0, 0, 1, 1]], float),
             "status": np.array([0, 0], np.int32), "offsets": np.array([0, 0, 0], np.int64),
             "var": np.zeros(0, np.int32), "l": np.zeros(0), "u": np.zeros(0)}
    with pytest.raises(Exception):
        _gpu_fp(pkg, p, np.array(d["x"]), cache=cache, repair_max=1)
