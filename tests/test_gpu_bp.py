"""GPU bound propagation (bp_propagate through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.gpu_helpers import compare, run_gpu
from tests.helpers import fnum, golden_problem, load_golden, milp_from_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


@pytest.mark.parametrize("fname", ["knapsack_3var.json", "continuous_2var.json", "infinite_bounds.json",
                                   "cover_infeasible.json"])
def test_golden(pkg, fname):
    d = load_golden(fname)
    for case in d["cases"]:
        p = golden_problem(d, case)
        lb = np.array([fnum(x) for x in case["lb"]])
        ub = np.array([fnum(x) for x in case["ub"]])
        gl, gu, r = run_gpu(pkg.Problem(p), lb, ub)
        assert r["status"] == case["status"] and r["rounds"] == case["rounds"], (case["note"], r)
        assert r["nnz_updates"] == case["nnz_updates"], case["note"]
        np.testing.assert_array_equal(gl, [fnum(x) for x in case["out_lb"]], err_msg=case["note"])
        np.testing.assert_array_equal(gu, [fnum(x) for x in case["out_ub"]], err_msg=case["note"])


def test_binary_knapsack_full(pkg):
    """2k x 5k all-binary instance (exact arithmetic): everything bit-exact."""
    p = synth.binary_knapsack()
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    gl, gu, gr = run_gpu(pkg.Problem(p), p.lb, p.ub)
    assert compare(p, gl, gu, gr, ol, ou, orr)


@pytest.mark.parametrize("k", [2, 5, 40])
def test_chain(pkg, k):
    A = np.zeros((k - 1, k))
    for i in range(k - 1):
        A[i, i], A[i, i + 1] = 1.0, -1.0
    lb, ub = np.zeros(k), np.full(k, 10.0)
    ub[-1] = 0.0
    p = milp_from_dense(A, np.zeros(k - 1), lb, ub, np.ones(k))
    gl, gu, r = run_gpu(pkg.Problem(p), lb, ub)
    assert r["rounds"] == k and r["nnz_updates"] == 6 * k - 8 and r["status"] == 0
    np.testing.assert_array_equal(gu, np.zeros(k))


SWEEP = [
    # (seed, m, n, len_lo, len_hi, kwargs)
    (1, 50, 40, 1, 6, dict()),
    (2, 300, 200, 1, 40, dict(inf_fraction=0.2)),
    (3, 300, 500, 2, 12, dict(integer_coefs=True, int_fraction=1.0)),
    (4, 200, 300, 1, 30, dict(eq_fraction=0.3, inf_fraction=0.1)),
    (5, 120, 2000, 200, 1500, dict()),                 # warp rows and chunked rows, ragged tails
    (6, 60, 6000, 500, 5000, dict(integer_coefs=True)),
    (7, 400, 300, 0, 3, dict(empty_rows=20)),          # empty and single-nonzero rows
    (8, 500, 400, 1, 60, dict(neg_fraction=0.9, inf_fraction=0.3)),
    (9, 200, 300, 30, 300, dict(slack_scale=0.01)),
    (10, 1000, 800, 1, 20, dict(int_fraction=0.0)),    # all continuous
]


@pytest.mark.parametrize("case", SWEEP, ids=[f"s{c[0]}" for c in SWEEP])
@pytest.mark.parametrize("fix", [0, 10])
def test_random_sweep(pkg, case, fix):
    seed, m, n, lo, hi, kw = case
    p = synth.random_milp(seed, m, n, len_lo=lo, len_hi=hi, **kw)
    lb, ub = synth.tighten_random(seed, p, fix, planted=(seed % 2 == 0))
    ol, ou, orr, _ = oracle.Problem(p).bp(lb, ub)
    gl, gu, gr = run_gpu(pkg.Problem(p), lb, ub)
    feasible = fix == 0 or seed % 2 == 0          # the planted point is inside the start bounds
    if not compare(p, gl, gu, gr, ol, ou, orr, planted=p.x0 if feasible else None):
        pytest.skip(f"oracle reported {orr['fragile']} fragile decisions")


def test_round_limit_and_theta(pkg):
    p = synth.random_milp(11, 300, 200, len_lo=2, len_hi=20, int_fraction=0.0)
    for mr in (1, 2, 3):
        for theta in (0.0, 1e-3, 0.1):
            ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub, max_rounds=mr, theta=theta)
            gl, gu, gr = run_gpu(pkg.Problem(p), p.lb, p.ub, max_rounds=mr, theta=theta)
            compare(p, gl, gu, gr, ol, ou, orr)


def test_entry_crossing_and_empty(pkg):
    p = milp_from_dense(np.ones((1, 2)), [5.0], np.zeros(2), np.ones(2), [1, 0])
    gl, gu, r = run_gpu(pkg.Problem(p), [0.0, 2.0], [1.0, 1.0])
    assert r["status"] == 1 and r["rounds"] == 0 and r["first_infeasible_var"] == 1
    q = milp_from_dense(np.zeros((0, 3)), np.zeros(0), np.zeros(3), np.ones(3), [1, 1, 0])
    gl, gu, r = run_gpu(pkg.Problem(q), np.zeros(3), np.ones(3))
    assert r["status"] == 0 and r["rounds"] == 0 and r["nnz_updates"] == 0


def test_host_bounds_and_determinism(pkg):
    p = synth.random_milp(12, 2000, 3000, len_lo=1, len_hi=400, inf_fraction=0.05)
    prob = pkg.Problem(p)
    hl, hu = p.lb.copy(), p.ub.copy()
    hr = prob.propagate(hl, hu)                      # host arrays: library copies in/out
    gl, gu, gr = run_gpu(prob, p.lb, p.ub)
    gl2, gu2, gr2 = run_gpu(prob, p.lb, p.ub)
    assert hr == gr == gr2
    for a, b in ((hl, gl), (hu, gu), (gl2, gl), (gu2, gu)):
        assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_invalid_input_rejected(pkg):
    from paper_2510_20499_gb300.synth import Milp
    base = dict(m=1, n=2, g=np.array([1.0]), lb=np.zeros(2), ub=np.ones(2),
                is_int=np.ones(2, dtype=np.uint8), c=np.zeros(2))
    for rp, cl, vl in [([0, 2], [1, 0], [1.0, 1.0]), ([0, 2], [0, 5], [1.0, 1.0]), ([0, 2], [0, 1], [0.0, 1.0])]:
        q = Milp(row_ptr=np.array(rp, dtype=np.int64), col=np.array(cl, dtype=np.int32), val=np.array(vl), **base)
        with pytest.raises(pkg.GpuBpError) as e:
            pkg.Problem(q)
        assert e.value.code == pkg.BP_ERR_INVALID


@pytest.fixture(scope="module")
def mixed_big():
    p = synth.mixed_powerlaw()
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    return p, ol, ou, orr


def test_mixed_powerlaw_full_size(pkg, mixed_big):
    """The 200k x 500k, 5M-nonzero power-law instance (the benchmark workload), in the same
    launch configuration the benchmark times."""
    p, ol, ou, orr = mixed_big
    assert orr["fragile"] == 0
    gl, gu, gr = run_gpu(pkg.Problem(p), p.lb, p.ub)
    assert compare(p, gl, gu, gr, ol, ou, orr)


def test_mixed_powerlaw_infinite_bounds(pkg):
    p = synth.mixed_powerlaw(seed=77, m=20_000, n=50_000, nnz=500_000, max_row=20_000, inf_fraction=0.05)
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    gl, gu, gr = run_gpu(pkg.Problem(p), p.lb, p.ub)
    if not compare(p, gl, gu, gr, ol, ou, orr, planted=p.x0):
        pytest.skip("fragile")
