"""Failure detection without a GPU fault, and determinism.

Every device-side wait of the propagation kernel gives up after a bounded spin and reports
BP_ERR_TIMEOUT through the result.  The test makes one block leave the rounds without arriving
at the grid barrier (a test-only environment variable read at launch), so the other blocks'
waits run out; the launch must end by itself with that status, and the same handle must then
propagate correctly.  The persistent local search is tested the same way.  Nothing faults or
traps the device."""
import time

import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.gpu_helpers import assert_bounds_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def _dev(p):
    import torch
    return torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda")


def test_barrier_timeout_is_reported_and_the_handle_recovers(pkg, monkeypatch):
    p = synth.random_milp(404, 3000, 5000, len_lo=1, len_hi=60, integer_coefs=True, int_fraction=0.8)
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    assert orr["rounds"] >= 2
    prob = pkg.Problem(p)
    monkeypatch.setenv("GPUBP_TEST_SKIP_BLOCK", "5")
    lb, ub = _dev(p)
    t0 = time.time()
    r = prob.propagate(lb, ub)
    assert r["error"] == pkg.BP_ERR_TIMEOUT, r
    assert time.time() - t0 < 60
    monkeypatch.delenv("GPUBP_TEST_SKIP_BLOCK")
    lb, ub = _dev(p)
    r = prob.propagate(lb, ub)
    assert r["error"] == 0
    for key in ("status", "rounds", "nnz_updates", "n_changed"):
        assert r[key] == orr[key], (key, r[key], orr[key])
    assert_bounds_match(p, lb.cpu().numpy(), ub.cpu().numpy(), ol, ou)


def test_repeated_runs_are_bit_identical(pkg):
    """Ten propagations of a 500k-nonzero mixed instance (chunked rows, continuous bounds):
    every result field and every bound bit-identical, and the same as the oracle's verdict."""
    p = synth.mixed_powerlaw(seed=91, m=20_000, n=50_000, nnz=500_000, max_row=20_000)
    prob = pkg.Problem(p)
    runs = []
    for _ in range(10):
        lb, ub = _dev(p)
        r = prob.propagate(lb, ub)
        runs.append((r, lb.cpu().numpy().view(np.int64), ub.cpu().numpy().view(np.int64)))
    r0, l0, u0 = runs[0]
    assert r0["error"] == 0
    for r, l, u in runs[1:]:
        assert r == r0
        np.testing.assert_array_equal(l, l0)
        np.testing.assert_array_equal(u, u0)
    _, _, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    if orr["fragile"] == 0:
        assert (r0["status"], r0["rounds"], r0["nnz_updates"]) == (orr["status"], orr["rounds"], orr["nnz_updates"])


def test_local_search_barrier_timeout_is_reported_and_the_search_recovers(pkg, monkeypatch):
    """The persistent local search's grid barriers wait boundedly too: with one block leaving
    the search without arriving, the call ends by itself with BP_ERR_TIMEOUT, and the same handle
    then searches exactly as the oracle does."""
    import torch
    from oracle import local_mip as lm
    p = synth.knapsack_cover(seed=91, m=2000, n=4000, nnz=40_000)
    x0 = np.clip((np.random.default_rng(3).random(p.n) < 0.5).astype(float), p.lb, p.ub)
    prob = pkg.Problem(p)
    lb, ub = _dev(p)
    monkeypatch.setenv("GPUBP_TEST_SKIP_BLOCK", "5")
    x = torch.tensor(x0, device="cuda")
    w = torch.ones(p.m, dtype=torch.float64, device="cuda")
    t0 = time.time()
    with pytest.raises(pkg.GpuBpError) as err:
        prob.local_search(lb, ub, x, w, iterations=20)
    assert err.value.code == pkg.BP_ERR_TIMEOUT
    assert time.time() - t0 < 60
    monkeypatch.delenv("GPUBP_TEST_SKIP_BLOCK")
    x = torch.tensor(x0, device="cuda")
    w = torch.ones(p.m, dtype=torch.float64, device="cuda")
    r = prob.local_search(lb, ub, x, w, iterations=20)
    ox, ow, orr = lm.search(p, p.lb, p.ub, x0, np.ones(p.m), 20)
    np.testing.assert_array_equal(x.cpu().numpy(), ox)
    np.testing.assert_array_equal(w.cpu().numpy(), ow)
    assert r["moves"] == orr["moves"]
