"""Batched propagation of uneven instances (bp_propagate_batch) against independent oracle runs."""
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


def _batch(count, seed, lo=300, hi=30_000, infeasible=()):
    parts = synth.uneven_batch(seed=seed, count=count, nnz_lo=lo, nnz_hi=hi)
    for i in infeasible:
        # tighten one instance until it is infeasible: fix variables far from the planted point
        q = parts[i]
        rng = np.random.default_rng(i)
        for j in rng.choice(q.n, size=max(1, q.n // 3), replace=False):
            q.lb[j] = q.ub[j] = q.ub[j] if q.x0[j] < q.ub[j] / 2 else q.lb[j]
    big, ro, co = synth.block_diagonal(parts)
    return parts, big, ro, co


def _run(pkg, big, ro, co, lb, ub, **kw):
    import torch
    prob = pkg.Problem(big)
    prob.set_instances(ro, co)
    gl = torch.tensor(lb, device="cuda")
    gu = torch.tensor(ub, device="cuda")
    res = prob.propagate_batch(gl, gu, **kw)
    torch.cuda.synchronize()
    return gl.cpu().numpy(), gu.cpu().numpy(), pkg.batch_results(res), prob


def _compare_instances(parts, ro, co, gl, gu, gres, **kw):
    for i, q in enumerate(parts):
        ol, ou, orr, _ = oracle.Problem(q).bp(q.lb, q.ub, **kw)
        g = gres[i]
        if orr["fragile"]:
            continue
        assert g["error"] == 0
        for key in ("status", "rounds", "nnz_updates", "n_changed"):
            assert g[key] == orr[key], (i, key, g[key], orr[key])
        for key, off in (("first_infeasible_row", ro[i]), ("first_infeasible_var", co[i])):
            want = orr[key] + off if orr[key] >= 0 else -1
            assert g[key] == want, (i, key)
        assert_bounds_match(q, gl[co[i]:co[i + 1]], gu[co[i]:co[i + 1]], ol, ou)


def test_uneven_batch_matches_independent_runs(pkg):
    parts, big, ro, co = _batch(24, seed=123, infeasible=(3, 10))
    gl, gu, gres, _ = _run(pkg, big, ro, co, big.lb, big.ub)
    assert any(r["status"] == 1 for r in gres)
    _compare_instances(parts, ro, co, gl, gu, gres)


def test_batch_round_limit(pkg):
    parts, big, ro, co = _batch(10, seed=7)
    gl, gu, gres, _ = _run(pkg, big, ro, co, big.lb, big.ub, max_rounds=2)
    _compare_instances(parts, ro, co, gl, gu, gres, max_rounds=2)


def test_single_instance_batch_equals_plain(pkg):
    import torch
    p = synth.random_milp(8, 500, 600, len_lo=1, len_hi=50)
    gl, gu, gres, prob = _run(pkg, p, [0, p.m], [0, p.n], p.lb, p.ub)
    hl = torch.tensor(p.lb, device="cuda")
    hu = torch.tensor(p.ub, device="cuda")
    r = prob.propagate(hl, hu)
    assert gres[0] == r
    assert np.array_equal(hl.cpu().numpy(), gl) and np.array_equal(hu.cpu().numpy(), gu)


def test_graph_captured_batch(pkg):
    """The batched call captured in a CUDA graph and replayed gives the same results each time
    (the stamp base advances on the device)."""
    import torch
    parts, big, ro, co = _batch(16, seed=99)
    prob = pkg.Problem(big)
    prob.set_instances(ro, co)
    lb0 = torch.tensor(big.lb, device="cuda")
    ub0 = torch.tensor(big.ub, device="cuda")
    lb, ub = lb0.clone(), ub0.clone()
    res = torch.empty(16 * 12, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        prob.propagate_batch(lb, ub, results=res)      # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lb.copy_(lb0)
        ub.copy_(ub0)
        prob.propagate_batch(lb, ub, results=res)
    outs = []
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        outs.append((lb.cpu().numpy().copy(), ub.cpu().numpy().copy(), pkg.batch_results(res)))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1]) and o[2] == outs[0][2]
    _compare_instances(parts, ro, co, outs[0][0], outs[0][1], outs[0][2])


def test_set_instances_rejects_crossing_rows(pkg):
    parts, big, ro, co = _batch(3, seed=1, lo=100, hi=300)
    prob = pkg.Problem(big)
    with pytest.raises(pkg.GpuBpError):
        prob.set_instances(ro, [0, co[2], co[1] + 1, co[3]] if co[2] > co[1] + 1 else [0, 1, 2, co[3]])


def test_uneven_batch_full_size_autotuned(pkg):
    """The benchmark's batch (64 instances, nnz log-uniform in [1e3, 5e5], 5.4M nonzeros) in
    the configurations the benchmark times: the default split points and the ones bp_autotune
    picks.  Every instance against its own oracle run."""
    import torch
    parts = synth.uneven_batch()
    big, ro, co = synth.block_diagonal(parts)
    prob = pkg.Problem(big)
    prob.set_instances(ro, co)
    lb0 = torch.tensor(big.lb, device="cuda")
    ub0 = torch.tensor(big.ub, device="cuda")

    def run():
        gl, gu = lb0.clone(), ub0.clone()
        res = prob.propagate_batch(gl, gu)
        torch.cuda.synchronize()
        return gl.cpu().numpy(), gu.cpu().numpy(), pkg.batch_results(res)

    gl, gu, gres = run()
    _compare_instances(parts, ro, co, gl, gu, gres)
    prob.autotune(lb0, ub0, reps=1)
    gl2, gu2, gres2 = run()
    # the tuned piece length may sum rows in another order: every decision is the same, integer
    # bounds are identical and continuous bounds agree within the 1e-9 relative tolerance
    assert gres2 == gres
    ints = big.is_int == 1
    np.testing.assert_array_equal(gl2[ints], gl[ints])
    np.testing.assert_array_equal(gu2[ints], gu[ints])
    np.testing.assert_allclose(gl2, gl, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gu2, gu, rtol=1e-9, atol=1e-9)
    _compare_instances(parts, ro, co, gl2, gu2, gres2)
