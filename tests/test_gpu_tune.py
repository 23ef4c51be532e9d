"""Row-class split points and grid shape (bp_set_tuning, bp_autotune): every configuration
computes the oracle's result; the autotuner keeps one whose results equal the defaults'."""
import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.gpu_helpers import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


CONFIGS = [(9, 257, 2, 256), (2, 2, 2, 256), (2, 65, 1, 64), (5, 129, 2, 128), (9, 9, 1, 32),
           (5, 257, 1, 256), (2, 257, 2, 32), (9, 65, 2, 64), (2, 257, 1, 128)]


def exact_problems():
    return [
        synth.binary_knapsack(),
        # every length class, integer data (exact sums): results must be bit-identical
        synth.random_milp(41, 600, 900, len_lo=1, len_hi=300, integer_coefs=True, int_fraction=1.0),
        synth.random_milp(42, 80, 6000, len_lo=2, len_hi=4000, integer_coefs=True, int_fraction=1.0),
    ]


def test_defaults(pkg):
    prob = pkg.Problem(synth.binary_knapsack())
    t = prob.get_tuning()
    assert t["warp_min"] == 2 and t["block_min"] == 257 and t["blocks_per_sm"] >= 1 and t["chunk_len"] == 256


@pytest.mark.parametrize("cfg", CONFIGS, ids=[f"w{c[0]}-b{c[1]}-g{c[2]}-c{c[3]}" for c in CONFIGS])
def test_every_configuration_matches_oracle(pkg, cfg):
    for p in exact_problems():
        lb, ub = synth.tighten_random(7, p, 12, planted=True)
        ol, ou, orr, _ = oracle.Problem(p).bp(lb, ub)
        prob = pkg.Problem(p)
        if cfg[2] > prob.get_tuning()["blocks_per_sm"]:
            pytest.skip("fewer resident blocks per SM on this device")
        prob.set_tuning(*cfg)
        assert prob.get_tuning() == dict(warp_min=cfg[0], block_min=cfg[1], blocks_per_sm=cfg[2], chunk_len=cfg[3])
        gl, gu, gr = run_gpu(prob, lb, ub)
        assert compare(p, gl, gu, gr, ol, ou, orr), "oracle saw a fragile decision on exact data"


def test_invalid_tuning_rejected(pkg):
    prob = pkg.Problem(synth.binary_knapsack())
    bps = prob.get_tuning()["blocks_per_sm"]
    for bad in [(1, 257, 1, 256), (10, 257, 1, 256), (9, 8, 1, 256), (9, 258, 1, 256), (9, 257, 0, 256),
                (9, 257, bps + 1, 256), (9, 257, 1, 300), (9, 257, 1, 512), (9, 257, 1, 2048), (9, 257, 1, 16)]:
        with pytest.raises(pkg.GpuBpError) as e:
            prob.set_tuning(*bad)
        assert e.value.code == pkg.BP_ERR_INVALID
    assert prob.get_tuning()["warp_min"] == 2


def test_autotune_single_keeps_results(pkg):
    import torch
    p = synth.random_milp(43, 3000, 4000, len_lo=1, len_hi=3000, inf_fraction=0.05, eq_fraction=0.2)
    prob = pkg.Problem(p)
    ol, ou, orr, _ = oracle.Problem(p).bp(p.lb, p.ub)
    before = run_gpu(prob, p.lb, p.ub)
    rep = prob.autotune(torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda"), reps=2)
    assert rep["tried"] >= 16 and rep["best_ms"] <= rep["default_ms"]
    assert prob.get_tuning() == rep["best"]
    after = run_gpu(prob, p.lb, p.ub)
    assert after[2] == before[2]
    if not orr["fragile"]:
        assert compare(p, *after, ol, ou, orr)


def test_autotune_batch_keeps_results(pkg):
    import torch
    parts = synth.uneven_batch(seed=77, count=16, nnz_lo=300, nnz_hi=40_000)
    big, ro, co = synth.block_diagonal(parts)
    prob = pkg.Problem(big)
    prob.set_instances(ro, co)
    lb0 = torch.tensor(big.lb, device="cuda")
    ub0 = torch.tensor(big.ub, device="cuda")
    lb, ub = lb0.clone(), ub0.clone()
    r0 = pkg.batch_results(prob.propagate_batch(lb, ub))
    b0 = (lb.cpu().numpy(), ub.cpu().numpy())
    rep = prob.autotune(lb0, ub0, reps=2)
    assert rep["tried"] >= 16
    lb, ub = lb0.clone(), ub0.clone()
    r1 = pkg.batch_results(prob.propagate_batch(lb, ub))
    assert r1 == r0
    ints = big.is_int == 1
    np.testing.assert_array_equal(lb.cpu().numpy()[ints], b0[0][ints])
    np.testing.assert_array_equal(ub.cpu().numpy()[ints], b0[1][ints])
    np.testing.assert_allclose(lb.cpu().numpy(), b0[0], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ub.cpu().numpy(), b0[1], rtol=1e-9, atol=1e-9)
