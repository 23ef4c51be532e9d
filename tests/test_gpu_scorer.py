"""The learned scorer on the GPU (tcgen05 MLP, features, gradient, Adam) against the oracle."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2510_20499_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def bf16_tensor(X):
    import torch
    return torch.tensor(np.asarray(X, dtype=np.float32), device="cuda").to(torch.bfloat16)


def random_theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(mlp.NPARAM) * scale).astype(np.float32)


def test_closed_form_network_is_exact(pkg):
    """W1 = [I; -I; 0], W2 = I, W3 = [[1..1, 1..1], [1..1, -1..-1]]: the logits are
    sum |x| + 0.5 and sum x - 0.25 exactly (small multiples of 1/4): every operand layout,
    descriptor and accumulator column must be right.  1000 rows: 7 full tiles and a ragged one."""
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][:16] = np.eye(16)
    d["W1"][16:32] = -np.eye(16)
    d["W2"] = np.eye(64)
    d["W3"][0, :32] = 1.0
    d["W3"][1, :16] = 1.0
    d["W3"][1, 16:32] = -1.0
    d["b3"] = np.array([0.5, -0.25])
    theta = mlp.pack(d).astype(np.float32)
    X = np.random.default_rng(3).integers(-8, 9, size=(1000, 16)) / 4.0
    s = pkg.Scorer()
    s.set_params(theta)
    z = s.forward(bf16_tensor(X)).cpu().numpy()
    np.testing.assert_array_equal(z[:, 0], np.abs(X).sum(axis=1) + 0.5)
    np.testing.assert_array_equal(z[:, 1], X.sum(axis=1) - 0.25)


def grid_case(seed, rows):
    """Parameters and features on dyadic grids small enough that every product and every partial
    sum of both hidden layers is exact in FP32, in any order: X = k/16 (|k| <= 32), W1 = j/64
    (|j| <= 8), b1 = i/1024 (|pre-activation| <= 4.25, multiples of 2^-10), W2 = j/64 (|j| <= 16),
    b2 = i/2^16 (|pre-activation| <= 69, multiples of 2^-16, below 2^7 = 2^23 units).  Both sides
    then round every hidden value alike, and the outputs differ only by FP32 accumulation error
    in the last layer."""
    rng = np.random.default_rng(seed)
    P = {"W1": rng.integers(-8, 9, (64, 16)) / 64.0, "b1": rng.integers(-256, 257, 64) / 1024.0,
         "W2": rng.integers(-16, 17, (64, 64)) / 64.0, "b2": rng.integers(-4096, 4097, 64) / 65536.0,
         "W3": rng.integers(-16, 17, (2, 64)) / 64.0, "b3": rng.standard_normal(2).astype(np.float32).astype(np.float64)}
    theta = mlp.pack(P).astype(np.float32)
    assert (theta.astype(np.float64) == mlp.pack(P)).all()
    X = rng.integers(-32, 33, (rows, 16)) / 16.0
    return theta, X


def test_forward_exact_grid(pkg):
    """Every row agrees with the oracle to FP32 accuracy (1e-5 relative): on the grid no hidden
    value can round differently, so no row is exempt."""
    theta, X = grid_case(23, 3001)
    s = pkg.Scorer()
    s.set_params(theta)
    z = s.forward(bf16_tensor(X)).cpu().numpy().astype(np.float64)
    zo, _ = mlp.forward(theta.astype(np.float64), X)
    rel = np.abs(z - zo) / (1.0 + np.abs(zo))
    assert rel.max() < 1e-5, rel.max()


def test_forward_matches_oracle(pkg):
    """Random features and parameters: every row agrees within 1e-3 relative except rows where the
    oracle shows that a hidden value may round to the other BF16 neighbour under FP32
    accumulation (mlp.bf16_flip_rows); their number is reported."""
    rng = np.random.default_rng(21)
    theta = random_theta(21)
    X = mlp.bf16(rng.standard_normal((1537, 16)))
    s = pkg.Scorer()
    s.set_params(theta)
    z = s.forward(bf16_tensor(X)).cpu().numpy().astype(np.float64)
    zo, _ = mlp.forward(theta.astype(np.float64), X)
    rel = (np.abs(z - zo) / (1.0 + np.abs(zo))).max(axis=1)
    flip = mlp.bf16_flip_rows(theta.astype(np.float64), X)
    print(f"\nrows that may round a hidden value differently: {int(flip.sum())} of {len(flip)}; "
          f"largest difference elsewhere {rel[~flip].max() if (~flip).any() else 0.0:.2e}, "
          f"in those rows {rel[flip].max() if flip.any() else 0.0:.2e}")
    assert (rel[~flip] <= 1e-3).all(), rel[~flip].max()


def test_empty_and_single_row(pkg):
    import torch
    s = pkg.Scorer()
    s.set_params(random_theta(5))
    out = s.forward(torch.empty((0, 16), dtype=torch.bfloat16, device="cuda"))
    assert out.shape == (0, 2)
    X = mlp.bf16(np.random.default_rng(6).standard_normal((1, 16)))
    z = s.forward(bf16_tensor(X)).cpu().numpy()
    zo, _ = mlp.forward(random_theta(5).astype(np.float64), X)
    np.testing.assert_allclose(z, zo, rtol=2e-2, atol=2e-2)


def labels_for(X, rng, missing=0.2):
    Y = np.stack([(X[:, 0] + X[:, 1] > 0), (X[:, 2] - 0.5 * X[:, 3] > 0)], axis=1).astype(np.float32)
    Y[rng.random(Y.shape) < missing] = np.nan
    return Y


def test_gradient_matches_oracle(pkg):
    import torch
    rng = np.random.default_rng(31)
    theta = random_theta(31, 0.2)
    X = mlp.bf16(rng.standard_normal((1000, 16)))
    Y = labels_for(X, rng)
    s = pkg.Scorer()
    s.set_params(theta)
    g, loss = s.gradient(bf16_tensor(X), torch.tensor(Y, device="cuda"))
    lo, go = mlp.loss_grad(theta.astype(np.float64), X, Y.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-3)
    o = 0
    for name, shape in mlp.SHAPES:
        k = int(np.prod(shape))
        a, b = g[o:o + k].astype(np.float64), go[o:o + k]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-7, (name, np.linalg.norm(a - b), np.linalg.norm(b))
        o += k
    assert np.linalg.norm(g - go) <= 1e-2 * np.linalg.norm(go)


def test_gradient_directional_finite_difference(pkg):
    """Central difference of the GPU loss along a direction that moves every parameter by 2%
    (well above one BF16 unit) against the GPU gradient."""
    import torch
    rng = np.random.default_rng(41)
    theta = random_theta(41, 0.2)
    X = mlp.bf16(rng.standard_normal((2048, 16)))
    Y = torch.tensor(labels_for(X, rng, 0.0), device="cuda")
    Xg = bf16_tensor(X)
    s = pkg.Scorer()
    s.set_params(theta)
    g, _ = s.gradient(Xg, Y)
    d = (np.sign(rng.standard_normal(mlp.NPARAM)) * np.abs(theta) * 0.02).astype(np.float32)
    s.set_params(theta + d)
    _, lp = s.gradient(Xg, Y)
    s.set_params(theta - d)
    _, lm = s.gradient(Xg, Y)
    fd = (lp - lm) / 2.0
    an = float(np.dot(g.astype(np.float64), d))
    assert abs(fd - an) <= 0.1 * abs(an) + 1e-5, (fd, an)


def test_adam_step_matches_oracle(pkg):
    import torch
    rng = np.random.default_rng(51)
    theta = random_theta(51, 0.2)
    X = mlp.bf16(rng.standard_normal((640, 16)))
    Y = torch.tensor(labels_for(X, rng), device="cuda")
    Xg = bf16_tensor(X)
    s = pkg.Scorer()
    s.set_params(theta)
    opt = mlp.Adam(mlp.NPARAM)
    want = theta.astype(np.float64)
    for _ in range(3):
        g, _ = s.gradient(Xg, Y)
        s.train_step(Xg, Y, 1e-2)
        want = opt.step(want, g.astype(np.float64), 1e-2)
        got = s.get_params().astype(np.float64)
        np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)
        want = got      # continue from the GPU's float32 parameters


def test_training_reduces_loss(pkg):
    import torch
    rng = np.random.default_rng(61)
    X = mlp.bf16(rng.standard_normal((4096, 16)))
    Y = torch.tensor(labels_for(X, rng, 0.0), device="cuda")
    Xg = bf16_tensor(X)
    s = pkg.Scorer(seed=3)
    l0 = s.train_step(Xg, Y, 1e-2)
    for _ in range(200):
        loss = s.train_step(Xg, Y, 1e-2)
    assert loss < 0.3 * l0, (l0, loss)


def test_save_load_roundtrip(pkg):
    s = pkg.Scorer(seed=9)
    theta = s.get_params()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "scorer.bin")
        s.save(path)
        t = pkg.Scorer(seed=10)
        t.load(path)
        np.testing.assert_array_equal(t.get_params(), theta)
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(pkg.GpuBpError):
            t.load(path)


def test_init_matches_oracle_definition(pkg):
    s = pkg.Scorer(seed=7)
    want = mlp.init_params(7, oracle.uniform)
    np.testing.assert_allclose(s.get_params(), want, rtol=1e-6, atol=1e-7)


def test_features_match_oracle(pkg):
    import torch
    p = synth.random_milp(71, 600, 900, len_lo=1, len_hi=40, inf_fraction=0.05, eq_fraction=0.2)
    rng = np.random.default_rng(71)
    x = np.clip(p.x0 + rng.normal(0, 0.3, p.n), p.lb, np.minimum(p.ub, 1e6))
    prob = pkg.Problem(p)
    lb = torch.tensor(p.lb, device="cuda")
    ub = torch.tensor(p.ub, device="cuda")
    ints = np.flatnonzero(p.is_int == 1).astype(np.int32)
    # probing cache on 40 integer variables
    pv = ints[:40]
    boxes = np.array([oracle.probe_split(1, p.lb[j], p.ub[j]) for j in pv])
    c = prob.probe_batch(lb, ub, torch.tensor(pv, device="cuda"), torch.tensor(boxes, device="cuda"))
    c["pairs"] = torch.tensor(pv, device="cuda")
    c["boxes"] = torch.tensor(boxes, device="cuda")
    feat = prob.scorer_features(torch.tensor(x, device="cuda"), lb, ub, torch.tensor(ints, device="cuda"), cache=c)
    got = feat.float().cpu().numpy().astype(np.float64)
    cache_h = dict(var=pv, status=c["status"].cpu().numpy(), offsets=c["offsets"].cpu().numpy())
    want = mlp.features(p, x, p.lb, p.ub, ints, cache=cache_h)
    diff = np.abs(got - want)
    ulp = np.maximum(np.abs(want), 2.0 ** -126) * 2.0 ** -7
    assert np.all(diff <= ulp), np.argwhere(diff > ulp)[:5]
    assert np.mean(diff == 0) > 0.99


def test_scores_scatter(pkg):
    import torch
    s = pkg.Scorer(seed=2)
    X = mlp.bf16(np.random.default_rng(8).standard_normal((300, 16)))
    vars_ = torch.tensor(np.random.default_rng(9).permutation(1000)[:300].astype(np.int32), device="cuda")
    order = torch.full((1000,), -7.0, dtype=torch.float64, device="cuda")
    up = torch.full((1000,), -7.0, dtype=torch.float64, device="cuda")
    logits = s.scores(bf16_tensor(X), vars_, order, up)
    v = vars_.cpu().numpy()
    z = logits.cpu().numpy().astype(np.float64)
    o, u = order.cpu().numpy(), up.cpu().numpy()
    np.testing.assert_array_equal(o[v], z[:, 0])
    np.testing.assert_allclose(u[v], 1 / (1 + np.exp(-z[:, 1])), rtol=1e-12)
    rest = np.setdiff1d(np.arange(1000), v)
    assert np.all(o[rest] == -7.0) and np.all(u[rest] == -7.0)


@pytest.mark.parametrize("runs", [1, 2, 4])
def test_labels_match_oracle(pkg, runs):
    """scorer_labels over `runs` feasible results against the oracle's trajectory labels
    (weights 1, 1/2, 1/4: the float32 sums are exact)."""
    import torch
    rng = np.random.default_rng(runs)
    n = 3000
    x = np.where(rng.random(n) < 0.2, rng.integers(0, 5, n).astype(float), rng.uniform(0, 5, n))
    x[:8] = [0.5, 1.5, 2.0, 0.49999999999999994, 3.5, 4.0, 0.25, 0.75]    # ties and integral values
    outs = [np.floor(x) + (rng.random(n) < 0.5) for _ in range(runs)]
    vars_ = rng.permutation(n)[:2500].astype(np.int32)
    want = mlp.trajectory_labels(x, outs, vars_)
    xd = torch.tensor(x, device="cuda")
    vd = torch.tensor(vars_, device="cuda")
    lab = torch.full((len(vars_), 2), 7.0, dtype=torch.float32, device="cuda")
    for i, o in enumerate(outs):
        pkg.scorer_labels(xd, torch.tensor(o, device="cuda"), vd, lab, weight=1.0 / runs, first=(i == 0))
    got = lab.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    np.testing.assert_array_equal(got[~np.isnan(got)], want[~np.isnan(want)])


def test_checkpoint_resumes_training(pkg):
    """Three Adam steps, save, load into a fresh scorer, three more steps: the same parameters as
    six steps without the interruption (the training step is deterministic)."""
    import torch
    rng = np.random.default_rng(71)
    X = bf16_tensor(rng.standard_normal((1000, 16)))
    Y = torch.tensor(labels_for(mlp.bf16(rng.standard_normal((1000, 16))), rng), device="cuda")
    a = pkg.Scorer(seed=4)
    for _ in range(6):
        a.train_step(X, Y, 1e-2)
    b = pkg.Scorer(seed=4)
    for _ in range(3):
        b.train_step(X, Y, 1e-2)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ckpt.bin")
        b.save(path)
        c = pkg.Scorer(seed=99)
        c.load(path)
    for _ in range(3):
        c.train_step(X, Y, 1e-2)
    np.testing.assert_array_equal(c.get_params(), a.get_params())
