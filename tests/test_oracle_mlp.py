"""Pins of the scorer oracle (features, BF16 rounding, MLP forward/backward, loss, Adam) against
a library rounding routine, closed forms, finite differences and a hand-worked example."""
import math

import numpy as np
import pytest

from oracle import mlp
from tests.helpers import load_golden, milp_from_dense


def test_bf16_matches_library_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(50_000) * np.exp(rng.uniform(-85, 85, 50_000))).astype(np.float32)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 2.0 ** -130, 3 * 2.0 ** -134, 65535.0],
                    dtype=np.float32)
    x = np.concatenate([x, ties, np.float32([0.0, -0.0, np.inf, -np.inf, 3.0e38])]).astype(np.float64)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)
    assert mlp.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0          # tie to even
    assert mlp.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6


def test_forward_closed_form():
    """W1 = [I; -I; 0], W2 = I, W3 = [[1..1, 1..1], [1..1, -1..-1]]: H1 = [relu(x), relu(-x), 0],
    so Z3 = (sum |x| + b3_0, sum x + b3_1)."""
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][:16] = np.eye(16)
    d["W1"][16:32] = -np.eye(16)
    d["W2"] = np.eye(64)
    d["W3"][0, :32] = 1.0
    d["W3"][1, :16] = 1.0
    d["W3"][1, 16:32] = -1.0
    d["b3"] = np.array([0.5, -0.25])
    theta = mlp.pack(d)
    X = mlp.bf16(np.random.default_rng(3).integers(-8, 9, size=(40, 16)) / 4.0)
    Z3, _ = mlp.forward(theta, X)
    np.testing.assert_array_equal(Z3[:, 0], np.abs(X).sum(axis=1) + 0.5)
    np.testing.assert_array_equal(Z3[:, 1], X.sum(axis=1) - 0.25)


def test_forward_rounds_both_hidden_layers_to_bf16():
    """Each hidden layer is rounded to BF16 (8 significant bits) before the next layer: with
    x_0 = 1, W1[0, 0] = 1 and b1[0] = 2^-10, H1[0] = bf16(1 + 2^-10) = 1; with W2[0, 0] = 1 and
    b2[0] = 2^-10, H2[0] = bf16(1 + 2^-10) = 1 again; W3[0, 0] = 1 then gives Z3[0] = 1 exactly
    (without either rounding it would be 1 + 2^-10 or 1 + 2^-9)."""
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][0, 0] = 1.0
    d["b1"][0] = 2.0 ** -10
    d["W2"][0, 0] = 1.0
    d["b2"][0] = 2.0 ** -10
    d["W3"][0, 0] = 1.0
    X = np.zeros((1, 16))
    X[0, 0] = 1.0
    Z3, cache = mlp.forward(mlp.pack(d), X)
    assert cache["H1"][0, 0] == 1.0 and cache["H2"][0, 0] == 1.0
    assert Z3[0, 0] == 1.0
    Zf, _ = mlp.forward(mlp.pack(d), X, quantize=False)
    assert Zf[0, 0] == 1.0 + 2.0 ** -9


def test_loss_values():
    Z3 = np.zeros((4, 2))
    Y = np.array([[1, 0], [0, np.nan], [np.nan, np.nan], [1, 1]], dtype=float)
    loss, dz = mlp.loss_and_dz3(Z3, Y)
    assert loss == pytest.approx(2 * math.log(2.0))
    np.testing.assert_allclose(dz[:, 0], [-0.5 / 3, 0.5 / 3, 0.0, -0.5 / 3])
    np.testing.assert_allclose(dz[:, 1], [0.25, 0.0, 0.0, -0.25])


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    theta = rng.standard_normal(mlp.NPARAM) * 0.3
    X = rng.standard_normal((24, 16))
    Y = rng.integers(0, 2, size=(24, 2)).astype(float)
    Y[rng.random((24, 2)) < 0.25] = np.nan
    _, g = mlp.loss_grad(theta, X, Y, quantize=False)
    idx = rng.choice(mlp.NPARAM, size=300, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, mlp.NPARAM - 2, 0, 16 * 64 + 3]])   # biases and W1
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_grad(tp, X, Y, quantize=False)[0] - mlp.loss_grad(tm, X, Y, quantize=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_quantized_gradient_close_to_exact():
    rng = np.random.default_rng(12)
    theta = rng.standard_normal(mlp.NPARAM) * 0.3
    X = mlp.bf16(rng.standard_normal((256, 16)))
    Y = rng.integers(0, 2, size=(256, 2)).astype(float)
    _, gq = mlp.loss_grad(theta, X, Y)
    _, ge = mlp.loss_grad(theta, X, Y, quantize=False)
    assert np.linalg.norm(gq - ge) <= 0.05 * np.linalg.norm(ge)


def test_adam_closed_form():
    """First step: m^ = g, v^ = g^2, so the update is -lr g / (|g| + eps).  Second step with
    gradient h: m = 0.09 g + 0.1 h, v = 0.000999 g^2 + 0.001 h^2, bias corrections 0.19 and
    0.001999."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    h = np.array([1.0, 1.0, -1.0, 2.0])
    opt = mlp.Adam(4)
    t1 = opt.step(np.zeros(4), g, 0.1)
    np.testing.assert_allclose(t1, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    t2 = opt.step(t1, h, 0.1)
    m = (0.09 * g + 0.1 * h) / 0.19
    v = (0.000999 * g * g + 0.001 * h * h) / 0.001999
    np.testing.assert_allclose(t2, t1 - 0.1 * m / (np.sqrt(v) + 1e-8), rtol=1e-12)


def test_init_params_range():
    from oracle import uniform
    theta = mlp.init_params(7, uniform)
    P = mlp.unpack(theta)
    assert np.all(np.abs(P["W1"]) <= math.sqrt(6 / 16)) and np.all(np.abs(P["W2"]) <= math.sqrt(6 / 64))
    assert np.all(P["b1"] == 0) and np.all(P["b3"] == 0)
    assert abs(P["W2"].mean()) < 0.05 and P["W2"].std() == pytest.approx(math.sqrt(6 / 64) / math.sqrt(3), rel=0.1)


def test_features_hand_example():
    d = load_golden("scorer_features.json")
    p = milp_from_dense(d["A"], d["g"], d["lb"], d["ub"], d["is_int"])
    p.c = np.array(d["c"])
    F = mlp.raw_features(p, d["x"], d["lb"], d["ub"], [0, 1, 2], cache=d["cache"])
    np.testing.assert_allclose(F, np.array(d["features"], dtype=float), rtol=1e-12, atol=1e-12)


def test_features_infinite_bounds_excluded_from_slack():
    # x1 unbounded above with a negative coefficient: row 0's minimal activity is infinite, so
    # it contributes to neither S_0 nor S_1
    p = milp_from_dense([[1.0, -1.0], [2.0, 0.0]], [1.0, 3.0], [0, 0], [1, np.inf], [1, 0])
    F = mlp.raw_features(p, [0.5, 1.0], [0, 0], [1, np.inf], [0, 1])
    assert F[0, 14] == pytest.approx((2 / 3) ** 2) and F[1, 14] == 0.0
    assert F[1, 5] == pytest.approx(math.log1p(1e9))


def test_standardize():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((1000, 16)) * 5 + 3
    F[:, 7] = 1.0                                   # constant
    S = mlp.standardize(F)
    assert np.all(S[:, 7] == 0)
    np.testing.assert_allclose(S[:, :7].mean(axis=0), 0, atol=0.01)
    np.testing.assert_allclose(S[:, :7].std(axis=0), 1, atol=0.01)
    assert np.array_equal(S, mlp.bf16(S))


def test_training_reduces_loss():
    rng = np.random.default_rng(9)
    X = mlp.bf16(rng.standard_normal((512, 16)))
    Y = np.stack([(X[:, 0] + X[:, 1] > 0), (X[:, 2] - 0.5 * X[:, 3] > 0)], axis=1).astype(float)
    from oracle import uniform
    theta = mlp.init_params(3, uniform)
    opt = mlp.Adam(mlp.NPARAM)
    l0 = mlp.loss_grad(theta, X, Y)[0]
    for _ in range(150):
        loss, g = mlp.loss_grad(theta, X, Y)
        theta = opt.step(theta, g, 1e-2)
    assert loss < 0.3 * l0, (l0, loss)


def test_trajectory_labels_hand_worked():
    """x = (0.3, 0.5, 2.0, 6.7), two feasible runs fixing (0, 1, 2, 7) and (1, 1, 2, 6).
    Nearest integers floor(x + 1/2) = (0, 1, 2, 7): order labels (1/2, 1, 1, 1/2).  Fixed above
    x: (0, 1, -, 1) and (1, 1, -, 0): direction labels (1/2, 1, NaN, 1/2); x = 2 is integral.
    Only the listed variables (3, 0) are labelled, in that order."""
    x = np.array([0.3, 0.5, 2.0, 6.7])
    runs = [np.array([0.0, 1.0, 2.0, 7.0]), np.array([1.0, 1.0, 2.0, 6.0])]
    Y = mlp.trajectory_labels(x, runs, np.arange(4))
    np.testing.assert_array_equal(Y[:, 0], [0.5, 1.0, 1.0, 0.5])
    np.testing.assert_array_equal(Y[[0, 1, 3], 1], [0.5, 1.0, 0.5])
    assert np.isnan(Y[2, 1])
    np.testing.assert_array_equal(mlp.trajectory_labels(x, runs, [3, 0]), Y[[3, 0]])
    assert np.isnan(mlp.trajectory_labels(x, [], [0, 1])).all()


def test_bf16_flip_rows():
    """A pre-activation on a BF16 rounding boundary is flagged; one on a BF16 value with a small
    error bound is not.  Row 0: x = (1 + 2^-8, 0, ...) with W1[0, 0] = 1 gives exactly the
    midpoint between the BF16 neighbours 1 and 1 + 2^-7; row 1: x = (1, 0, ...) gives 1.  All
    other weights are 0, so every other pre-activation is 0 with a zero error bound."""
    theta = np.zeros(mlp.NPARAM)
    P = mlp.unpack(theta)
    P["W1"][0, 0] = 1.0
    theta = mlp.pack(P)
    X = np.zeros((2, mlp.IN))
    X[0, 0] = 1.0 + 2.0 ** -8
    X[1, 0] = 1.0
    np.testing.assert_array_equal(mlp.bf16_flip_rows(theta, X), [True, False])


def test_standardize_closed_form():
    """Population standardisation: a feature column (0, 2) has mean 1 and standard deviation 1,
    so it becomes (-1, 1) (the sample deviation sqrt(2) would give -0.707, 0.707)."""
    F = np.zeros((2, 16))
    F[:, 0] = [0.0, 2.0]
    S = mlp.standardize(F)
    np.testing.assert_array_equal(S[:, 0], [-1.0, 1.0])
    assert np.all(S[:, 1:] == 0)


def test_binary_flag_and_range_cap():
    """Feature 6 (binary) needs an integer variable with range at most 1: a continuous variable
    in [0, 1] has 0; feature 5 is log(1 + range) with the range capped at 1e9, also for a finite
    range of 1e12."""
    p = milp_from_dense([[1.0, 1.0, 1.0]], [5.0], [0, 0, 0], [1, 1, 1e12], [1, 0, 1])
    F = mlp.raw_features(p, [0.5, 0.5, 3.0], [0, 0, 0], [1, 1, 1e12], [0, 1, 2])
    assert list(F[:, 6]) == [1.0, 0.0, 0.0]
    assert F[2, 5] == math.log1p(1e9)
