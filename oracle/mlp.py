"""Oracle of the learned rounding scorer: features, the 16-64-64-2 MLP, its loss, gradients and
Adam.  No counterpart in the paper: the scorer re-ranks the variables of bulk
fix-and-propagate (Section 2.3, Algorithm 1) and proposes the rounding direction of ambiguous
fractions; propagation still judges every fixing.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg, never by the library.
Plain NumPy in float64.  The GPU computes with BF16 operands and FP32 accumulation; this oracle
rounds to BF16 (round to nearest, ties to even) at exactly the same points and keeps every
other value in float64:
  forward:  X (features) -> H1 = bf16(relu(X W1q^T + b1)) -> H2 = bf16(relu(H1 W2q^T + b2))
            -> Z3 = H2 W3q^T + b3, with Wq = bf16(W) (weights are FP32 masters);
  backward: dZ3 = (sigmoid(Z3) - y) / (labels of that head), missing labels (NaN) give 0;
            dZ2q = bf16((dZ3 W3q) * [H2 > 0]), dZ1q = bf16((dZ2q W2q) * [H1 > 0]);
            dW3 = dZ3^T H2, dW2 = dZ2q^T H1, dW1 = dZ1q^T X, db = column sums of dZ3, dZ2q, dZ1q.

Parameter vector (5,378 floats): W1 [64 x 16], b1 [64], W2 [64 x 64], b2 [64], W3 [2 x 64],
b3 [2]; each weight matrix is [out x in], row-major.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 16, 64, 2
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
TOL = 1e-6
FEATURES = ["degree", "log_degree", "objective", "up_locks", "down_locks", "log_range", "is_binary", "is_int",
            "frac", "frac_dist_half", "cache_impl_down", "cache_impl_up", "cache_infeas_down", "cache_infeas_up",
            "implied_slack", "abs_coef_sum"]


def bf16(x):
    """Round float64 values to the nearest bfloat16 value (8 significant bits, exponent range of
    float32, subnormal spacing 2^-133), ties to even; values that round to 2^128 or beyond become
    +-inf, NaN stays NaN.  Returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.array(x, dtype=np.float64, copy=True)
    fin = np.isfinite(x) & (x != 0)
    _, e = np.frexp(x[fin])                 # x = m 2^e, 0.5 <= |m| < 1
    e = np.maximum(e, -125)                 # below 2^-126 the spacing stays 2^-133
    scale = np.ldexp(1.0, 8 - e)            # 8 significant bits
    r = np.rint(x[fin] * scale) / scale     # rint: ties to even
    r = np.where(np.abs(r) >= 2.0 ** 128, np.copysign(np.inf, r), r)
    out[fin] = r
    return out


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAM
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed, uniform):
    """He-uniform weights, zero biases: parameter i of matrix L (1-based) is
    (2u - 1) sqrt(6 / fan_in), u = uniform(seed, 1000 + L, i, 0) (the counter-based generator of
    the rounding draws)."""
    d = {}
    for L, (name, shape) in enumerate(SHAPES):
        if name.startswith("b"):
            d[name] = np.zeros(shape)
            continue
        layer = int(name[1])
        lim = math.sqrt(6.0 / shape[1])
        k = int(np.prod(shape))
        d[name] = np.array([(2.0 * uniform(seed, 1000 + layer, i, 0) - 1.0) * lim for i in range(k)]).reshape(shape)
    return pack(d)


def forward(theta, X, quantize=True):
    """Returns (Z3, cache) for features X [rows x 16] (already BF16 values)."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    P = unpack(theta)
    W1, W2, W3 = q(P["W1"]), q(P["W2"]), q(P["W3"])
    X = np.asarray(X, dtype=np.float64)
    H1 = q(np.maximum(X @ W1.T + P["b1"], 0.0))
    H2 = q(np.maximum(H1 @ W2.T + P["b2"], 0.0))
    Z3 = H2 @ W3.T + P["b3"]
    return Z3, dict(X=X, H1=H1, H2=H2, W1=W1, W2=W2, W3=W3)


def _gamma(k, u):
    return k * u / (1.0 - k * u)


def bf16_flip_rows(theta, X, u32=2.0 ** -22):
    """Rows whose forward pass may round a hidden value to the other neighbouring BF16 value on a
    device that accumulates in FP32: some pre-activation (X W1q^T + b1, or H1 W2q^T + b2) lies
    within the accumulation error bound of a BF16 rounding boundary.  The bound holds for any
    summation order (Higham, Lemma 3.4: |error| <= gamma_k sum |terms|, k = inputs + 1 for the
    bias), with u32 the unit roundoff assumed per FP32 operation (2^-22: twice round-to-nearest's,
    since a tensor core's accumulation rounding is not specified); BF16 x BF16 products are exact
    in FP32.  In the other rows both sides round every hidden value alike, and the outputs differ
    only by FP32 accumulation error.  Returns a bool array over rows."""
    q = bf16
    P = unpack(theta)
    W1, W2 = q(P["W1"]), q(P["W2"])
    X = np.asarray(X, dtype=np.float64)
    pre1 = X @ W1.T + P["b1"]
    w1 = _gamma(IN + 1, u32) * (np.abs(X) @ np.abs(W1).T + np.abs(P["b1"]))
    flip = (q(np.maximum(pre1 - w1, 0.0)) != q(np.maximum(pre1 + w1, 0.0))).any(axis=1)
    H1 = q(np.maximum(pre1, 0.0))
    pre2 = H1 @ W2.T + P["b2"]
    w2 = _gamma(HID + 1, u32) * (np.abs(H1) @ np.abs(W2).T + np.abs(P["b2"]))
    flip |= (q(np.maximum(pre2 - w2, 0.0)) != q(np.maximum(pre2 + w2, 0.0))).any(axis=1)
    return flip


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def loss_and_dz3(Z3, Y):
    """Binary cross-entropy with logits per head, averaged over that head's labels (NaN labels
    are missing); returns (loss, dL/dZ3)."""
    Y = np.asarray(Y, dtype=np.float64)
    valid = ~np.isnan(Y)
    cnt = valid.sum(axis=0)
    y = np.where(valid, Y, 0.0)
    # log(1 + e^z) - y z, computed stably
    per = np.maximum(Z3, 0.0) - Z3 * y + np.log1p(np.exp(-np.abs(Z3)))
    loss = 0.0
    dz = np.zeros_like(Z3)
    for h in range(Z3.shape[1]):
        if cnt[h] == 0:
            continue
        loss += per[valid[:, h], h].sum() / cnt[h]
        dz[:, h] = np.where(valid[:, h], (sigmoid(Z3[:, h]) - y[:, h]) / cnt[h], 0.0)
    return loss, dz


def backward(theta, cache, dZ3, quantize=True):
    """Gradient of the loss with respect to the parameter vector, given dL/dZ3."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    X, H1, H2 = cache["X"], cache["H1"], cache["H2"]
    W2, W3 = cache["W2"], cache["W3"]
    dZ2 = q((dZ3 @ W3) * (H2 > 0))
    dZ1 = q((dZ2 @ W2) * (H1 > 0))
    g = dict(W3=dZ3.T @ H2, b3=dZ3.sum(axis=0), W2=dZ2.T @ H1, b2=dZ2.sum(axis=0), W1=dZ1.T @ X,
             b1=dZ1.sum(axis=0))
    return pack(g)


def loss_grad(theta, X, Y, quantize=True):
    Z3, cache = forward(theta, X, quantize)
    loss, dz = loss_and_dz3(Z3, Y)
    return loss, backward(theta, cache, dz, quantize)


class Adam:
    """Adam (Kingma and Ba, 2015) with bias correction, in float64."""

    def __init__(self, n, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, theta, grad, lr):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mhat = self.m / (1 - self.b1 ** self.t)
        vhat = self.v / (1 - self.b2 ** self.t)
        return theta - lr * mhat / (np.sqrt(vhat) + self.eps)


# ------------------------------------------------------------------------------- features
def raw_features(p, x, lb, ub, vars_, cache=None):
    """The 16 raw features (FEATURES order) of the variables `vars_` under bounds lb/ub and the
    fractional point x.  cache: dict(var, status, offsets) of a probing cache (branch 2i is the
    down branch of pair i), or None.  Row activities: minimal activity over the row's terms with
    infinite contributions counted, not summed; the implied slack sum S_j uses the rows with no
    infinite term, slack = max(g - L_min, tol) (as in the rounding order of Section 2.3)."""
    m, n = p.m, p.n
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    row_of = np.repeat(np.arange(m), np.diff(p.row_ptr))
    col = np.asarray(p.col, dtype=np.int64)
    a = np.asarray(p.val, dtype=np.float64)
    bnd = np.where(a > 0, lb[col], ub[col])
    inf = ~np.isfinite(bnd) | (np.abs(bnd) >= 1e20)
    minfin = np.bincount(row_of, weights=np.where(inf, 0.0, a * np.where(inf, 0.0, bnd)), minlength=m)
    ninf = np.bincount(row_of, weights=inf.astype(np.float64), minlength=m)
    g = np.asarray(p.g, dtype=np.float64)
    ok = (ninf == 0) & np.isfinite(g) & (g < 1e20)
    slack = np.where(ok, np.maximum(g - minfin, TOL), 1.0)
    s_term = np.where(ok[row_of], (a / slack[row_of]) ** 2, 0.0)
    deg = np.bincount(col, minlength=n).astype(np.float64)
    upl = np.bincount(col, weights=(a > 0).astype(np.float64), minlength=n)
    dnl = np.bincount(col, weights=(a < 0).astype(np.float64), minlength=n)
    S = np.bincount(col, weights=s_term, minlength=n)
    absum = np.bincount(col, weights=np.abs(a), minlength=n)
    v = np.asarray(vars_, dtype=np.int64)
    rng = ub[v] - lb[v]
    rng = np.where(~np.isfinite(rng) | (rng > 1e9), 1e9, rng)
    frac = x[v] - np.floor(x[v])
    is_i = (np.asarray(p.is_int)[v] != 0).astype(np.float64)
    c = np.asarray(p.c, dtype=np.float64)[v] if getattr(p, "c", None) is not None else np.zeros(len(v))
    out = np.zeros((len(v), 16))
    out[:, 0] = deg[v]
    out[:, 1] = np.log1p(deg[v])
    out[:, 2] = c
    out[:, 3] = upl[v]
    out[:, 4] = dnl[v]
    out[:, 5] = np.log1p(rng)
    out[:, 6] = ((is_i == 1.0) & (rng <= 1.0)).astype(np.float64)
    out[:, 7] = is_i
    out[:, 8] = frac
    out[:, 9] = np.abs(frac - 0.5)
    out[:, 14] = S[v]
    out[:, 15] = absum[v]
    if cache is not None:
        pair_of = {}
        for i, w in enumerate(np.asarray(cache["var"])):
            pair_of.setdefault(int(w), i)
        off = np.asarray(cache["offsets"])
        st = np.asarray(cache["status"])
        for r, j in enumerate(v):
            i = pair_of.get(int(j))
            if i is None:
                continue
            out[r, 10] = float(off[2 * i + 1] - off[2 * i])
            out[r, 11] = float(off[2 * i + 2] - off[2 * i + 1])
            out[r, 12] = float(st[2 * i] == 1)
            out[r, 13] = float(st[2 * i + 1] == 1)
    return out


def standardize(F):
    """Per-feature standardisation over the given variables (population variance; a constant
    feature becomes 0), then BF16."""
    F = np.asarray(F, dtype=np.float64)
    mean = F.mean(axis=0)
    std = np.sqrt(((F - mean) ** 2).mean(axis=0))
    std = np.where(std < 1e-12, 1.0, std)
    return bf16((F - mean) / std)


def features(p, x, lb, ub, vars_, cache=None):
    return standardize(raw_features(p, x, lb, ub, vars_, cache))


# ------------------------------------------------------------------------------- labels
def trajectory_labels(x, x_outs, vars_):
    """Training labels of the variables `vars_` from the results x_out of fix-and-propagate runs
    that ended feasible (all integer variables fixed, propagation feasible).  Column 0: the share
    of runs that fixed the variable to the nearest integer of x, floor(x + 1/2) (the order label:
    a variable whose nearest value holds is fixed early).  Column 1: the share of runs that fixed
    it above x (the rounding-direction label); NaN (no label) where x is integral.  With no run
    both columns are NaN."""
    v = np.asarray(vars_, dtype=np.int64)
    xv = np.asarray(x, dtype=np.float64)[v]
    Y = np.zeros((len(v), 2))
    if len(x_outs) == 0:
        Y[:] = np.nan
        return Y
    w = 1.0 / len(x_outs)
    near = np.floor(xv + 0.5)
    for xo in x_outs:
        fixed = np.asarray(xo, dtype=np.float64)[v]
        Y[:, 0] += w * (fixed == near)
        Y[:, 1] += w * (fixed > xv)
    Y[xv == np.floor(xv), 1] = np.nan
    return Y
