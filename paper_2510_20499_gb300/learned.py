"""The learned rounding order of fix-and-propagate: trajectory collection, training and use.

No counterpart in the paper.  A 16-64-64-2 MLP (the library's `Scorer`) sees per-variable
features at the propagated start bounds and outputs an order score and the probability of
rounding up.  Training labels come from runs of the plain method (the paper's Section 2.3
order and rounding distribution) that ended feasible: column 0 is the share of those runs
that fixed the variable to the nearest integer of x, column 1 the share that fixed it above
x.  In use, the score ranks the integer variables within their class in place of the
per-bulk implied-slack order, and the up probability replaces the random band of the rounding
distribution; propagation still judges every fixing, and without a scorer the paper's order
is used.

Host orchestration only: every step runs in the library's kernels through the C ABI
(bp_propagate, scorer_features, fix_and_propagate, scorer_labels, scorer_train_step,
scorer_scores).  PyTorch holds the device buffers and draws the minibatch order.
"""
from __future__ import annotations

from . import Scorer, scorer_labels  # noqa: F401  (re-exported for callers)


def _torch():
    import torch
    return torch


def start_bounds(prob, lb, ub):
    """The propagated start bounds of fix-and-propagate (a copy of lb/ub, propagated)."""
    l, u = lb.clone(), ub.clone()
    r = prob.propagate(l, u)
    return l, u, r


def int_vars(prob):
    torch = _torch()
    return torch.tensor(prob.int_vars, dtype=torch.int32, device=prob.device)


def collect(prob, x, lb, ub, seeds, cache=None, **fp_kw):
    """Features and labels of one instance.  Runs plain fix_and_propagate once per seed and
    labels the integer variables from the runs that ended feasible.

    Returns dict(feat: nint x 16 BF16, labels: nint x 2 float32 or None when no run was
    feasible, feasible: count, runs: the result dicts)."""
    torch = _torch()
    l, u, _ = start_bounds(prob, lb, ub)
    iv = int_vars(prob)
    feat = prob.scorer_features(x, l, u, iv, cache=cache)
    outs, runs = [], []
    for s in seeds:
        xo, r = prob.fix_and_propagate(x, lb, ub, seed=int(s), cache=cache, **fp_kw)
        runs.append(r)
        if r["status"] == 0:
            outs.append(xo)
    labels = None
    if outs:
        labels = torch.empty((iv.numel(), 2), dtype=torch.float32, device=prob.device)
        for i, xo in enumerate(outs):
            scorer_labels(x, xo, iv, labels, weight=1.0 / len(outs), first=(i == 0))
    return dict(feat=feat, labels=labels, feasible=len(outs), runs=runs)


def train(scorer, data, epochs=6, batch=4096, lr=3e-3, seed=0):
    """Adam on the labelled rows of `data` (dicts from collect), in shuffled minibatches.
    Returns the mean batch loss of every epoch."""
    torch = _torch()
    rows = [d for d in data if d["labels"] is not None and d["feat"].shape[0] > 0]
    if not rows:
        return []
    X = torch.cat([d["feat"] for d in rows])
    Y = torch.cat([d["labels"] for d in rows])
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    losses = []
    for _ in range(int(epochs)):
        perm = torch.randperm(X.shape[0], generator=g).to(X.device)
        tot, nb = 0.0, 0
        for b in range(0, X.shape[0], batch):
            idx = perm[b:b + batch]
            tot += scorer.train_step(X.index_select(0, idx).contiguous(), Y.index_select(0, idx).contiguous(), lr)
            nb += 1
        losses.append(tot / nb)
    return losses


def scores(prob, scorer, x, lb, ub, cache=None):
    """The fix_and_propagate inputs (order_score, up_prob: float64 device tensors of n) that
    the scorer proposes for one instance."""
    torch = _torch()
    l, u, _ = start_bounds(prob, lb, ub)
    iv = int_vars(prob)
    order = torch.zeros(prob.n, dtype=torch.float64, device=prob.device)
    up = torch.full((prob.n,), 0.5, dtype=torch.float64, device=prob.device)
    if iv.numel():
        feat = prob.scorer_features(x, l, u, iv, cache=cache)
        scorer.scores(feat, iv, order, up)
    return order, up
