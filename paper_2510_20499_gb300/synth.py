"""Seeded synthetic MILP instances shaped like the paper's workloads.

The paper measures on MIPLIB2017 (Section 3), which is not available here; these
generators stand in for it.  They build problems in the paper's form (Section 1):
rows ``sum_i a_ki x_i <= g_k``, bounds ``l <= x <= u``, some variables integer.  The
module holds no propagation arithmetic: it only draws instances, and both the GPU path
and the CPU oracle read the arrays it returns.

Every generator takes an integer seed and uses numpy's PCG64 generator, so an instance is
a pure function of (generator, seed, sizes).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2510020499


@dataclasses.dataclass
class Milp:
    """A MILP ``min c.x  s.t.  A x <= g,  lb <= x <= ub,  x_j integer where is_int[j]``.

    A is in CSR form: ``row_ptr`` (int64, m+1), ``col`` (int32, nnz, strictly increasing
    within a row), ``val`` (float64, nnz).  Infinite bounds are +-inf.
    """
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    g: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    is_int: np.ndarray
    c: np.ndarray
    x0: np.ndarray | None = None   # planted feasible point, when the generator has one
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _dedup_columns(rng, row_of, n, cols):
    """Redraws repeated columns inside a row until every row's columns are distinct,
    then sorts each row's columns ascending.  row_of is nondecreasing."""
    cols = cols.astype(np.int64)
    while True:
        key = row_of.astype(np.int64) * n + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(len(ks), dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            break
        idx = order[dup]
        cols[idx] = rng.integers(0, n, size=len(idx))
    key = row_of.astype(np.int64) * n + cols
    order = np.argsort(key, kind="stable")
    return cols[order].astype(np.int32)


def _csr_from_lengths(rng, lengths, n):
    lengths = np.asarray(lengths, dtype=np.int64)
    row_ptr = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    row_of = np.repeat(np.arange(len(lengths), dtype=np.int64), lengths)
    cols = rng.integers(0, n, size=nnz)
    cols = _dedup_columns(rng, row_of, n, cols)
    return row_ptr, cols, row_of


def _fix_total(rng, lengths, target, lo=1, hi=None):
    """Adds or removes single nonzeros on random rows until sum(lengths) == target."""
    lengths = lengths.copy()
    diff = int(target - lengths.sum())
    while diff != 0:
        k = int(rng.integers(0, len(lengths)))
        if diff > 0 and (hi is None or lengths[k] < hi):
            lengths[k] += 1
            diff -= 1
        elif diff < 0 and lengths[k] > lo:
            lengths[k] -= 1
            diff += 1
    return lengths


def binary_knapsack(seed: int = SEED_BASE + 1, m: int = 2000, n: int = 5000,
                    len_lo: int = 5, len_hi: int = 15, n_fixed: int = 50) -> Milp:
    """Small all-binary instance (plain BP to fixpoint, 2k x 5k, ~20k nonzeros).

    Row lengths uniform in [len_lo, len_hi], columns uniform without replacement,
    coefficients integers uniform in [1, 10], g = floor(0.5 * row sum); n_fixed random
    variables are then fixed to a random 0/1 value (l = u)."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(len_lo, len_hi + 1, size=m)
    row_ptr, col, row_of = _csr_from_lengths(rng, lengths, n)
    val = rng.integers(1, 11, size=len(col)).astype(np.float64)
    rowsum = np.bincount(row_of, weights=val, minlength=m)
    g = np.floor(0.5 * rowsum)
    lb = np.zeros(n)
    ub = np.ones(n)
    fixed = rng.choice(n, size=n_fixed, replace=False)
    v = rng.integers(0, 2, size=n_fixed).astype(np.float64)
    lb[fixed] = v
    ub[fixed] = v
    is_int = np.ones(n, dtype=np.uint8)
    c = rng.standard_normal(n)
    return Milp(m, n, row_ptr, col, val, g, lb, ub, is_int, c, name=f"binary_knapsack_{m}x{n}")


def _zipf_lengths(rng, count, s, cap):
    out = rng.zipf(s, size=count)
    bad = out > cap
    while bad.any():
        out[bad] = rng.zipf(s, size=int(bad.sum()))
        bad = out > cap
    return out.astype(np.float64)


def mixed_powerlaw(seed: int = SEED_BASE + 2, m: int = 200_000, n: int = 500_000,
                   nnz: int = 5_000_000, zipf_s: float = 1.5, max_row: int = 100_000,
                   eq_fraction: float = 0.2, inf_fraction: float = 0.0) -> Milp:
    """Large mixed instance (plain BP, 200k x 500k, 5M nonzeros, power-law rows).

    Variables: 60% binary, 20% integer in [0, 100], 20% continuous in [0, 1000], types
    assigned over a random permutation.  Row lengths: Zipf(s) draws truncated at max_row,
    rescaled so that the total is nnz exactly (one row pinned at max_row, every row >= 1).
    Columns uniform without replacement, coefficients N(0, 10) rounded to 1e-3 (zeros
    redrawn).  A planted point x0 (uniform in the bounds, integral for integer variables)
    makes the problem feasible: a fraction eq_fraction of the rows come as equality pairs
    (a.x <= b, -a.x <= -b, b = a.x0); the others are a.x <= a.x0 + slack with slack uniform
    in [0, 0.05 * sum_j |a_j| (u_j - l_j)].  inf_fraction of the continuous variables get an
    infinite lower bound, upper bound or both."""
    rng = np.random.default_rng(seed)
    n_pairs = int(round(m * eq_fraction / 2))
    n_base = m - n_pairs               # rows before the second row of each pair is added
    raw = _zipf_lengths(rng, n_base, zipf_s, max_row)
    pinned = int(rng.integers(0, n_base))
    is_eq = np.zeros(n_base, dtype=bool)
    cand = np.setdiff1d(np.arange(n_base), [pinned])
    is_eq[rng.choice(cand, size=n_pairs, replace=False)] = True
    weight = np.where(is_eq, 2.0, 1.0)
    rest = nnz - max_row
    raw[pinned] = 0.0
    scale = rest / float((raw * weight).sum())
    lengths = np.maximum(1, np.rint(raw * scale)).astype(np.int64)
    lengths = np.minimum(lengths, max_row)
    lengths[pinned] = max_row
    # fix the total on inequality rows only (an equality row counts twice)
    total = int((lengths * weight.astype(np.int64)).sum())
    ineq = np.flatnonzero(~is_eq & (np.arange(n_base) != pinned))
    sub = _fix_total(rng, lengths[ineq], lengths[ineq].sum() + (nnz - total), lo=1, hi=max_row)
    lengths[ineq] = sub
    assert int((lengths * weight.astype(np.int64)).sum()) == nnz

    # variable types and bounds
    perm = rng.permutation(n)
    n_bin, n_int = int(0.6 * n), int(0.2 * n)
    is_int = np.zeros(n, dtype=np.uint8)
    lb = np.zeros(n)
    ub = np.zeros(n)
    bins, ints, conts = perm[:n_bin], perm[n_bin:n_bin + n_int], perm[n_bin + n_int:]
    is_int[bins] = 1
    ub[bins] = 1.0
    is_int[ints] = 1
    ub[ints] = 100.0
    ub[conts] = 1000.0
    x0 = np.zeros(n)
    x0[bins] = rng.integers(0, 2, size=len(bins))
    x0[ints] = rng.integers(0, 101, size=len(ints))
    x0[conts] = rng.uniform(0.0, 1000.0, size=len(conts))

    base_ptr, base_col, base_row = _csr_from_lengths(rng, lengths, n)
    base_nnz = len(base_col)
    val = np.round(rng.normal(0.0, 10.0, size=base_nnz), 3)
    zero = val == 0.0
    while zero.any():
        val[zero] = np.round(rng.normal(0.0, 10.0, size=int(zero.sum())), 3)
        zero = val == 0.0
    ax0 = np.bincount(base_row, weights=val * x0[base_col], minlength=n_base)
    rng_w = np.bincount(base_row, weights=np.abs(val) * (ub[base_col] - lb[base_col]), minlength=n_base)
    slack = rng.uniform(0.0, 1.0, size=n_base) * 0.05 * rng_w
    g_base = np.where(is_eq, ax0, ax0 + slack)

    # expand equality rows into two <= rows, then shuffle the row order
    rows_src = np.concatenate([np.arange(n_base), np.flatnonzero(is_eq)])
    sign = np.concatenate([np.ones(n_base), -np.ones(n_pairs)])
    order = rng.permutation(len(rows_src))
    rows_src, sign = rows_src[order], sign[order]
    out_len = lengths[rows_src]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(out_len, out=row_ptr[1:])
    # gather the nonzeros of each source row
    starts = base_ptr[rows_src]
    idx = np.repeat(starts - row_ptr[:-1], out_len) + np.arange(nnz, dtype=np.int64)
    col = base_col[idx]
    out_val = val[idx] * np.repeat(sign, out_len)
    g = g_base[rows_src] * sign

    if inf_fraction > 0:
        k = int(round(inf_fraction * len(conts)))
        pick = rng.choice(conts, size=k, replace=False)
        kind = rng.integers(0, 3, size=k)
        lb[pick[kind != 1]] = -np.inf
        ub[pick[kind != 0]] = np.inf
    c = rng.standard_normal(n)
    return Milp(m, n, row_ptr, col.astype(np.int32), out_val, g, lb, ub, is_int, c, x0=x0,
                name=f"mixed_powerlaw_{m}x{n}_{nnz}")


def knapsack_cover(seed: int = SEED_BASE + 3, m: int = 50_000, n: int = 100_000,
                   nnz: int = 1_000_000, len_lo: int = 5, len_hi: int = 40) -> Milp:
    """All-binary probing instance (50k x 100k, 1M nonzeros).

    Row lengths uniform in [len_lo, len_hi], rescaled to total nnz.  Half the rows are
    knapsacks a.x <= floor(0.5 sum a) with a uniform in [1, 20]; the other half are weighted
    covers a.x >= ceil(0.3 sum a), stored as -a.x <= -ceil(0.3 sum a)."""
    rng = np.random.default_rng(seed)
    raw = rng.integers(len_lo, len_hi + 1, size=m).astype(np.float64)
    lengths = np.maximum(1, np.rint(raw * (nnz / raw.sum()))).astype(np.int64)
    lengths = _fix_total(rng, lengths, nnz, lo=1)
    row_ptr, col, row_of = _csr_from_lengths(rng, lengths, n)
    a = rng.integers(1, 21, size=len(col)).astype(np.float64)
    rowsum = np.bincount(row_of, weights=a, minlength=m)
    cover = np.zeros(m, dtype=bool)
    cover[rng.choice(m, size=m // 2, replace=False)] = True
    g = np.where(cover, -np.ceil(0.3 * rowsum), np.floor(0.5 * rowsum))
    val = np.where(cover[row_of], -a, a)
    lb = np.zeros(n)
    ub = np.ones(n)
    is_int = np.ones(n, dtype=np.uint8)
    c = rng.standard_normal(n)
    return Milp(m, n, row_ptr, col, val, g, lb, ub, is_int, c, name=f"knapsack_cover_{m}x{n}")


def random_milp(seed: int, m: int, n: int, len_lo: int = 1, len_hi: int = 8,
                int_fraction: float = 0.5, bin_fraction: float = 0.5,
                neg_fraction: float = 0.5, inf_fraction: float = 0.0,
                eq_fraction: float = 0.0, empty_rows: int = 0, integer_coefs: bool = False,
                coef_scale: float = 10.0, slack_scale: float = 0.05) -> Milp:
    """Small general instance for parity sweeps: mixed variable types, coefficients of
    either sign, optional infinite bounds, equality pairs and empty rows, planted-point
    right-hand sides (so the problem is feasible unless it is tightened further)."""
    rng = np.random.default_rng(seed)
    len_hi = max(len_lo, min(len_hi, n))
    lengths = rng.integers(len_lo, len_hi + 1, size=m)
    if empty_rows:
        lengths[rng.choice(m, size=min(empty_rows, m), replace=False)] = 0
    row_ptr, col, row_of = _csr_from_lengths(rng, lengths, n)
    nnz = len(col)
    if integer_coefs:
        mag = rng.integers(1, 11, size=nnz).astype(np.float64)
    else:
        mag = np.round(rng.uniform(0.1, coef_scale, size=nnz), 3)
        mag[mag == 0.0] = 0.5
    sgn = np.where(rng.uniform(size=nnz) < neg_fraction, -1.0, 1.0)
    val = mag * sgn
    is_int = (rng.uniform(size=n) < int_fraction).astype(np.uint8)
    is_bin = (rng.uniform(size=n) < bin_fraction) & (is_int == 1)
    lb = np.zeros(n)
    ub = np.where(is_bin, 1.0, np.where(is_int == 1, 20.0, 100.0))
    x0 = np.where(is_int == 1, rng.integers(0, 21, size=n).astype(np.float64), rng.uniform(0, 100, size=n))
    x0 = np.minimum(x0, ub)
    ax0 = np.bincount(row_of, weights=val * x0[col], minlength=m)
    rng_w = np.bincount(row_of, weights=np.abs(val) * (ub[col] - lb[col]), minlength=m)
    g = ax0 + rng.uniform(0.0, 1.0, size=m) * slack_scale * rng_w
    if eq_fraction > 0 and m >= 2:
        # turn row pairs (2i, 2i+1) into a.x <= b, -a.x <= -b with the row 2i's pattern
        k = int(m * eq_fraction / 2)
        for i in rng.choice(m // 2, size=k, replace=False):
            r0, r1 = 2 * i, 2 * i + 1
            l0 = row_ptr[r0 + 1] - row_ptr[r0]
            l1 = row_ptr[r1 + 1] - row_ptr[r1]
            if l0 != l1:
                continue
            col[row_ptr[r1]:row_ptr[r1 + 1]] = col[row_ptr[r0]:row_ptr[r0 + 1]]
            val[row_ptr[r1]:row_ptr[r1 + 1]] = -val[row_ptr[r0]:row_ptr[r0 + 1]]
            b = float(np.dot(val[row_ptr[r0]:row_ptr[r0 + 1]], x0[col[row_ptr[r0]:row_ptr[r0 + 1]]]))
            g[r0], g[r1] = b, -b
    if inf_fraction > 0:
        cont = np.flatnonzero(is_int == 0)
        k = int(round(inf_fraction * len(cont)))
        if k:
            pick = rng.choice(cont, size=k, replace=False)
            kind = rng.integers(0, 3, size=k)
            lb[pick[kind != 1]] = -np.inf
            ub[pick[kind != 0]] = np.inf
    c = rng.standard_normal(n)
    return Milp(m, n, row_ptr, col.astype(np.int32), val, g, lb, ub, is_int, c, x0=x0,
                name=f"random_{m}x{n}_s{seed}")


def tighten_random(seed: int, p: Milp, k: int, planted: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Start bounds for a propagation test: the problem's bounds with k random integer
    variables fixed to a random value of their domain, or to the planted point's value
    (planted=True, when the problem has one, which keeps it feasible)."""
    rng = np.random.default_rng(seed)
    lb, ub = p.lb.copy(), p.ub.copy()
    ints = np.flatnonzero(p.is_int == 1)
    if len(ints) == 0 or k == 0:
        return lb, ub
    pick = rng.choice(ints, size=min(k, len(ints)), replace=False)
    for j in pick:
        if planted and p.x0 is not None:
            v = float(np.clip(np.rint(p.x0[j]), lb[j], ub[j]))
        else:
            lo = lb[j] if np.isfinite(lb[j]) else -5.0
            hi = ub[j] if np.isfinite(ub[j]) else lo + 10.0
            v = float(rng.integers(int(math.ceil(lo)), int(math.floor(hi)) + 1))
        lb[j] = ub[j] = v
    return lb, ub


def block_diagonal(parts: list[Milp]) -> tuple[Milp, np.ndarray, np.ndarray]:
    """Concatenates instances into one block-diagonal problem; returns it with the row and
    column offsets of each part (length len(parts)+1)."""
    ro = np.zeros(len(parts) + 1, dtype=np.int64)
    co = np.zeros(len(parts) + 1, dtype=np.int64)
    for i, q in enumerate(parts):
        ro[i + 1] = ro[i] + q.m
        co[i + 1] = co[i] + q.n
    ptrs, cols, vals = [np.zeros(1, dtype=np.int64)], [], []
    base = 0
    for i, q in enumerate(parts):
        ptrs.append(q.row_ptr[1:] + base)
        base += q.nnz
        cols.append(q.col.astype(np.int64) + co[i])
        vals.append(q.val)
    M, N = int(ro[-1]), int(co[-1])
    big = Milp(M, N, np.concatenate(ptrs), np.concatenate(cols).astype(np.int32), np.concatenate(vals),
               np.concatenate([q.g for q in parts]), np.concatenate([q.lb for q in parts]),
               np.concatenate([q.ub for q in parts]), np.concatenate([q.is_int for q in parts]),
               np.concatenate([q.c for q in parts]), name=f"block_{len(parts)}")
    return big, ro, co


def uneven_batch(seed: int = SEED_BASE + 4, count: int = 64, nnz_lo: float = 1e3,
                 nnz_hi: float = 5e5) -> list[Milp]:
    """Instances of uneven size for batched propagation: nnz log-uniform in
    [nnz_lo, nnz_hi], m/n uniform in [0.2, 2], mean row length uniform in [5, 40]; half of
    the variables integer (half of those binary, half in [0, 100]), the rest continuous in
    [0, 1000]; integer coefficients +-[1, 10]; planted-point right-hand sides."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        sub = np.random.default_rng((seed << 16) + i)
        nnz = int(round(math.exp(sub.uniform(math.log(nnz_lo), math.log(nnz_hi)))))
        ratio = sub.uniform(0.2, 2.0)
        mean_len = sub.uniform(5.0, 40.0)
        m = max(1, int(round(nnz / mean_len)))
        n = max(int(math.ceil(2 * mean_len)) + 1, int(round(m / ratio)))
        raw = sub.integers(max(1, int(mean_len / 2)), int(1.5 * mean_len) + 1, size=m)
        lengths = np.maximum(1, np.rint(raw * (nnz / raw.sum()))).astype(np.int64)
        lengths = np.minimum(lengths, n)
        lengths = _fix_total(sub, lengths, nnz, lo=1, hi=n)
        row_ptr, col, row_of = _csr_from_lengths(sub, lengths, n)
        val = sub.integers(1, 11, size=len(col)).astype(np.float64) * np.where(sub.uniform(size=len(col)) < 0.5, -1.0, 1.0)
        perm = sub.permutation(n)
        n_int = n // 2
        is_int = np.zeros(n, dtype=np.uint8)
        is_int[perm[:n_int]] = 1
        lb = np.zeros(n)
        ub = np.full(n, 1000.0)
        ub[perm[:n_int // 2]] = 1.0
        ub[perm[n_int // 2:n_int]] = 100.0
        x0 = np.where(is_int == 1, np.floor(sub.uniform(size=n) * (ub + 1)), sub.uniform(size=n) * ub)
        x0 = np.minimum(x0, ub)
        ax0 = np.bincount(row_of, weights=val * x0[col], minlength=m)
        rng_w = np.bincount(row_of, weights=np.abs(val) * (ub[col] - lb[col]), minlength=m)
        g = ax0 + sub.uniform(size=m) * 0.05 * rng_w
        c = sub.standard_normal(n)
        out.append(Milp(m, n, row_ptr, col, val, g, lb, ub, is_int, c, x0=x0, name=f"uneven_{i}"))
    del rng
    return out


def rounding_instance(index: int, nnz: int = 1_000_000, sigma: float = 0.3,
                      eq_fraction: float = 0.2) -> tuple[Milp, np.ndarray]:
    """Instance `index` of the learned-rounding workload and the fractional point it rounds.

    The problem is the mixed power-law instance scaled to `nnz` nonzeros (m = nnz / 25,
    n = nnz / 10, the longest row nnz / 50; 1M nonzeros: 40k x 100k), seed
    (SEED_BASE + 5) * 2^16 + index, objective N(0, 1), with a fraction eq_fraction of the rows
    as equality pairs (0.2 as in the large mixed instance; the 1M-nonzero experiment takes 0.01,
    with which the plain method reaches feasibility in part of the runs).  The fractional point
    stands in for an LP relaxation solution: the planted feasible point plus N(0, sigma) noise,
    clamped to the bounds.  It is close to a feasible point by construction (the planted one),
    which a real LP solution need not be."""
    seed = ((SEED_BASE + 5) << 16) + int(index)
    p = mixed_powerlaw(seed=seed, m=nnz // 25, n=nnz // 10, nnz=nnz, max_row=max(100, nnz // 50),
                       eq_fraction=eq_fraction)
    rng = np.random.default_rng(seed + 1)
    x = np.clip(p.x0 + rng.normal(0.0, sigma, p.n), p.lb, p.ub)
    p.name = f"rounding_{index}_{p.m}x{p.n}_{nnz}"
    return p, x
