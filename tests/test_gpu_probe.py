"""GPU batched double probing (bp_probe_batch through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2510_20499_gb300 import synth
from tests.helpers import golden_problem, load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def _pairs(p, rl, ru, count, seed):
    rng = np.random.default_rng(seed)
    cand = [j for j in range(p.n) if oracle.probe_split(p.is_int[j], rl[j], ru[j])]
    pick = rng.choice(cand, size=min(count, len(cand)), replace=False) if cand else []
    var = np.array(pick, dtype=np.int32)
    boxes = np.array([oracle.probe_split(p.is_int[j], rl[j], ru[j]) for j in var], dtype=np.float64).reshape(-1, 4)
    return var, boxes


def _gpu_probe(pkg, p, rl, ru, var, boxes, **kw):
    import torch
    prob = pkg.Problem(p)
    c = prob.probe_batch(torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda"),
                         torch.tensor(var, device="cuda"), torch.tensor(boxes, device="cuda"), **kw)
    return {k: v.cpu().numpy() for k, v in c.items()}


def _compare(p, g, o):
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["rounds"], o["rounds"])
    np.testing.assert_array_equal(g["nnz_updates"], o["nnz_updates"])
    np.testing.assert_array_equal(g["offsets"], o["offsets"])
    np.testing.assert_array_equal(g["var"], o["var"])
    ints = p.is_int[o["var"]] == 1
    np.testing.assert_array_equal(g["l"][ints], o["l"][ints])
    np.testing.assert_array_equal(g["u"][ints], o["u"][ints])
    for a, b in ((g["l"], o["l"]), (g["u"], o["u"])):
        fin = np.isfinite(b) & ~ints
        assert (np.abs(a[fin] - b[fin]) <= 1e-9 * np.maximum(1, np.abs(b[fin]))).all()
        np.testing.assert_array_equal(a[~np.isfinite(b)], b[~np.isfinite(b)])


def test_golden_probe(pkg):
    d = load_golden("probe_knapsack.json")
    p = golden_problem(d)
    rl, ru = np.array(d["root_lb"], float), np.array(d["root_ub"], float)
    g = _gpu_probe(pkg, p, rl, ru, np.array(d["var"], np.int32), np.array(d["boxes"], float))
    for e, want in enumerate(d["expect"]):
        assert g["status"][e] == want["status"]
        a, b = g["offsets"][e], g["offsets"][e + 1]
        got = [[int(g["var"][q]), float(g["l"][q]), float(g["u"][q])] for q in range(a, b)]
        assert got == [[int(x[0]), float(x[1]), float(x[2])] for x in want["entries"]], want["note"]


@pytest.mark.parametrize("seed", range(4))
def test_knapsack_cover_probes(pkg, seed):
    p = synth.knapsack_cover(seed=40 + seed, m=2000, n=4000, nnz=40_000)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    assert r["status"] == oracle.FIXPOINT
    var, boxes = _pairs(p, rl, ru, 300, seed)
    o = P.probe_batch(rl, ru, var, boxes)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)


@pytest.mark.parametrize("seed", range(4))
def test_mixed_probes(pkg, seed):
    """General integers, continuous variables, infinite bounds, long rows, equality pairs."""
    p = synth.random_milp(500 + seed, m=600, n=800, len_lo=1, len_hi=300, inf_fraction=0.1,
                          eq_fraction=0.2, int_fraction=0.7)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    if r["status"] == oracle.INFEASIBLE:
        pytest.skip("root infeasible")
    var, boxes = _pairs(p, rl, ru, 200, seed)
    o = P.probe_batch(rl, ru, var, boxes)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)


@pytest.mark.parametrize("seed", range(3))
def test_powerlaw_probes(pkg, seed):
    """Short rows on average (12.5 nonzeros: 8 lanes per row in the probe kernel) with a power-law
    tail up to 500 nonzeros, so that long rows take many segments of a narrow lane group."""
    p = synth.mixed_powerlaw(seed=700 + seed, m=2000, n=5000, nnz=25_000, max_row=500, inf_fraction=0.1)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    if r["status"] == oracle.INFEASIBLE:
        pytest.skip("root infeasible")
    var, boxes = _pairs(p, rl, ru, 300, seed)
    o = P.probe_batch(rl, ru, var, boxes)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)


@pytest.mark.parametrize("lens", [(3, 9), (20, 60)])
def test_probe_lane_groups(pkg, lens):
    """Average row lengths that select 8 and 16 lanes per row (6 and 40 nonzeros)."""
    lo, hi = lens
    m, n = 2000, 4000
    p = synth.knapsack_cover(seed=60 + lo, m=m, n=n, nnz=m * (lo + hi) // 2, len_lo=lo, len_hi=hi)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    assert r["status"] == oracle.FIXPOINT
    var, boxes = _pairs(p, rl, ru, 300, lo)
    o = P.probe_batch(rl, ru, var, boxes)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)


def test_probe_round_limit_and_capacity(pkg):
    p = synth.knapsack_cover(seed=9, m=1000, n=2000, nnz=20_000)
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    var, boxes = _pairs(p, rl, ru, 100, 1)
    o = P.probe_batch(rl, ru, var, boxes, max_rounds=1)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes, max_rounds=1, cap=1)   # forces the capacity path
    _compare(p, g, o)


@pytest.fixture(scope="module")
def full_size():
    """The 50k x 100k, 1M-nonzero probing instance, its root fixpoint, the 2,048 pairs chosen by
    the priority order and the oracle's cache of them."""
    p = synth.knapsack_cover()
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    k1, k2, k3 = P.probe_priority(rl, ru)
    var = oracle.priority_order(k1, k2, k3)[:2048].astype(np.int32)
    boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=np.float64).reshape(-1, 4)
    return p, P, rl, ru, var, boxes, P.probe_batch(rl, ru, var, boxes)


def test_probes_full_size(pkg, full_size):
    p, P, rl, ru, var, boxes, o = full_size
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)


def test_probe_batch_graph_capture_full_size(pkg, full_size):
    """bp_probe_batch_async captured in a CUDA graph with the whole batch (bound keys, row caps,
    the persistent probe launch, offsets, the cache copy, the entry-count and index words) and
    replayed three times: every replay's cache equals the oracle's."""
    import torch
    p, P, rl, ru, var, boxes, o = full_size
    prob = pkg.Problem(p)
    d = {k: torch.tensor(a, device="cuda") for k, a in (("rl", rl), ("ru", ru), ("var", var), ("boxes", boxes))}
    ref = prob.probe_batch(d["rl"], d["ru"], d["var"], d["boxes"])     # sizes the scratch
    cap = int(ref["var"].numel()) + 256
    cache = pkg._probe_cache(torch, prob.device, len(var), cap)
    words = torch.zeros(2, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        prob.probe_batch_async(d["rl"], d["ru"], d["var"], d["boxes"], cache, words, stream=s)   # warm-up at size
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        prob.probe_batch_async(d["rl"], d["ru"], d["var"], d["boxes"], cache, words)
    for rep in range(3):
        for t in cache.values():
            t.zero_()
        words.zero_()
        g.replay()
        torch.cuda.synchronize()
        needed, bad = (int(x) for x in words.cpu())
        assert bad == 0 and needed == len(o["var"]), (needed, bad)
        got = {k: v.cpu().numpy() for k, v in cache.items()}
        got["var"], got["l"], got["u"] = got["var"][:needed], got["l"][:needed], got["u"][:needed]
        _compare(p, got, o)


def test_probe_cache_apply_full_size(pkg, full_size):
    """Bounds derived from the GPU's cache of the full-size batch equal those the oracle derives
    from its own cache (Section 2.2)."""
    import torch
    p, P, rl, ru, var, boxes, o = full_size
    prob = pkg.Problem(p)
    c = prob.probe_batch(torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda"),
                         torch.tensor(var, device="cuda"), torch.tensor(boxes, device="cuda"))
    gl, gu = torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda")
    gr = prob.probe_cache_apply(gl, gu, c)
    ol, ou, orr = P.probe_cache_apply(rl, ru, o)
    assert gr == orr, (gr, orr)
    np.testing.assert_array_equal(gl.cpu().numpy(), ol)
    np.testing.assert_array_equal(gu.cpu().numpy(), ou)
    print(f"\nprobing cache of {len(var)} pairs: {orr['fixed_pairs']} variables fixed by an infeasible branch, "
          f"{orr['tightened']} variables tightened, status {orr['status']}")


@pytest.mark.parametrize("case", range(4))
def test_probe_cache_apply_golden(pkg, case):
    """The hand-worked cases of the oracle's pin (Section 2.2), probed and applied on the GPU."""
    import torch
    from tests.helpers import milp_from_dense
    c = load_golden("probe_apply.json")["cases"][case]
    p = milp_from_dense(np.array(c["A"], float), c["g"], np.array(c["lb"], float), np.array(c["ub"], float),
                        np.array(c["is_int"]))
    prob = pkg.Problem(p)
    gl, gu = torch.tensor(p.lb, device="cuda"), torch.tensor(p.ub, device="cuda")
    prob.propagate(gl, gu)
    rl, ru = gl.cpu().numpy(), gu.cpu().numpy()
    var = np.array(c["probe"], dtype=np.int32)
    boxes = np.array([oracle.probe_split(p.is_int[j], rl[j], ru[j]) for j in var], dtype=float).reshape(-1, 4)
    cache = prob.probe_batch(gl, gu, torch.tensor(var, device="cuda"), torch.tensor(boxes, device="cuda"))
    r = prob.probe_cache_apply(gl, gu, cache)
    for k in ("status", "first_infeasible_pair", "first_infeasible_var", "fixed_pairs"):
        assert r[k] == c[k], (k, r, c["note"])
    if "out_lb" in c:
        np.testing.assert_array_equal(gl.cpu().numpy(), c["out_lb"])
        np.testing.assert_array_equal(gu.cpu().numpy(), c["out_ub"])
        assert r["tightened"] == c["tightened"]


@pytest.mark.parametrize("seed", range(4))
def test_probe_cache_apply_random(pkg, seed):
    """Random mixed problems with integer variables probed: the GPU's derived bounds and result
    equal the oracle's (caches compared first)."""
    import torch
    p = synth.random_milp(700 + seed, 400, 600, len_lo=2, len_hi=20, integer_coefs=True, int_fraction=0.8,
                          slack_scale=0.05, eq_fraction=0.1)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    if r["status"] == oracle.INFEASIBLE:
        pytest.skip("root infeasible")
    var, boxes = _pairs(p, rl, ru, 200, seed)
    o = P.probe_batch(rl, ru, var, boxes)
    prob = pkg.Problem(p)
    c = prob.probe_batch(torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda"),
                         torch.tensor(var, device="cuda"), torch.tensor(boxes, device="cuda"))
    _compare(p, {k: v.cpu().numpy() for k, v in c.items()}, o)
    gl, gu = torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda")
    gr = prob.probe_cache_apply(gl, gu, c)
    ol, ou, orr = P.probe_cache_apply(rl, ru, o)
    assert gr == orr
    ints = p.is_int == 1
    np.testing.assert_array_equal(gl.cpu().numpy()[ints], ol[ints])
    np.testing.assert_array_equal(gu.cpu().numpy()[ints], ou[ints])
    np.testing.assert_allclose(gl.cpu().numpy(), ol, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gu.cpu().numpy(), ou, rtol=1e-9, atol=1e-9)


def _gpu_priority(pkg, p, lb, ub):
    import torch
    prob = pkg.Problem(p)
    k1, k2, k3, order = prob.probe_priority(torch.tensor(lb, device="cuda"), torch.tensor(ub, device="cuda"))
    return k1.cpu().numpy(), k2.cpu().numpy(), k3.cpu().numpy(), order.cpu().numpy()


def test_priority_golden(pkg):
    d = load_golden("priority_small.json")
    p = golden_problem(d)
    k1, k2, k3, order = _gpu_priority(pkg, p, np.array(d["lb"], float), np.array(d["ub"], float))
    np.testing.assert_array_equal(k1, d["key1"])
    np.testing.assert_array_equal(k2, d["key2"])
    np.testing.assert_array_equal(k3, d["key3"])
    np.testing.assert_array_equal(order, d["order"])


@pytest.mark.parametrize("seed", range(3))
def test_priority_exact_data(pkg, seed):
    """Integer coefficients and bounds: keys and order identical to the oracle's."""
    p = synth.knapsack_cover(seed=60 + seed, m=5000, n=10_000, nnz=100_000)
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    o1, o2, o3 = P.probe_priority(rl, ru)
    g1, g2, g3, gord = _gpu_priority(pkg, p, rl, ru)
    np.testing.assert_array_equal(g1, o1)
    np.testing.assert_array_equal(g2, o2)
    np.testing.assert_array_equal(g3, o3)
    np.testing.assert_array_equal(gord, oracle.priority_order(o1, o2, o3))


def test_priority_general_data(pkg):
    """Non-integer data (activities summed in another order): key1 identical, key2 and key3
    within 1e-9 relative, and the GPU order sorted by the GPU keys."""
    p = synth.random_milp(77, m=3000, n=4000, len_lo=1, len_hi=60, inf_fraction=0.05, int_fraction=0.8)
    P = oracle.Problem(p)
    rl, ru, r, _ = P.bp(p.lb, p.ub)
    o1, o2, o3 = P.probe_priority(rl, ru)
    g1, g2, g3, gord = _gpu_priority(pkg, p, rl, ru)
    np.testing.assert_array_equal(g1, o1)
    for g, o in ((g2, o2), (g3, o3)):
        fin = np.isfinite(o)
        np.testing.assert_array_equal(np.isfinite(g), fin)
        assert (np.abs(g[fin] - o[fin]) <= 1e-9 * np.maximum(1, np.abs(o[fin]))).all()
    assert sorted(gord.tolist()) == np.flatnonzero(o1 >= 0).tolist()
    keys = [(-g1[j], -g2[j], g3[j], j) for j in gord]
    assert keys == sorted(keys)


def test_probe_index_out_of_range(pkg):
    """A variable index outside [0, n) is reported (BP_ERR_INVALID), never dereferenced, and the
    handle stays usable: the same call with valid indices then matches the oracle."""
    import torch
    p = synth.knapsack_cover(seed=11, m=300, n=600, nnz=4000)
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    var, boxes = _pairs(p, rl, ru, 40, 3)
    prob = pkg.Problem(p)
    dl, du = torch.tensor(rl, device="cuda"), torch.tensor(ru, device="cuda")
    for bad in (p.n, -1):
        v = var.copy()
        v[7] = bad
        with pytest.raises(pkg.GpuBpError) as e:
            prob.probe_batch(dl, du, torch.tensor(v, device="cuda"), torch.tensor(boxes, device="cuda"))
        assert e.value.code == pkg.BP_ERR_INVALID
    c = prob.probe_batch(dl, du, torch.tensor(var, device="cuda"), torch.tensor(boxes, device="cuda"))
    _compare(p, {k: x.cpu().numpy() for k, x in c.items()}, P.probe_batch(rl, ru, var, boxes))


def _stars(sizes):
    """Binary stars: hub h with spokes s, one row x_h - x_s <= 0 per spoke (the hub at 1 forces
    every spoke to 1 in one round)."""
    n = len(sizes) + sum(sizes)
    rows, hubs, j = [], [], len(sizes)
    for h, size in enumerate(sizes):
        hubs.append(h)
        for s in range(j, j + size):
            rows.append((h, s))
        j += size
    m = len(rows)
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = np.tile(np.array([1.0, -1.0]), m)
    return synth.Milp(m, n, np.arange(0, 2 * m + 1, 2, dtype=np.int64), col, val, np.zeros(m), np.zeros(n),
                      np.ones(n), np.ones(n, dtype=np.uint8), np.zeros(n)), hubs


def test_probes_beyond_the_sparse_table(pkg):
    """Pairs whose branches touch more variables than a block's sparse table holds (4,096 slots:
    a hub fixing 12,000 or 4,500 spokes) go to the dense pass; the others stay in the sparse
    pass.  Both together must equal the oracle: statuses, rounds, work and every implied bound."""
    p, hubs = _stars([12_000, 4_500, 3_000, 1_000, 50, 5])
    P = oracle.Problem(p)
    rl, ru = p.lb.copy(), p.ub.copy()
    spokes = np.random.default_rng(4).choice(np.arange(len(hubs), p.n), 300, replace=False)
    var = np.concatenate([np.array(hubs), spokes]).astype(np.int32)
    boxes = np.array([oracle.probe_split(1, 0.0, 1.0) for _ in var], dtype=np.float64).reshape(-1, 4)
    o = P.probe_batch(rl, ru, var, boxes)
    g = _gpu_probe(pkg, p, rl, ru, var, boxes)
    _compare(p, g, o)
    counts = np.diff(o["offsets"])
    assert counts[1] == 12_001 and counts[3] == 4_501   # the up branches: the hub and every spoke
