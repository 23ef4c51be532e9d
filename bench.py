"""Benchmark: bound propagation throughput (nnz-updates/s) on the large mixed MILP.

Workload: the 200k-row, 500k-variable, 5M-nonzero power-law instance (60% binary, 20% general
integer, 20% continuous; Zipf(1.5) row lengths up to 100k; equality pairs), synthetic and
seeded.  A step is one bp_propagate from the instance's default bounds to the fixpoint through
the C ABI (all rounds, worklist of changed rows), including the copy of the start bounds into
the propagated arrays.  The unit of work is the nnz-update: the nonzeros of every row the
propagation processes, summed over rounds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain sequential C) on the same workload.
Multi-GPU runs (torchrun) propagate one independent replica per GPU (no data exchange); the
value is the sum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BP nnz-updates/s & probes/s (FP64, % HBM peak); batched vs plain on same GPU"
UNIT = "nnz-updates/s"
WORKLOAD = "mixed power-law MILP 200k rows x 500k vars, 5M nnz (Zipf 1.5 rows <= 100k, 60/20/20 bin/int/cont, 20% equality rows)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the probing, batch, learned and scorer measurements")
    ap.add_argument("--extras", default="probing,batch,fp,learned,scorer,pdhg,local_mip,efp",
                    help="comma-separated subset of the extra measurements to run (learned_full, the "
                         "160/40-instance learned-order experiment at 1M nonzeros, is not in the default set)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tensor_peak():
    """Dense BF16 TFLOP/s for a kernel timed alone (the measured burst figure, else the fallback)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"])
    return 1900.0


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def finish(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import statistics
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# DRAM bytes (read + write) of one bp_kernel launch on this workload, from the ncu capture
# summarised in profiles/bp_kernel_mixed_powerlaw_5M.md; reported only while the kernel's
# sources are the ones that capture was taken on.
NCU_TRAFFIC = {"sources_sha256_16": "4ea1c434c63a4110", "bytes": 219_092_224}
KERNEL_SOURCES = ["bp_engine.cu", "bp_device.cuh", "bp_host.h"]


def kernel_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2510_20499_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return NCU_TRAFFIC["bytes"] if h.hexdigest()[:16] == NCU_TRAFFIC["sources_sha256_16"] else None


def algorithmic_bytes(trace_rows, trace_nnz, trace_chg, n):
    """Bytes the propagation must move: per nonzero processed its column index (4 B) and
    coefficient (8 B); per worklist row its extent (8 B); per changed variable its new bounds
    written and read back (32 B); per launch the start bounds in (16 B / var), both bound
    buffers initialised (32 B / var) and the final bounds read and written out (32 B / var)."""
    return int(12 * sum(trace_nnz) + 8 * sum(trace_rows) + 32 * sum(trace_chg) + 80 * n)


def whole_job(units, ms, device):
    """Whole-job totals over the ranks of the process group (one replica per rank, no exchange
    on the data path): the units all ranks processed and the slowest rank's time.  Without a
    process group: the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units, ms
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([int(units)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return int(u.item()), float(t.item())


def run_reference(args):
    import oracle
    from paper_2510_20499_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = synth.mixed_powerlaw()
    P = oracle.Problem(p)
    for _ in range(args.warmup):
        P.bp(p.lb, p.ub)
    nnz = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, r, _ = P.bp(p.lb, p.ub)
        nnz += r["nnz_updates"]
    dt = time.perf_counter() - t0
    v = nnz / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "single CPU thread"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full propagations of the workload"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _milp_arrays(p):
    return dict(m=p.m, n=p.n, row_ptr=p.row_ptr, col=p.col, val=p.val, g=p.g, lb=p.lb, ub=p.ub, is_int=p.is_int)


def _oracle_problem(d):
    import oracle
    from paper_2510_20499_gb300 import synth
    p = synth.Milp(d["m"], d["n"], d["row_ptr"], d["col"], d["val"], d["g"], d["lb"], d["ub"], d["is_int"],
                   np.zeros(d["n"]))
    return p, oracle.Problem(p)


def _probe_worker(args):
    """One worker of the all-core probing baseline: the oracle's probe batch on its share of the
    pairs; returns its own compute time."""
    d, rl, ru, var, boxes = args
    _, P = _oracle_problem(d)
    t0 = time.perf_counter()
    P.probe_batch(rl, ru, var, boxes)
    return time.perf_counter() - t0


def _bp_worker(args):
    """One worker of the all-core batch baseline: the oracle's propagation of its instances."""
    nnz = 0
    t = 0.0
    for d in args:
        p, P = _oracle_problem(d)
        t0 = time.perf_counter()
        _, _, r, _ = P.bp(p.lb, p.ub)
        t += time.perf_counter() - t0
        nnz += r["nnz_updates"]
    return t, nnz


def all_core_baselines():
    """The oracle over all host cores for the two workloads of independent units: the 4,096
    probes of the probing workload (pairs split evenly over the workers) and the 64 instances of
    the batch (balanced by size).  Workers are spawned processes, each timing only its own
    compute; the throughput divides all units by the slowest worker's time."""
    import concurrent.futures
    import multiprocessing as mp
    import oracle
    from paper_2510_20499_gb300 import synth
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    out = {"cores": cores, "kind": "oracle",
           "cpu": platform_cpu()}
    p = synth.knapsack_cover()
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    k1, k2, k3 = P.probe_priority(rl, ru)
    var = oracle.priority_order(k1, k2, k3)[:2048].astype(np.int32)
    boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=np.float64).reshape(-1, 4)
    d = _milp_arrays(p)
    chunks = [(d, rl, ru, var[i::cores].copy(), boxes[i::cores].copy()) for i in range(cores)]
    with concurrent.futures.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
        times = list(ex.map(_probe_worker, chunks))
    out["probing"] = {"probes_per_s": 2 * len(var) / max(times),
                      "sample": f"all {len(var)} priority pairs = {2 * len(var)} propagations over {cores} workers"}
    parts = synth.uneven_batch()
    order = np.argsort([-q.nnz for q in parts])
    shares = [[] for _ in range(cores)]
    for i, k in enumerate(order):                   # snake order: balances the uneven sizes
        r = i % (2 * cores)
        shares[r if r < cores else 2 * cores - 1 - r].append(_milp_arrays(parts[k]))
    with concurrent.futures.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
        res = list(ex.map(_bp_worker, [sh for sh in shares if sh]))
    out["batch"] = {"nnz_updates_per_s": sum(r[1] for r in res) / max(r[0] for r in res),
                    "sample": f"all {len(parts)} instances over {cores} workers"}
    return out


def platform_cpu():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                for key in ("model name", "CPU part", "Hardware"):
                    if line.startswith(key):
                        return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(p, budget_s=12.0):
    import oracle
    P = oracle.Problem(p)
    nnz, runs = 0, 0
    t0 = time.perf_counter()
    while runs == 0 or time.perf_counter() - t0 < budget_s:
        _, _, r, _ = P.bp(p.lb, p.ub)
        nnz += r["nnz_updates"]
        runs += 1
    dt = time.perf_counter() - t0
    out = {"value": nnz / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{runs} full propagations of the workload ({dt:.1f} s, single thread)"}
    out["probing"] = cpu_probing_baseline()
    out["all_cores"] = all_core_baselines()
    return out


def cpu_probing_baseline(pairs=512):
    """The oracle's double probing on the probing workload (knapsack/cover 50k x 100k, 1M nnz),
    on the first `pairs` variables of the priority order (a bounded sample of the 2,048 the GPU
    probes), single thread."""
    import numpy as np
    import oracle
    from paper_2510_20499_gb300 import synth
    p = synth.knapsack_cover()
    P = oracle.Problem(p)
    rl, ru, _, _ = P.bp(p.lb, p.ub)
    k1, k2, k3 = P.probe_priority(rl, ru)
    var = oracle.priority_order(k1, k2, k3)[:pairs].astype(np.int32)
    boxes = np.array([oracle.probe_split(1, rl[j], ru[j]) for j in var], dtype=np.float64).reshape(-1, 4)
    t0 = time.perf_counter()
    P.probe_batch(rl, ru, var, boxes)
    dt = time.perf_counter() - t0
    return {"probes_per_s": 2 * len(var) / dt, "cores": 1, "kind": "oracle",
            "sample": f"{len(var)} priority pairs = {2 * len(var)} propagations ({dt:.1f} s, single thread)"}


def probing_extra(pkg, torch, dev):
    """Probes/s on the 50k x 100k, 1M-nonzero knapsack/cover instance: 2,048 variables (the
    top of the priority order) at 0 and 1, i.e. 4,096 propagations, in one batched launch,
    against one bp_propagate_from launch per branch on the same GPU."""
    import numpy as np
    from paper_2510_20499_gb300 import synth
    p = synth.knapsack_cover()
    prob = pkg.Problem(p)
    rl = torch.tensor(p.lb, device=dev)
    ru = torch.tensor(p.ub, device=dev)
    prob.propagate(rl, ru)
    _, _, _, order = prob.probe_priority(rl, ru)
    var = order[:2048].contiguous()
    P = int(var.numel())
    lo = rl[var.long()]
    hi = ru[var.long()]
    boxes = torch.stack([lo, lo, hi, hi], dim=1).contiguous()      # binaries: [l, l] and [u, u]
    c = prob.probe_batch(rl, ru, var, boxes)                       # warm-up, sizes the cache
    cap = int(c["var"].numel()) + 1024
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = prob.probe_batch(rl, ru, var, boxes, cap=cap)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    t_batch = float(np.median(times))
    nnz = int(c["nnz_updates"].sum().item())
    # one launch per branch
    hv = var.cpu().numpy()
    hb = boxes.cpu().numpy()
    wl, wu = rl.clone(), ru.clone()
    vt = torch.empty(1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(P):
        vt.fill_(int(hv[i]))
        for b in range(2):
            wl.copy_(rl)
            wu.copy_(ru)
            wl[int(hv[i])] = float(hb[i, 2 * b])
            wu[int(hv[i])] = float(hb[i, 2 * b + 1])
            prob.propagate_from(wl, wu, vt, sync=False)
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1)
    # algorithmic bytes: 12 B per nonzero processed (column, coefficient) and 20 B per cache entry
    # written (variable, bounds); the bound gathers of the branches' few variables hit L2
    entries = int(c["var"].numel())
    pbytes = 12 * nnz + 20 * entries
    hbm, _ = peaks()
    return {"workload": "knapsack/cover 50k x 100k, 1M nnz; 2,048 priority pairs = 4,096 propagations",
            "roofline": {"bound": "hbm", "kernel": "probe_kernel (whole call)", "bytes": pbytes,
                         "achieved": pbytes / (t_batch / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": pbytes / (t_batch / 1e3) / 1e9 / hbm},
            "probes_per_s": 2 * P / (t_batch / 1e3), "ms_batched": t_batch,
            "probes_per_s_plain": 2 * P / (t_plain / 1e3), "ms_plain": t_plain,
            "speedup_batched_vs_plain": t_plain / t_batch, "nnz_updates": nnz,
            "cache_entries": int(c["var"].numel())}


def batch_extra(pkg, torch, dev):
    """Aggregate nnz-updates/s of 64 uneven instances (nnz log-uniform in [1e3, 5e5]) in one
    persistent launch captured in a CUDA graph, with the default row-class split points and
    with the ones bp_autotune picks for this batch."""
    import numpy as np
    from paper_2510_20499_gb300 import synth
    parts = synth.uneven_batch()
    big, ro, co = synth.block_diagonal(parts)
    prob = pkg.Problem(big)
    prob.set_instances(ro, co)
    lb0 = torch.tensor(big.lb, device=dev)
    ub0 = torch.tensor(big.ub, device=dev)
    lb, ub = lb0.clone(), ub0.clone()
    res = torch.empty(len(parts) * pkg.C.sizeof(pkg.BpResult) // 4, dtype=torch.int32, device=dev)

    def graph_ms():
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            prob.propagate_batch(lb, ub, results=res)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            lb.copy_(lb0)
            ub.copy_(ub0)
            prob.propagate_batch(lb, ub, results=res)
        times = []
        for _ in range(5):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return float(np.median(times)), pkg.batch_results(res)

    t_def, rs = graph_ms()
    rep = prob.autotune(lb0, ub0, reps=3)
    t_tuned, rs_tuned = graph_ms()
    assert rs_tuned == rs
    nnz = sum(r["nnz_updates"] for r in rs)
    t_best = min(t_def, t_tuned)
    bbytes = 12 * nnz + 80 * big.n    # per nonzero processed; bounds in, both buffers, bounds out
    hbm, _ = peaks()
    return {"workload": f"{len(parts)} uneven instances, {big.nnz} nnz total (one graph-captured launch)",
            "roofline": {"bound": "hbm", "kernel": "bp_kernel (batch)", "bytes": bbytes,
                         "achieved": bbytes / (t_best / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bbytes / (t_best / 1e3) / 1e9 / hbm},
            "nnz_updates_per_s": nnz / (min(t_def, t_tuned) / 1e3), "ms": min(t_def, t_tuned),
            "nnz_updates": nnz, "ms_default": t_def, "ms_autotuned": t_tuned, "autotune": rep,
            "rounds_max": max(r["rounds"] for r in rs),
            "infeasible": sum(1 for r in rs if r["status"] == 1)}


def _verified(pkg, torch, prob, p, xo):
    """A FEASIBLE fix-and-propagate result checked again: integer values integral, a fresh
    propagation from the original bounds with the integer variables fixed not infeasible, and
    (with SciPy) a continuous completion within 1e-6 of every row (HiGHS)."""
    import numpy as np
    ints = p.is_int == 1
    if not (xo[ints] == np.round(xo[ints])).all():
        return False
    lo, hi = p.lb.copy(), p.ub.copy()
    lo[ints] = hi[ints] = xo[ints]
    lt, ut = torch.tensor(lo, device=prob.device), torch.tensor(hi, device=prob.device)
    if prob.propagate(lt, ut)["status"] == 1:
        return False
    try:
        import scipy.sparse as sp
        from scipy.optimize import linprog
    except ImportError:
        return True
    A = sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))
    cont = np.flatnonzero(~ints)
    rhs = p.g - A[:, np.flatnonzero(ints)] @ xo[ints] + 1e-6
    r = linprog(np.zeros(len(cont)), A_ub=A[:, cont], b_ub=rhs, bounds=list(zip(p.lb[cont], p.ub[cont])),
                method="highs")
    return r.status == 0


def _sign_test(wins, losses):
    """Two-sided exact sign test p-value for `wins` against `losses` (ties dropped)."""
    import math
    k, n = min(wins, losses), wins + losses
    if n == 0:
        return None
    return min(1.0, 2.0 * sum(math.comb(n, i) for i in range(k + 1)) / 2.0 ** n)


def learned_experiment(pkg, torch, dev, nnz, eq_fraction, train_idx, train_seeds, test_idx, test_seeds,
                       lp_iterations=0):
    """Train the scorer on the plain trajectories of `train_idx` rounding instances (one run per
    seed of `train_seeds`, labels from the runs that ended feasible), then run both orders with
    the same seeds on the held-out `test_idx` instances.  Feasible means verified again (fresh
    propagation with the integers fixed, and a continuous completion by HiGHS).  Bulks to
    feasibility are compared paired: over the (instance, seed) runs that both orders solve.
    lp_iterations > 0: the point to round is the approximate LP (pdhg_solve from zero, that many
    iterations, restarts every 100) instead of the planted point plus noise."""
    import numpy as np
    from paper_2510_20499_gb300 import learned, synth
    fp = dict(bulk_rule=1, fraction=0.01)
    t0 = time.perf_counter()
    data = []
    for i in train_idx:
        p, x = synth.rounding_instance(i, nnz, eq_fraction=eq_fraction)
        prob = pkg.Problem(p)
        xd, lb, ub = (torch.tensor(a, device=dev) for a in (x, p.lb, p.ub))
        if lp_iterations:
            xd = _lp_point(prob, p, lb, ub, torch, dev, lp_iterations)
        d = learned.collect(prob, xd, lb, ub, seeds=train_seeds, **fp)
        d["runs"] = None
        data.append(d)
        del prob
    scorer = pkg.Scorer(seed=3)
    losses = learned.train(scorer, data, epochs=6, batch=4096, lr=3e-3, seed=0)
    t_train = time.perf_counter() - t0
    out = {"nnz": nnz, "eq_fraction": eq_fraction,
           "point": f"approximate LP ({lp_iterations} PDHG iterations)" if lp_iterations else "planted + N(0, 0.3)",
           "train": {"instances": len(train_idx), "seeds": len(train_seeds),
                     "runs": len(train_idx) * len(train_seeds),
                     "feasible_runs": int(sum(d["feasible"] for d in data)),
                     "labelled_instances": int(sum(d["labels"] is not None for d in data)),
                     "labelled_rows": int(sum(d["feat"].shape[0] for d in data if d["labels"] is not None)),
                     "loss_first_last": [losses[0], losses[-1]] if losses else None, "seconds": t_train}}
    del data
    arms = {"plain": [], "learned": []}
    t_run = {"plain": 0.0, "learned": 0.0}
    t1 = time.perf_counter()
    for i in test_idx:
        p, x = synth.rounding_instance(i, nnz, eq_fraction=eq_fraction)
        prob = pkg.Problem(p)
        xd, lb, ub = (torch.tensor(a, device=dev) for a in (x, p.lb, p.ub))
        if lp_iterations:
            xd = _lp_point(prob, p, lb, ub, torch, dev, lp_iterations)
        order, up = learned.scores(prob, scorer, xd, lb, ub)
        for s in test_seeds:
            for arm, kw in (("plain", {}), ("learned", dict(order_score=order, up_prob=up))):
                torch.cuda.synchronize()
                ta = time.perf_counter()
                xo, r = prob.fix_and_propagate(xd, lb, ub, seed=s, **kw, **fp)
                t_run[arm] += time.perf_counter() - ta
                r["verified"] = r["status"] == 0 and _verified(pkg, torch, prob, p, xo.cpu().numpy())
                arms[arm].append(r)
        del prob
    for arm, rs in arms.items():
        ok = [r for r in rs if r["verified"]]
        out[arm] = {"runs": len(rs), "feasible_reported": sum(r["status"] == 0 for r in rs),
                    "feasible_verified": len(ok),
                    "bulks_to_feasibility": float(np.mean([r["bulks"] for r in ok])) if ok else None,
                    "bulks_mean_all_runs": float(np.mean([r["bulks"] for r in rs])),
                    "fixed_by_choice_mean": float(np.mean([r["fixed_by_choice"] for r in rs])),
                    "seconds_per_run": t_run[arm] / len(rs)}
    both = [(a["bulks"], b["bulks"]) for a, b in zip(arms["plain"], arms["learned"]) if a["verified"] and b["verified"]]
    wins = sum(bl < bp for bp, bl in both)
    losses_ = sum(bl > bp for bp, bl in both)
    only_p = sum(a["verified"] and not b["verified"] for a, b in zip(arms["plain"], arms["learned"]))
    only_l = sum(b["verified"] and not a["verified"] for a, b in zip(arms["plain"], arms["learned"]))
    out["paired"] = {
        "runs_both_feasible": len(both),
        "bulks_plain": float(np.mean([q[0] for q in both])) if both else None,
        "bulks_learned": float(np.mean([q[1] for q in both])) if both else None,
        "bulks_ratio_learned_over_plain": (float(np.mean([q[1] for q in both]) / np.mean([q[0] for q in both]))
                                           if both else None),
        "learned_fewer_bulks": wins, "learned_more_bulks": losses_, "same_bulks": len(both) - wins - losses_,
        "sign_test_p": _sign_test(wins, losses_),
        "feasible_plain_only": only_p, "feasible_learned_only": only_l,
        "feasibility_sign_test_p": _sign_test(only_l, only_p)}
    out["test_seconds"] = time.perf_counter() - t1
    return out


def _lp_point(prob, p, lb, ub, torch, dev, iterations):
    """The approximate LP's primal iterate (pdhg_solve from zero, restarts every 100)."""
    x = torch.zeros(p.n, dtype=torch.float64, device=dev).clamp_(lb, ub)
    y = torch.zeros(p.m, dtype=torch.float64, device=dev)
    prob.pdhg(lb, ub, x, y, iterations=iterations, restart_period=100)
    return x


def learned_extra(pkg, torch, dev):
    """The learned rounding order against the paper's order in fix-and-propagate (1% of the
    integer variables per bulk), at two sizes.  100k nonzeros (20% equality pairs): trained on 16
    instances x 8 seeds, tested on 12 held-out instances x 4 seeds.  1M nonzeros (1% equality
    pairs, with which the plain method reaches feasibility in part of the runs): trained on 16
    instances x 4 seeds, tested on 8 held-out instances x 2 seeds, once from the planted point
    plus noise and once from the approximate LP (2,000 PDHG iterations).  The full 1M experiment
    (160 training and 40 test instances) is the separate `learned_full` extra."""
    out = {"workload": "rounding instances (mixed power-law, planted point + N(0, 0.3) as the fractional point)"}
    out["100k_nnz"] = learned_experiment(pkg, torch, dev, 100_000, 0.2, range(16), range(100, 108),
                                         range(1000, 1012), range(1, 5))
    out["1m_nnz"] = learned_experiment(pkg, torch, dev, 1_000_000, 0.01, range(16), range(100, 104),
                                       range(2000, 2008), range(1, 3))
    out["1m_nnz_lp_point"] = learned_experiment(pkg, torch, dev, 1_000_000, 0.01, range(16), range(100, 104),
                                                range(2000, 2008), range(1, 3), lp_iterations=2000)
    return out


def learned_full_extra(pkg, torch, dev):
    """The learned rounding order at 1M nonzeros (1% equality pairs): trained on 160 instances x
    2 seeds, tested on 40 held-out instances x 4 seeds (several minutes on one GPU)."""
    out = {"workload": "rounding instances (mixed power-law, planted point + N(0, 0.3) as the fractional point)"}
    out["1m_nnz"] = learned_experiment(pkg, torch, dev, 1_000_000, 0.01, range(160), range(100, 102),
                                       range(2000, 2040), range(1, 5))
    return out


def fp_extra(pkg, torch, dev):
    """Plain fix-and-propagate (the paper's order, 1% bulks) on the 1M-nonzero rounding instance:
    seconds per run, bulks per second, and the bytes the bulks must move (12 B per nonzero the
    candidate propagations process, plus per bulk the two candidate vectors' bounds, filled from
    the current ones: 2 x 32 B per variable)."""
    from paper_2510_20499_gb300 import synth
    p, x = synth.rounding_instance(2000, 1_000_000)
    prob = pkg.Problem(p)
    xd, lb, ub = (torch.tensor(a, device=dev) for a in (x, p.lb, p.ub))
    kw = dict(bulk_rule=1, fraction=0.01, seed=1)
    prob.fix_and_propagate(xd, lb, ub, **kw)          # warm-up (loads the instance pair)
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, r = prob.fix_and_propagate(xd, lb, ub, **kw)
        runs.append((time.perf_counter() - t0, r))
    t, r = sorted(runs, key=lambda q: q[0])[1]
    fbytes = 12 * r["nnz_updates"] + r["bulks"] * 64 * p.n
    hbm, _ = peaks()
    return {"workload": f"rounding instance 2000 ({p.m} x {p.n}, {p.nnz} nnz), 1% bulks, seed 1",
            "seconds_per_run": t, "bulks": r["bulks"], "bulks_per_s": r["bulks"] / t,
            "us_per_bulk": 1e6 * t / r["bulks"], "status": r["status"], "nnz_updates": r["nnz_updates"],
            "roofline": {"bound": "hbm", "kernel": "fix_and_propagate (whole run)", "bytes": fbytes,
                         "achieved": fbytes / t / 1e9, "peak": hbm, "unit": "GB/s", "frac": fbytes / t / 1e9 / hbm}}


def pdhg_extra(pkg, torch, dev):
    """The approximate LP (pdhg_solve) on the benchmark instance (200k x 500k, 5M nonzeros;
    infinite bounds boxed at +-1000, objective N(0, 1)): time per PDHG iteration from the
    difference of a 220- and a 20-iteration call (the start and the KKT evaluation cancel), and
    its roofline.  Algorithmic bytes per iteration: both copies of the matrix (CSR for A xe,
    transpose for A^T y: 12 B per nonzero each), per variable x, c, l, u read, x+ and the
    extrapolation written, the extrapolation read by the rows and the restart sum read and
    written (72 B), per row y, g read, y+ written and the restart sum read and written (40 B).
    Then the same 220 iterations with 10 passes of Ruiz preconditioning: the KKT measures of the
    original problem beside the unscaled ones, and the call's time."""
    import numpy as np
    from paper_2510_20499_gb300 import synth
    p = synth.mixed_powerlaw()
    p.lb = np.where(np.isfinite(p.lb), p.lb, -1000.0)
    p.ub = np.where(np.isfinite(p.ub), p.ub, 1000.0)
    p.c = np.random.default_rng(5).normal(0, 1, p.n)
    prob = pkg.Problem(p)
    lb, ub = torch.tensor(p.lb, device=dev), torch.tensor(p.ub, device=dev)

    def run(iters, scaling=0):
        x = torch.zeros(p.n, dtype=torch.float64, device=dev)
        y = torch.zeros(p.m, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = prob.pdhg(lb, ub, x, y, iterations=iters, restart_period=100, scaling_iterations=scaling)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r
    run(20)
    t_short = min(run(20)[0] for _ in range(3))
    runs = [run(220) for _ in range(3)]
    t_long, r = min(runs, key=lambda q: q[0])
    per_it = (t_long - t_short) / 200.0
    # the same 220 iterations on the Ruiz-scaled problem (10 passes), measures of the original
    run(220, 10)
    t_sc, r_sc = run(220, 10)
    bytes_it = 24 * p.nnz + 72 * p.n + 40 * p.m
    hbm, _ = peaks()
    return {"workload": f"mixed power-law {p.m} x {p.n}, {p.nnz} nnz (bounds boxed at +-1000, c ~ N(0, 1)), "
                        "restarts every 100",
            "ms_per_iteration": per_it, "iterations_per_s": 1e3 / per_it,
            "after_220": {k: r[k] for k in ("primal_residual", "dual_residual", "primal_obj", "dual_obj")},
            "after_220_ruiz10": dict({k: r_sc[k] for k in ("primal_residual", "dual_residual", "primal_obj", "dual_obj")},
                                     ms_call=t_sc),
            "roofline": {"bound": "hbm", "kernel": "k_pdhg_cols + k_pdhg_rows + k_pdhg_long (one iteration)",
                         "bytes": bytes_it, "achieved": bytes_it / per_it / 1e6, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_it / per_it / 1e6 / hbm}}


def local_mip_extra(pkg, torch, dev):
    """The local search's move scoring (local_search_mtm) on the knapsack/cover instance (50k x
    100k, 1M nonzeros) from a random 0/1 point: time per iteration (every violated row's
    candidates scored in full, the best applied or the weights bumped) from the difference of a
    1,100- and a 100-iteration call, and the violation left."""
    import numpy as np
    from paper_2510_20499_gb300 import synth
    p = synth.knapsack_cover()
    prob = pkg.Problem(p)
    lb, ub = torch.tensor(p.lb, device=dev), torch.tensor(p.ub, device=dev)
    x0 = np.clip((np.random.default_rng(3).random(p.n) < 0.5).astype(float), p.lb, p.ub)

    def run(iters):
        x = torch.tensor(x0, device=dev)
        w = torch.ones(p.m, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = prob.local_search(lb, ub, x, w, iterations=iters)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r
    run(100)
    t_short = min(run(100)[0] for _ in range(3))
    t_long, r = min((run(1100) for _ in range(3)), key=lambda q: q[0])
    per_it = (t_long - t_short) / 1000.0
    r0 = run(0)[1]
    return {"workload": f"knapsack/cover {p.m} x {p.n}, {p.nnz} nnz, random 0/1 start",
            "ms_per_iteration": per_it, "iterations_per_s": 1e3 / per_it,
            "start": {"violated": r0["violated"], "weighted_violation": r0["weighted_violation"]},
            "after_1100": {k: r[k] for k in ("moves", "bumps", "violated", "weighted_violation")}}


def efp_extra(pkg, torch, dev):
    """The extended feasibility pump (extended_fp, generation mode) on the knapsack/cover instance
    (50k x 100k, 1M nonzeros, objective N(0, 1)): where the feasible point was found, rounds,
    cycle breaks, wall time of the call (CUDA events), and the point checked row by row; the
    improvement mode (ten rounds with the objective cut, each incumbent polished by the local
    search's objective moves); then 2,000 iterations of the local
    search with its objective moves from the generation mode's point (time per iteration, the
    incumbent's objective, the incumbent checked row by row)."""
    import numpy as np
    import scipy.sparse as sp
    from paper_2510_20499_gb300 import synth
    p = synth.knapsack_cover()
    p.c = np.random.default_rng(7).normal(0, 1, p.n)
    prob = pkg.Problem(p)
    lb, ub = torch.tensor(p.lb, device=dev), torch.tensor(p.ub, device=dev)
    kw = dict(rounds=10, lp_iterations=300, ls_iterations=200, seed=1)
    prob.extended_fp(lb, ub, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x, r = prob.extended_fp(lb, ub, **kw)
    e1.record()
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    A = sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))
    fin = np.isfinite(p.g)
    ok = bool(((A @ xh)[fin] <= p.g[fin] + 1e-9).all()) and bool(((xh >= p.lb) & (xh <= p.ub)).all())
    out = {"workload": f"knapsack/cover {p.m} x {p.n}, {p.nnz} nnz, c ~ N(0, 1); " + ", ".join(f"{k}={v}" for k, v in kw.items()),
           "seconds": e0.elapsed_time(e1) / 1e3, "result": r, "point_satisfies_every_row": ok,
           "objective": float(p.c @ xh)}
    # improvement mode: the objective cut at each incumbent, each incumbent polished by the local
    # search's objective moves, ten rounds
    e0.record()
    xi, ri = prob.extended_fp(lb, ub, improve=True, polish=True, **dict(kw, rounds=10))
    e1.record()
    torch.cuda.synchronize()
    xih = xi.cpu().numpy()
    oki = bool(((A @ xih)[fin] <= p.g[fin] + 1e-9).all()) and bool(((xih >= p.lb) & (xih <= p.ub)).all())
    out["improvement_mode"] = {"rounds": 10, "polish": True, "seconds": e0.elapsed_time(e1) / 1e3, "result": ri,
                               "point_satisfies_every_row": oki, "objective_checked": float(p.c @ xih)}
    if r["status"] == 0:
        # the local search's objective moves (lift, breakthrough) from the pump's feasible point
        iters = 2000
        xs = x.clone()
        w = torch.ones(p.m, dtype=torch.float64, device=dev)
        xb = torch.empty_like(xs)
        torch.cuda.synchronize()
        e0.record()
        ro = prob.local_search_objective(lb, ub, xs, w, xb, iterations=iters)
        e1.record()
        torch.cuda.synchronize()
        bh = xb.cpu().numpy()
        okb = bool(((A @ bh)[fin] <= p.g[fin] + 1e-9).all()) and bool(((bh >= p.lb) & (bh <= p.ub)).all())
        out["objective_moves"] = {
            "iterations": iters, "ms_per_iteration": e0.elapsed_time(e1) / iters,
            "result": {k: ro[k] for k in ("moves", "bumps", "lifts", "breakthroughs", "improvements", "found",
                                          "best_objective", "obj_weight", "violated")},
            "best_satisfies_every_row": okb, "best_objective_checked": float(p.c @ bh)}
    return out


def scorer_extra(pkg, torch, dev, tflops_peak):
    """The scorer's forward and training-step throughput on 1M rows of BF16 features (the
    tcgen05 MLP kernel k_mlp), against the measured BF16 tensor peak."""
    scorer = pkg.Scorer(seed=3)
    rows = 1_000_000
    g = torch.Generator(device="cpu")
    g.manual_seed(0)
    X = torch.randn(rows, 16, generator=g).to(dev).to(torch.bfloat16)
    Y = (torch.rand(rows, 2, generator=g) > 0.5).float().to(dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 20
    t_f = timed(lambda: scorer.forward(X))
    t_t = timed(lambda: scorer.train_step(X, Y, 1e-6, want_loss=False))
    fl_f = 2 * (16 * 64 + 64 * 64 + 64 * 2)          # forward flops per row
    fl_t = 3 * fl_f                                   # forward + input and weight gradients
    achieved = fl_f * rows / (t_f / 1e3) / 1e12
    return {"rows": rows, "forward_ms": t_f, "forward_rows_per_s": rows / (t_f / 1e3),
            "train_step_ms": t_t, "train_rows_per_s": rows / (t_t / 1e3),
            "roofline": {"bound": "tensor", "kernel": "k_mlp (forward)", "achieved": achieved,
                         "peak": tflops_peak, "unit": "TFLOP/s", "frac": achieved / tflops_peak,
                         "train_achieved": fl_t * rows / (t_t / 1e3) / 1e12}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import paper_2510_20499_gb300 as pkg
    from paper_2510_20499_gb300 import synth

    p = synth.mixed_powerlaw()
    prob = pkg.Problem(p)
    dev = torch.device("cuda", local)
    lb0 = torch.tensor(p.lb, device=dev)
    ub0 = torch.tensor(p.ub, device=dev)
    lb, ub = lb0.clone(), ub0.clone()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    # one traced run (untimed) gives the round structure for the byte count
    MR = 10000
    tr = torch.zeros(4 * MR, dtype=torch.int64, device=dev)
    lb.copy_(lb0)
    ub.copy_(ub0)
    r0 = prob.propagate(lb, ub, trace=tr, max_rounds=MR)
    t = tr[: 4 * r0["rounds"]].view(-1, 4).cpu().numpy()
    bytes_launch = algorithmic_bytes(t[:, 0], t[:, 1], t[:, 2], p.n)

    def step(timed_events=None):
        lb.copy_(lb0)
        ub.copy_(ub0)
        if timed_events:
            timed_events[0].record(stream)
        r = prob.propagate(lb, ub, sync=False)
        if timed_events:
            timed_events[1].record(stream)
        return r

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, nnz = [], [], 0
    for i in range(args.steps):
        flush.fill_(float(i))                     # L2 flushed between timed steps (untimed)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        lb.copy_(lb0)
        ub.copy_(ub0)
        e[1].record(stream)
        r = prob.propagate(lb, ub, sync=False)
        e[2].record(stream)
        torch.cuda.synchronize()
        step_ms.append(e[0].elapsed_time(e[2]))
        kern_ms.append(e[1].elapsed_time(e[2]))
        nnz += r0["nnz_updates"]
    torch.cuda.synchronize()
    res = prob.propagate(lb.copy_(lb0), ub.copy_(ub0))
    assert res == r0, (res, r0)
    clocks = sampler.finish()
    nnz_all, total_ms = whole_job(nnz, float(sum(step_ms)), dev)
    value = nnz_all / (total_ms / 1e3)

    # end to end through the C ABI with host (pinned) bounds: copies inside the timed region
    hl = torch.empty(p.n, dtype=torch.float64).pin_memory()
    hu = torch.empty(p.n, dtype=torch.float64).pin_memory()
    hl0, hu0 = torch.from_numpy(p.lb.copy()), torch.from_numpy(p.ub.copy())
    e2e_ms = []
    for i in range(max(3, args.steps // 2)):
        hl.copy_(hl0)
        hu.copy_(hu0)
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr = prob.propagate(hl.numpy(), hu.numpy())     # library copies H2D, propagates, copies D2H
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert rr == r0
    e2e_value = r0["nnz_updates"] * world / (np.median(e2e_ms) / 1e3)

    hbm, peak_kind = peaks()
    kern_avg = float(np.mean(kern_ms))
    achieved = bytes_launch / (kern_avg / 1e3) / 1e9
    fp64_peak = pkg.fp64_rate()                      # measured here: FP64 FMA TFLOP/s
    fp64_achieved = 2.0 * r0["nnz_updates"] / (kern_avg / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rounds": r0["rounds"], "nnz_updates_per_step": r0["nnz_updates"],
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * p.n,
                "d2h_bytes_per_step": 16 * p.n + 48},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": kernel_traffic(),
                     "peak_kind": peak_kind, "bytes_per_launch": bytes_launch, "kernel": "bp_kernel",
                     "launch_ms": kern_avg,
                     "fp64": {"achieved": fp64_achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": fp64_achieved / fp64_peak,
                              "note": "one FMA (2 flops) per nonzero-update of the activities; peak: bp_fp64_rate, "
                                      "measured in this run"}},
    }
    if rank == 0 and not args.no_extras:
        todo = [e for e in args.extras.split(",") if e]
        bad = [e for e in todo
               if e not in ("probing", "batch", "fp", "learned", "learned_full", "scorer", "pdhg", "local_mip", "efp")]
        if bad:
            raise SystemExit(f"unknown extras: {bad}")
        fns = {"probing": lambda: probing_extra(pkg, torch, dev), "batch": lambda: batch_extra(pkg, torch, dev),
               "fp": lambda: fp_extra(pkg, torch, dev),
               "learned": lambda: learned_extra(pkg, torch, dev),
               "learned_full": lambda: learned_full_extra(pkg, torch, dev),
               "pdhg": lambda: pdhg_extra(pkg, torch, dev), "local_mip": lambda: local_mip_extra(pkg, torch, dev),
               "efp": lambda: efp_extra(pkg, torch, dev),
               "scorer": lambda: scorer_extra(pkg, torch, dev, tensor_peak())}
        out["extras"] = {e: fns[e]() for e in todo}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
