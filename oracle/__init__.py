"""CPU oracle for bound propagation, probing, probe priority and fix-and-propagate.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg, never by the library.  The C sources next to this file are plain
sequential IEEE-double code (built with -ffp-contract=off); this module only marshals
numpy arrays into them.  It shares no code with the GPU library.

Problems are passed as any object with the attributes m, n, row_ptr (int64), col (int32),
val (float64), g (float64) and is_int (uint8).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["bp_oracle.c", "fp_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")

FIXPOINT, INFEASIBLE, ROUND_LIMIT = 0, 1, 2
TOL = 1e-6


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


class BpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("rounds", C.c_int32),
                ("first_infeasible_row", C.c_int32), ("first_infeasible_var", C.c_int32),
                ("nnz_updates", C.c_int64), ("n_changed", C.c_int64),
                ("candidates", C.c_int64), ("fragile", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ApplyResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("first_infeasible_pair", C.c_int32), ("first_infeasible_var", C.c_int32),
                ("fixed_pairs", C.c_int32), ("tightened", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_load.restype = C.c_void_p
        L.orc_load.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                               C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_uint8),
                               C.POINTER(C.c_int32)]
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_normalize.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_bp.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                             C.c_int32, C.c_double, C.c_int32, C.c_int32, C.POINTER(BpResult),
                             C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_probe_split.argtypes = [C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.orc_probe_split.restype = C.c_int
        L.orc_probe_batch.restype = C.c_int64
        L.orc_probe_batch.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                      C.c_double, C.c_int32, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64]
        L.orc_probe_cache_apply.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(ApplyResult)]
        L.orc_probe_priority.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]
        _bind_fp(L)
    return _lib


class FpParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("bulk_rule", C.c_int32), ("fraction", C.c_double),
                ("last_single", C.c_int32), ("theta", C.c_double), ("max_rounds", C.c_int32),
                ("order_score", C.POINTER(C.c_double)), ("up_prob", C.POINTER(C.c_double)),
                ("repair_max", C.c_int32), ("repair_cycles", C.c_int32)]


class FpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("bulks", C.c_int32), ("bp_runs", C.c_int32), ("recoveries", C.c_int32),
                ("fixed_by_choice", C.c_int32), ("refuted", C.c_int32), ("nnz_updates", C.c_int64),
                ("fragile", C.c_int64), ("repairs", C.c_int32), ("repair_runs", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Cache(C.Structure):
    _fields_ = [("npairs", C.c_int32), ("var", C.POINTER(C.c_int32)), ("boxes", C.POINTER(C.c_double)),
                ("status", C.POINTER(C.c_int32)), ("offsets", C.POINTER(C.c_int64)),
                ("ent_var", C.POINTER(C.c_int32)), ("ent_l", C.POINTER(C.c_double)),
                ("ent_u", C.POINTER(C.c_double))]


def _bind_fp(L):
    L.orc_fix_and_propagate.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(Cache), C.POINTER(FpParams),
                                        C.POINTER(C.c_double), C.POINTER(FpResult)]
    L.orc_repair_step.restype = C.c_int32
    L.orc_repair_step.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32, C.c_int32,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_uint8),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.orc_implied_slack.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    L.orc_uniform.restype = C.c_double
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_splitmix64.argtypes = [C.c_uint64]


def uniform(seed, bulk, var, draw):
    return lib().orc_uniform(seed, bulk, var, draw)


def splitmix64(z):
    return lib().orc_splitmix64(z)


class Problem:
    """An oracle-side copy of a problem (CSR plus transpose)."""

    def __init__(self, milp):
        L = lib()
        self.m, self.n = int(milp.m), int(milp.n)
        self.row_ptr = np.ascontiguousarray(milp.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(milp.col, dtype=np.int32)
        self.val = np.ascontiguousarray(milp.val, dtype=np.float64)
        self.g = np.ascontiguousarray(milp.g, dtype=np.float64)
        self.is_int = np.ascontiguousarray(milp.is_int, dtype=np.uint8)
        err = C.c_int32(0)
        h = L.orc_load(self.m, self.n, _p(self.row_ptr, C.c_int64), _p(self.col, C.c_int32),
                       _p(self.val, C.c_double), _p(self.g, C.c_double), _p(self.is_int, C.c_uint8),
                       C.byref(err))
        if not h:
            raise ValueError(f"oracle rejected the problem (code {err.value})")
        self.h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self.h = None

    def normalize(self, lb, ub):
        lb = np.array(lb, dtype=np.float64)
        ub = np.array(ub, dtype=np.float64)
        lib().orc_normalize(self.h, _p(lb, C.c_double), _p(ub, C.c_double))
        return lb, ub

    def bp(self, lb, ub, w0=None, theta=1e-3, max_rounds=10000, mode=0, dlb=None, dub=None,
           trace=False):
        """Bound propagation; returns (lb, ub, result dict, (dlb, dub)).  With trace=True the
        result dict also holds the rows and nonzeros of every round."""
        lb = np.array(lb, dtype=np.float64)
        ub = np.array(ub, dtype=np.float64)
        dl = np.zeros(self.n) if dlb is None else np.array(dlb, dtype=np.float64)
        du = np.zeros(self.n) if dub is None else np.array(dub, dtype=np.float64)
        r = BpResult()
        if w0 is None:
            wp, wl = None, 0
        else:
            w0 = np.ascontiguousarray(w0, dtype=np.int32)
            wp, wl = _p(w0, C.c_int32), len(w0)
        tr = tn = None
        if trace:
            tr = np.zeros(max(1, max_rounds), dtype=np.int64)
            tn = np.zeros(max(1, max_rounds), dtype=np.int64)
        lib().orc_bp(self.h, _p(lb, C.c_double), _p(ub, C.c_double), _p(dl, C.c_double),
                     _p(du, C.c_double), wp, wl, float(theta), int(max_rounds), int(mode),
                     C.byref(r), None if tr is None else _p(tr, C.c_int64),
                     None if tn is None else _p(tn, C.c_int64))
        out = r.as_dict()
        if trace:
            out["trace_rows"] = tr[:r.rounds].copy()
            out["trace_nnz"] = tn[:r.rounds].copy()
        return lb, ub, out, (dl, du)

    def probe_batch(self, root_l, root_u, var, boxes, theta=1e-3, max_rounds=10000, cap=None):
        root_l = np.ascontiguousarray(root_l, dtype=np.float64)
        root_u = np.ascontiguousarray(root_u, dtype=np.float64)
        var = np.ascontiguousarray(var, dtype=np.int32)
        boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1)
        P = len(var)
        status = np.zeros(2 * P, dtype=np.int32)
        rounds = np.zeros(2 * P, dtype=np.int32)
        nnzu = np.zeros(2 * P, dtype=np.int64)
        offs = np.zeros(2 * P + 1, dtype=np.int64)
        if cap is None:
            cap = max(1, 64 * P)
        while True:
            ev = np.zeros(cap, dtype=np.int32)
            el = np.zeros(cap)
            eu = np.zeros(cap)
            need = lib().orc_probe_batch(self.h, _p(root_l, C.c_double), _p(root_u, C.c_double), P,
                                         _p(var, C.c_int32), _p(boxes, C.c_double), float(theta),
                                         int(max_rounds), _p(status, C.c_int32), _p(rounds, C.c_int32),
                                         _p(nnzu, C.c_int64), _p(offs, C.c_int64), _p(ev, C.c_int32),
                                         _p(el, C.c_double), _p(eu, C.c_double), cap)
            if need <= cap:
                return dict(status=status, rounds=rounds, nnz_updates=nnzu, offsets=offs,
                            var=ev[:need], l=el[:need], u=eu[:need])
            cap = int(need)

    def probe_cache_apply(self, lb, ub, cache):
        """Global bounds from a probing cache (dict of probe_batch); returns (lb, ub, result)."""
        lb = np.array(lb, dtype=np.float64)
        ub = np.array(ub, dtype=np.float64)
        st = np.ascontiguousarray(cache["status"], dtype=np.int32)
        off = np.ascontiguousarray(cache["offsets"], dtype=np.int64)
        ev = np.ascontiguousarray(cache["var"], dtype=np.int32)
        el = np.ascontiguousarray(cache["l"], dtype=np.float64)
        eu = np.ascontiguousarray(cache["u"], dtype=np.float64)
        r = ApplyResult()
        lib().orc_probe_cache_apply(self.h, _p(lb, C.c_double), _p(ub, C.c_double), len(st) // 2, _p(st, C.c_int32),
                                    _p(off, C.c_int64), _p(ev, C.c_int32), _p(el, C.c_double), _p(eu, C.c_double),
                                    C.byref(r))
        return lb, ub, r.as_dict()

    def probe_priority(self, lb, ub):
        lb = np.ascontiguousarray(lb, dtype=np.float64)
        ub = np.ascontiguousarray(ub, dtype=np.float64)
        k1 = np.zeros(self.n, dtype=np.int32)
        k2 = np.zeros(self.n)
        k3 = np.zeros(self.n)
        lib().orc_probe_priority(self.h, _p(lb, C.c_double), _p(ub, C.c_double), _p(k1, C.c_int32),
                                 _p(k2, C.c_double), _p(k3, C.c_double))
        return k1, k2, k3


def _fix_and_propagate(self, x, lb, ub, seed=1, bulk_rule=0, fraction=0.01, last_single=36, theta=1e-3,
                       max_rounds=10000, cache=None, order_score=None, up_prob=None, repair_max=0, repair_cycles=8):
    """Fix-and-propagate (Algorithm 1); cache: dict from probe_batch plus 'pairs' and 'boxes'.
    repair_max > 0 turns the repair on (at most that many repairs per run, each at most
    repair_cycles propagations; not with a cache).  Returns (x_out, result dict)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    out = np.zeros(self.n)
    osc = None if order_score is None else np.ascontiguousarray(order_score, dtype=np.float64)
    upp = None if up_prob is None else np.ascontiguousarray(up_prob, dtype=np.float64)
    prm = FpParams(seed, bulk_rule, fraction, last_single, theta, max_rounds,
                   None if osc is None else _p(osc, C.c_double), None if upp is None else _p(upp, C.c_double),
                   int(repair_max), int(repair_cycles))
    res = FpResult()
    cp = None
    keep = []
    if cache is not None:
        arrs = [np.ascontiguousarray(cache["pairs"], dtype=np.int32),
                np.ascontiguousarray(cache["boxes"], dtype=np.float64).reshape(-1),
                np.ascontiguousarray(cache["status"], dtype=np.int32),
                np.ascontiguousarray(cache["offsets"], dtype=np.int64),
                np.ascontiguousarray(cache["var"], dtype=np.int32),
                np.ascontiguousarray(cache["l"], dtype=np.float64),
                np.ascontiguousarray(cache["u"], dtype=np.float64)]
        keep = arrs
        cp = Cache(len(arrs[0]), _p(arrs[0], C.c_int32), _p(arrs[1], C.c_double), _p(arrs[2], C.c_int32),
                   _p(arrs[3], C.c_int64), _p(arrs[4], C.c_int32), _p(arrs[5], C.c_double), _p(arrs[6], C.c_double))
    rc = lib().orc_fix_and_propagate(self.h, _p(x, C.c_double), _p(lb, C.c_double), _p(ub, C.c_double),
                                     C.byref(cp) if cp is not None else None, C.byref(prm), _p(out, C.c_double),
                                     C.byref(res))
    del keep
    if rc != 0:
        raise ValueError("the repair is defined without a probing cache")
    return out, res.as_dict()


Problem.fix_and_propagate = _fix_and_propagate


def _repair_step(self, l, u, row, var, lb, ub, chosen, cval):
    """One repair step (see fp_oracle.c) after an infeasible propagation with final bounds (l, u),
    first infeasible row `row` (or -1) and first crossing variable `var` (or -1).  Returns
    (moved variable or -1, new cval, fragile count)."""
    l = np.ascontiguousarray(l, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    ch = np.ascontiguousarray(chosen, dtype=np.uint8)
    cv = np.array(cval, dtype=np.float64)
    fr = C.c_int64(0)
    i = lib().orc_repair_step(self.h, _p(l, C.c_double), _p(u, C.c_double), int(row), int(var), _p(lb, C.c_double),
                              _p(ub, C.c_double), _p(ch, C.c_uint8), _p(cv, C.c_double), C.byref(fr))
    return int(i), cv, int(fr.value)


Problem.repair_step = _repair_step


def _implied_slack(self, lb, ub):
    """Implied slack S_i of every variable under bounds (lb, ub) (Section 2.3)."""
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    S = np.zeros(self.n)
    lib().orc_implied_slack(self.h, _p(lb, C.c_double), _p(ub, C.c_double), _p(S, C.c_double))
    return S


Problem.implied_slack = _implied_slack


def probe_split(is_int, l, u):
    """Branch boxes of an integer variable (Section 2.2); None when it is not probed."""
    out = (C.c_double * 4)()
    ok = lib().orc_probe_split(int(is_int), float(l), float(u), out)
    return (out[0], out[1], out[2], out[3]) if ok else None


def priority_order(k1, k2, k3, probeable_only=True):
    """Probe order: key1 descending, key2 descending, key3 ascending, index ascending."""
    idx = np.arange(len(k1))
    if probeable_only:
        idx = idx[k1 >= 0]
    # lexsort: last key is primary
    order = np.lexsort((idx, k3[idx], -k2[idx], -k1[idx]))
    return idx[order].astype(np.int32)
