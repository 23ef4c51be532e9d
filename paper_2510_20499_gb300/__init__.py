"""GB300 bound propagation, probing and fix-and-propagate for MILP.

Thin ctypes binding of the C ABI declared in include/gpubp.h.  It only marshals arguments:
every step of the computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  Importing works without a GPU; creating a problem needs the
compiled library and a CUDA device and raises otherwise (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpubp.so")

BP_OK, BP_ERR_INVALID, BP_ERR_CUDA, BP_ERR_OOM, BP_ERR_CAPACITY, BP_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
FIXPOINT, INFEASIBLE, ROUND_LIMIT = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1


class BpParams(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_rounds", C.c_int32), ("bounds_mem", C.c_int32),
                ("trace", C.c_void_p)]


class BpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("rounds", C.c_int32), ("first_infeasible_row", C.c_int32),
                ("first_infeasible_var", C.c_int32), ("nnz_updates", C.c_int64), ("n_changed", C.c_int64),
                ("error", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ProbeCache(C.Structure):
    _fields_ = [("status", C.c_void_p), ("rounds", C.c_void_p), ("nnz_updates", C.c_void_p),
                ("offsets", C.c_void_p), ("ent_var", C.c_void_p), ("ent_l", C.c_void_p),
                ("ent_u", C.c_void_p), ("cap", C.c_int64), ("needed", C.c_int64)]


class ProbeApplyResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("first_infeasible_pair", C.c_int32), ("first_infeasible_var", C.c_int32),
                ("fixed_pairs", C.c_int32), ("tightened", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class FpParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("bulk_rule", C.c_int32), ("last_single", C.c_int32),
                ("fraction", C.c_double), ("theta", C.c_double), ("max_rounds", C.c_int32),
                ("repair_max", C.c_int32), ("order_score", C.c_void_p), ("up_prob", C.c_void_p),
                ("repair_cycles", C.c_int32), ("reserved", C.c_int32)]


class FpCache(C.Structure):
    _fields_ = [("npairs", C.c_int32), ("reserved", C.c_int32), ("var", C.c_void_p), ("boxes", C.c_void_p),
                ("status", C.c_void_p), ("offsets", C.c_void_p), ("ent_var", C.c_void_p),
                ("ent_l", C.c_void_p), ("ent_u", C.c_void_p)]


class FpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("bulks", C.c_int32), ("bp_runs", C.c_int32), ("recoveries", C.c_int32),
                ("fixed_by_choice", C.c_int32), ("refuted", C.c_int32), ("nnz_updates", C.c_int64),
                ("repairs", C.c_int32), ("repair_runs", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PdhgParams(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restart_period", C.c_int32), ("step", C.c_double),
                ("primal_weight", C.c_double), ("objective", C.c_void_p), ("scaling_iterations", C.c_int32),
                ("reserved", C.c_int32)]


class PdhgResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("step", C.c_double),
                ("primal_weight", C.c_double), ("primal_residual", C.c_double), ("dual_residual", C.c_double),
                ("primal_obj", C.c_double), ("dual_obj", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LsParams(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("recompute_period", C.c_int32)]


class LsResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("moves", C.c_int32), ("bumps", C.c_int32), ("violated", C.c_int32),
                ("weighted_violation", C.c_double), ("objective", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LsObjParams(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("recompute_period", C.c_int32), ("obj_weight", C.c_double)]


class LsObjResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("moves", C.c_int32), ("bumps", C.c_int32), ("violated", C.c_int32),
                ("weighted_violation", C.c_double), ("objective", C.c_double), ("lifts", C.c_int32),
                ("breakthroughs", C.c_int32), ("improvements", C.c_int32), ("found", C.c_int32),
                ("best_objective", C.c_double), ("obj_weight", C.c_double), ("delta", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["found"] = bool(d["found"])
        return d


class EfpParams(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("lp_iterations", C.c_int32), ("ls_iterations", C.c_int32),
                ("cycle_window", C.c_int32), ("cycle_ratio", C.c_double), ("seed", C.c_uint64),
                ("improve", C.c_int32), ("polish", C.c_int32)]


class EfpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("found_at", C.c_int32), ("rounds", C.c_int32), ("cycles", C.c_int32),
                ("last_distance", C.c_double), ("improvements", C.c_int32), ("polished", C.c_int32),
                ("best_objective", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BpTuning(C.Structure):
    _fields_ = [("warp_min", C.c_int32), ("block_min", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("chunk_len", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class BpTuneReport(C.Structure):
    _fields_ = [("best", BpTuning), ("best_ms", C.c_float), ("default_ms", C.c_float), ("tried", C.c_int32),
                ("rejected", C.c_int32)]

    def as_dict(self):
        return dict(best=self.best.as_dict(), best_ms=self.best_ms, default_ms=self.default_ms, tried=self.tried,
                    rejected=self.rejected)


class GpuBpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gpubp error {code}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes); every symbol declared in include/gpubp.h
SIGNATURES = {
    "mip_load_csr": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                               C.POINTER(C.c_void_p)]),
    "mip_free": (C.c_int, [C.c_void_p]),
    "mip_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "mip_default_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bp_params_default": (None, [C.POINTER(BpParams)]),
    "bp_propagate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(BpParams), C.POINTER(BpResult),
                               C.c_void_p]),
    "bp_result_device": (C.c_void_p, [C.c_void_p]),
    "scorer_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]),
    "scorer_free": (None, [C.c_void_p]),
    "scorer_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "scorer_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "scorer_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_void_p, C.c_void_p]),
    "scorer_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "scorer_scores": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "scorer_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "scorer_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p,
                                    C.c_void_p]),
    "scorer_labels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_int32, C.c_void_p,
                                C.c_void_p]),
    "scorer_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "scorer_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "bp_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(BpTuning)]),
    "bp_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(BpTuning), C.c_void_p]),
    "bp_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(BpParams), C.c_int32,
                              C.POINTER(BpTuneReport), C.c_void_p]),
    "bp_propagate_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(BpParams),
                                       C.POINTER(BpResult), C.c_void_p]),
    "bp_propagate_from": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(BpParams),
                                    C.POINTER(BpResult), C.c_void_p]),
    "probe_split": (C.c_int, [C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_double)]),
    "bp_probe_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.POINTER(BpParams), C.POINTER(ProbeCache), C.c_void_p]),
    "bp_probe_batch_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.POINTER(BpParams), C.POINTER(ProbeCache), C.c_void_p, C.c_void_p]),
    "probe_cache_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(ProbeCache),
                                    C.POINTER(ProbeApplyResult), C.c_void_p]),
    "bp_probe_priority": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "fp_params_default": (None, [C.POINTER(FpParams)]),
    "efp_params_default": (None, [C.POINTER(EfpParams)]),
    "extended_fp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(EfpParams),
                              C.POINTER(EfpResult), C.c_void_p]),
    "local_search_mtm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(LsParams),
                                   C.POINTER(LsResult), C.c_void_p]),
    "local_search_objective": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(LsObjParams), C.POINTER(LsObjResult), C.c_void_p]),
    "pdhg_params_default": (None, [C.POINTER(PdhgParams)]),
    "pdhg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(PdhgParams),
                             C.POINTER(PdhgResult), C.c_void_p]),
    "fix_and_propagate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(FpCache),
                                    C.POINTER(FpParams), C.c_void_p, C.POINTER(FpResult), C.c_void_p]),
    "mip_set_instances": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "bp_propagate_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(BpParams), C.c_void_p,
                                     C.c_void_p]),
    "bp_fp64_rate": (C.c_int, [C.POINTER(C.c_double), C.c_void_p]),
    "bp_last_error": (C.c_char_p, []),
    "bp_version": (C.c_char_p, []),
}


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024   # BP_NOALLOC_SCRATCH_BYTES


def lib():
    """The loaded library; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GpuBpError(BP_ERR_CUDA, f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != BP_OK:
        raise GpuBpError(code, lib().bp_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise GpuBpError(BP_ERR_CUDA, "no CUDA device: the library has no CPU path")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def params(theta=1e-3, max_rounds=10000, bounds_mem=MEM_DEVICE, trace=None):
    p = BpParams()
    lib().bp_params_default(C.byref(p))
    p.theta, p.max_rounds, p.bounds_mem = float(theta), int(max_rounds), int(bounds_mem)
    p.trace = trace.data_ptr() if trace is not None else None
    return p


class Problem:
    """A MILP loaded into device memory (mip_load_csr).  `milp` has the attributes m, n,
    row_ptr, col, val, g, lb, ub, is_int and optionally c (numpy arrays)."""

    def __init__(self, milp, stream=None):
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.m, self.n = int(milp.m), int(milp.n)
        arrs = [torch.from_numpy(np.ascontiguousarray(milp.row_ptr, dtype=np.int64)),
                torch.from_numpy(np.ascontiguousarray(milp.col, dtype=np.int32)),
                torch.from_numpy(np.ascontiguousarray(milp.val, dtype=np.float64)),
                torch.from_numpy(np.ascontiguousarray(milp.g, dtype=np.float64)),
                torch.from_numpy(np.ascontiguousarray(milp.lb, dtype=np.float64)),
                torch.from_numpy(np.ascontiguousarray(milp.ub, dtype=np.float64)),
                torch.from_numpy(np.ascontiguousarray(milp.is_int, dtype=np.uint8))]
        c = getattr(milp, "c", None)
        if c is not None:
            arrs.append(torch.from_numpy(np.ascontiguousarray(c, dtype=np.float64)))
        d = [a.to(dev) for a in arrs]
        h = C.c_void_p()
        _check(lib().mip_load_csr(self.m, self.n, _ptr(d[0]), _ptr(d[1]), _ptr(d[2]), _ptr(d[3]), _ptr(d[4]),
                                  _ptr(d[5]), _ptr(d[6]), _ptr(d[7]) if c is not None else None, MEM_DEVICE,
                                  _stream(stream), C.byref(h)))
        self.h = h
        self.device = dev
        self.int_vars = np.flatnonzero(np.asarray(milp.is_int) != 0).astype(np.int32)   # host copy

    def close(self):
        if getattr(self, "h", None):
            lib().mip_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def default_bounds(self, stream=None):
        torch = _torch()
        lb = torch.empty(self.n, dtype=torch.float64, device=self.device)
        ub = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(lib().mip_default_bounds(self.h, _ptr(lb), _ptr(ub), _stream(stream)))
        return lb, ub

    def propagate(self, lb, ub, theta=1e-3, max_rounds=10000, stream=None, sync=True, trace=None):
        """bp_propagate on device tensors lb/ub (float64, modified in place) or host numpy
        arrays (copied in and out by the library).  Returns the result dict (after a stream
        synchronisation when sync=True).  trace: optional int64 device tensor of
        4 * max_rounds entries (rows, nonzeros, changed variables, end time in ns per round)."""
        host = isinstance(lb, np.ndarray)
        if trace is not None:
            assert trace.dtype.itemsize == 8 and trace.numel() >= 4 * max_rounds and trace.is_cuda
        prm = params(theta, max_rounds, MEM_HOST if host else MEM_DEVICE, trace)
        res = BpResult()
        if host:
            assert lb.dtype == np.float64 and ub.dtype == np.float64 and lb.flags.c_contiguous
            lp, up = C.c_void_p(lb.ctypes.data), C.c_void_p(ub.ctypes.data)
        else:
            assert lb.dtype.is_floating_point and lb.element_size() == 8 and lb.is_contiguous()
            lp, up = _ptr(lb), _ptr(ub)
        s = _stream(stream)
        _check(lib().bp_propagate(self.h, lp, up, C.byref(prm), C.byref(res), s))
        if sync:
            _torch().cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return res.as_dict()


def _probe_cache(torch, dev, P, cap):
    return dict(status=torch.empty(2 * P, dtype=torch.int32, device=dev),
                rounds=torch.empty(2 * P, dtype=torch.int32, device=dev),
                nnz_updates=torch.empty(2 * P, dtype=torch.int64, device=dev),
                offsets=torch.empty(2 * P + 1, dtype=torch.int64, device=dev),
                var=torch.empty(max(1, cap), dtype=torch.int32, device=dev),
                l=torch.empty(max(1, cap), dtype=torch.float64, device=dev),
                u=torch.empty(max(1, cap), dtype=torch.float64, device=dev))


def _probe_batch(prob, root_lb, root_ub, var, boxes, theta=1e-3, max_rounds=10000, cap=None, stream=None):
    """bp_probe_batch on device tensors: root bounds (float64, n), var (int32, P), boxes
    (float64, P x 4).  Returns the cache as device tensors; grows its capacity when needed."""
    torch = _torch()
    P = int(var.numel())
    cap = int(cap) if cap is not None else max(1024, 16 * P)
    prm = params(theta, max_rounds)
    while True:
        c = _probe_cache(torch, prob.device, P, cap)
        pc = ProbeCache(_ptr(c["status"]).value, _ptr(c["rounds"]).value, _ptr(c["nnz_updates"]).value,
                        _ptr(c["offsets"]).value, _ptr(c["var"]).value, _ptr(c["l"]).value, _ptr(c["u"]).value,
                        cap, 0)
        code = lib().bp_probe_batch(prob.h, _ptr(root_lb), _ptr(root_ub), P, _ptr(var), _ptr(boxes), C.byref(prm),
                                    C.byref(pc), _stream(stream))
        if code == BP_ERR_CAPACITY:
            cap = int(pc.needed)
            continue
        _check(code)
        n = int(pc.needed)
        c["var"], c["l"], c["u"] = c["var"][:n], c["l"][:n], c["u"][:n]
        return c


Problem.probe_batch = _probe_batch


def _cache_struct(c, cap=None):
    return ProbeCache(_ptr(c["status"]).value, _ptr(c["rounds"]).value, _ptr(c["nnz_updates"]).value,
                      _ptr(c["offsets"]).value, _ptr(c["var"]).value, _ptr(c["l"]).value, _ptr(c["u"]).value,
                      int(c["var"].numel()) if cap is None else int(cap), 0)


def _probe_batch_async(prob, root_lb, root_ub, var, boxes, cache, status_dev, theta=1e-3, max_rounds=10000,
                       stream=None):
    """bp_probe_batch_async into a preallocated cache (dict of device tensors as probe_batch
    returns, entries of its full capacity) and status_dev (int64 device tensor of 2: entries
    needed, index flag).  Nothing is synchronised: the call can be captured in a CUDA graph once a
    call of the same size has run."""
    prm = params(theta, max_rounds)
    pc = _cache_struct(cache)
    _check(lib().bp_probe_batch_async(prob.h, _ptr(root_lb), _ptr(root_ub), int(var.numel()), _ptr(var), _ptr(boxes),
                                      C.byref(prm), C.byref(pc), _ptr(status_dev), _stream(stream)))


def _probe_cache_apply(prob, lb, ub, cache, stream=None):
    """probe_cache_apply: bounds valid for every solution from a probing cache (dict of
    probe_batch); lb/ub (float64 device, the root bounds) are tightened in place.  Returns the
    result dict."""
    P = int(cache["status"].numel()) // 2
    pc = _cache_struct(cache)
    r = ProbeApplyResult()
    _check(lib().probe_cache_apply(prob.h, _ptr(lb), _ptr(ub), P, C.byref(pc), C.byref(r), _stream(stream)))
    return r.as_dict()


Problem.probe_batch_async = _probe_batch_async
Problem.probe_cache_apply = _probe_cache_apply


def _probe_priority(prob, lb, ub, stream=None):
    """bp_probe_priority on device bounds; returns (key1, key2, key3, order) device tensors,
    order holding only the probed variables."""
    torch = _torch()
    n = prob.n
    k1 = torch.empty(n, dtype=torch.int32, device=prob.device)
    k2 = torch.empty(n, dtype=torch.float64, device=prob.device)
    k3 = torch.empty(n, dtype=torch.float64, device=prob.device)
    order = torch.empty(max(1, n), dtype=torch.int32, device=prob.device)
    cnt = C.c_int32(0)
    _check(lib().bp_probe_priority(prob.h, _ptr(lb), _ptr(ub), _ptr(k1), _ptr(k2), _ptr(k3), _ptr(order),
                                   C.byref(cnt), _stream(stream)))
    return k1, k2, k3, order[:cnt.value]


Problem.probe_priority = _probe_priority


def _fix_and_propagate(prob, x, lb, ub, seed=1, bulk_rule=0, fraction=0.01, last_single=36, theta=1e-3,
                       max_rounds=10000, cache=None, order_score=None, up_prob=None, repair_max=0, repair_cycles=8,
                       stream=None):
    """fix_and_propagate on device tensors (x, lb, ub float64).  cache: the dict returned by
    probe_batch plus 'pairs' (int32 device) and 'boxes' (float64 device, P x 4).  repair_max > 0
    turns the repair on (at most that many per run, each at most repair_cycles propagations).
    Returns (x_out device tensor, result dict)."""
    torch = _torch()
    prm = FpParams()
    lib().fp_params_default(C.byref(prm))
    prm.seed, prm.bulk_rule, prm.fraction, prm.last_single = int(seed), int(bulk_rule), float(fraction), int(last_single)
    prm.theta, prm.max_rounds = float(theta), int(max_rounds)
    prm.repair_max, prm.repair_cycles = int(repair_max), int(repair_cycles)
    prm.order_score = order_score.data_ptr() if order_score is not None else None
    prm.up_prob = up_prob.data_ptr() if up_prob is not None else None
    fc = _fp_cache_struct(cache) if cache is not None else None
    out = torch.empty_like(x)
    res = FpResult()
    _check(lib().fix_and_propagate(prob.h, _ptr(x), _ptr(lb), _ptr(ub), C.byref(fc) if fc is not None else None,
                                   C.byref(prm), _ptr(out), C.byref(res), _stream(stream)))
    return out, res.as_dict()


Problem.fix_and_propagate = _fix_and_propagate


def _pdhg(prob, lb, ub, x, y, iterations=1000, restart_period=100, step=0.0, primal_weight=0.0, objective=None,
          scaling_iterations=0, stream=None):
    """pdhg_solve (the approximate LP) on device tensors: lb, ub (n), x (n) and y (m) float64; x
    and y are the warm start and receive the final iterate; objective: a float64 device tensor in
    place of the handle's objective, or None; scaling_iterations: Ruiz passes (0: none).
    Returns the result dict."""
    prm = PdhgParams(int(iterations), int(restart_period), float(step), float(primal_weight),
                     objective.data_ptr() if objective is not None else None, int(scaling_iterations), 0)
    res = PdhgResult()
    _check(lib().pdhg_solve(prob.h, _ptr(lb), _ptr(ub), _ptr(x), _ptr(y), C.byref(prm), C.byref(res),
                            _stream(stream)))
    return res.as_dict()


Problem.pdhg = _pdhg


def _local_search(prob, lb, ub, x, w, iterations=100, recompute_period=0, stream=None):
    """local_search_mtm on device tensors: lb, ub and x (n), w (m) float64; x and w are updated
    in place.  Returns the result dict."""
    prm = LsParams(int(iterations), int(recompute_period))
    res = LsResult()
    _check(lib().local_search_mtm(prob.h, _ptr(lb), _ptr(ub), _ptr(x), _ptr(w), C.byref(prm), C.byref(res),
                                  _stream(stream)))
    return res.as_dict()


Problem.local_search = _local_search


def _local_search_objective(prob, lb, ub, x, w, x_best, iterations=100, obj_weight=1.0, recompute_period=0,
                            stream=None):
    """local_search_objective on device tensors: lb, ub, x and x_best (n), w (m) float64; x and
    w are updated in place, x_best receives each incumbent.  Returns the result dict."""
    prm = LsObjParams(int(iterations), int(recompute_period), float(obj_weight))
    res = LsObjResult()
    _check(lib().local_search_objective(prob.h, _ptr(lb), _ptr(ub), _ptr(x), _ptr(w), _ptr(x_best), C.byref(prm),
                                        C.byref(res), _stream(stream)))
    return res.as_dict()


Problem.local_search_objective = _local_search_objective


def _extended_fp(prob, lb, ub, rounds=20, lp_iterations=500, ls_iterations=200, cycle_window=3, cycle_ratio=0.1,
                 seed=1, improve=False, polish=False, stream=None):
    """extended_fp (Algorithm 2; generation mode, or improvement mode with improve=True, each
    incumbent polished by the local search's objective moves with polish=True) on device bounds.
    Returns (x device tensor, result dict)."""
    torch = _torch()
    prm = EfpParams(int(rounds), int(lp_iterations), int(ls_iterations), int(cycle_window), float(cycle_ratio),
                    int(seed), 1 if improve else 0, 1 if polish else 0)
    res = EfpResult()
    x = torch.empty_like(lb)
    _check(lib().extended_fp(prob.h, _ptr(lb), _ptr(ub), _ptr(x), C.byref(prm), C.byref(res), _stream(stream)))
    return x, res.as_dict()


Problem.extended_fp = _extended_fp

RESULT_FIELDS = [f for f, _ in BpResult._fields_ if f != "reserved"]


def _set_instances(prob, row_off, col_off, stream=None):
    """mip_set_instances with host offsets (numpy int32, length ninst+1)."""
    ro = np.ascontiguousarray(row_off, dtype=np.int32)
    co = np.ascontiguousarray(col_off, dtype=np.int32)
    _check(lib().mip_set_instances(prob.h, len(ro) - 1, C.c_void_p(ro.ctypes.data), C.c_void_p(co.ctypes.data),
                                   MEM_HOST, _stream(stream)))
    prob.ninst = len(ro) - 1


def _propagate_batch(prob, lb, ub, results=None, theta=1e-3, max_rounds=10000, stream=None):
    """bp_propagate_batch on device bounds; results: an int64 device tensor of
    ninst * 6 words (bp_result layout) or None (allocated).  Asynchronous: returns the
    device results tensor; decode it with batch_results()."""
    torch = _torch()
    if results is None:
        results = torch.empty(prob.ninst * C.sizeof(BpResult) // 4, dtype=torch.int32, device=prob.device)
    prm = params(theta, max_rounds)
    _check(lib().bp_propagate_batch(prob.h, _ptr(lb), _ptr(ub), C.byref(prm), _ptr(results), _stream(stream)))
    return results


def batch_results(results):
    """Decodes a device results tensor of bp_propagate_batch into a list of dicts."""
    raw = results.cpu().numpy().tobytes()
    size = C.sizeof(BpResult)
    out = []
    for i in range(len(raw) // size):
        r = BpResult.from_buffer_copy(raw[i * size:(i + 1) * size])
        out.append(r.as_dict())
    return out


def _propagate_from(prob, lb, ub, vars_dev, theta=1e-3, max_rounds=10000, stream=None, sync=True):
    """bp_propagate_from: round 0 holds the rows of the variables in vars_dev (int32 device)."""
    prm = params(theta, max_rounds)
    res = BpResult()
    _check(lib().bp_propagate_from(prob.h, _ptr(lb), _ptr(ub), _ptr(vars_dev), int(vars_dev.numel()), C.byref(prm),
                                   C.byref(res), _stream(stream)))
    if sync:
        _torch().cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return res.as_dict()


def _propagate_noalloc(prob, lb, ub, theta=1e-3, max_rounds=10000, stream=None, sync=True):
    """bp_propagate_noalloc on device bounds: the propagation of propagate(), with its scratch in
    the library's fixed static device array (no allocation; calls on one device must not overlap)."""
    prm = params(theta, max_rounds)
    res = BpResult()
    _check(lib().bp_propagate_noalloc(prob.h, _ptr(lb), _ptr(ub), C.byref(prm), C.byref(res), _stream(stream)))
    if sync:
        _torch().cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return res.as_dict()


def _get_tuning(prob):
    t = BpTuning()
    _check(lib().bp_get_tuning(prob.h, C.byref(t)))
    return t.as_dict()


def _set_tuning(prob, warp_min, block_min, blocks_per_sm, chunk_len=256, stream=None):
    t = BpTuning(int(warp_min), int(block_min), int(blocks_per_sm), int(chunk_len))
    _check(lib().bp_set_tuning(prob.h, C.byref(t), _stream(stream)))


def _autotune(prob, lb, ub, reps=3, theta=1e-3, max_rounds=10000, stream=None):
    """bp_autotune on device start bounds; returns the report dict (the best configuration is
    left set on the handle)."""
    rep = BpTuneReport()
    prm = params(theta, max_rounds)
    _check(lib().bp_autotune(prob.h, _ptr(lb), _ptr(ub), C.byref(prm), int(reps), C.byref(rep), _stream(stream)))
    return rep.as_dict()


def _fp_cache_struct(cache):
    return FpCache(int(cache["pairs"].numel()), 0, cache["pairs"].data_ptr(), cache["boxes"].data_ptr(),
                   cache["status"].data_ptr(), cache["offsets"].data_ptr(), cache["var"].data_ptr(),
                   cache["l"].data_ptr(), cache["u"].data_ptr())


def _scorer_features(prob, x, lb, ub, vars_, cache=None, stream=None):
    """scorer_features: BF16 features (torch.bfloat16, nvars x 16) of the variables vars_
    (int32 device tensor) under device bounds lb/ub and point x.  cache: as for
    fix_and_propagate (probe_batch's dict plus 'pairs' and 'boxes') or None."""
    torch = _torch()
    nv = int(vars_.numel())
    feat = torch.empty((nv, 16), dtype=torch.bfloat16, device=prob.device)
    fc = _fp_cache_struct(cache) if cache is not None else None
    _check(lib().scorer_features(prob.h, _ptr(x), _ptr(lb), _ptr(ub), C.byref(fc) if fc is not None else None,
                                 _ptr(vars_), nv, _ptr(feat), _stream(stream)))
    return feat


class Scorer:
    """The learned rounding scorer (16-64-64-2 MLP on the tensor cores)."""

    NPARAM = 5378

    def __init__(self, seed=1):
        h = C.c_void_p()
        _check(lib().scorer_create(16, 64, 2, int(seed), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().scorer_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.NPARAM, dtype=np.float32)
        _check(lib().scorer_get_params(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.NPARAM
        _check(lib().scorer_set_params(self.h, C.c_void_p(t.ctypes.data)))

    def forward(self, feat, stream=None):
        torch = _torch()
        out = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        _check(lib().scorer_forward(self.h, _ptr(feat), int(feat.shape[0]), _ptr(out), _stream(stream)))
        return out

    def scores(self, feat, vars_, order_score=None, up_prob=None, stream=None):
        torch = _torch()
        logits = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        _check(lib().scorer_scores(self.h, _ptr(feat), _ptr(vars_), int(feat.shape[0]), _ptr(logits),
                                   _ptr(order_score), _ptr(up_prob), _stream(stream)))
        return logits

    def gradient(self, feat, labels, stream=None):
        g = np.zeros(self.NPARAM, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(lib().scorer_gradient(self.h, _ptr(feat), _ptr(labels), int(feat.shape[0]),
                                     C.c_void_p(g.ctypes.data), C.byref(loss), _stream(stream)))
        return g, float(loss.value)

    def train_step(self, feat, labels, lr, stream=None, want_loss=True):
        """One Adam step; returns the batch loss (the call then synchronises), or None with
        want_loss=False (asynchronous)."""
        loss = C.c_float(0.0)
        _check(lib().scorer_train_step(self.h, _ptr(feat), _ptr(labels), int(feat.shape[0]), float(lr),
                                       C.byref(loss) if want_loss else None, _stream(stream)))
        return float(loss.value) if want_loss else None

    def save(self, path):
        _check(lib().scorer_save(self.h, str(path).encode()))

    def load(self, path):
        _check(lib().scorer_load(self.h, str(path).encode()))


def scorer_labels(x, x_out, vars_, labels, weight=1.0, first=False, stream=None):
    """scorer_labels: adds one feasible fix_and_propagate result x_out to the labels
    (float32 device tensor, nvars x 2) of the variables vars_ (int32 device tensor)."""
    _check(lib().scorer_labels(_ptr(x), _ptr(x_out), _ptr(vars_), int(vars_.numel()), float(weight),
                               1 if first else 0, _ptr(labels), _stream(stream)))
    return labels


Problem.scorer_features = _scorer_features
Problem.get_tuning = _get_tuning
Problem.set_tuning = _set_tuning
Problem.autotune = _autotune
Problem.propagate_from = _propagate_from
Problem.propagate_noalloc = _propagate_noalloc
Problem.set_instances = _set_instances
Problem.propagate_batch = _propagate_batch


def probe_split(is_int, l, u):
    out = (C.c_double * 4)()
    ok = lib().probe_split(int(is_int), float(l), float(u), out)
    return (out[0], out[1], out[2], out[3]) if ok else None


def fp64_rate(stream=None):
    """The device's measured FP64 FMA throughput in TFLOP/s (bp_fp64_rate)."""
    v = C.c_double(0.0)
    _check(lib().bp_fp64_rate(C.byref(v), _stream(stream)))
    return v.value


def version():
    return lib().bp_version().decode()
