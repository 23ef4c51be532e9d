"""bp_propagate_noalloc (scratch in a fixed static device array) against bp_propagate (scratch
owned by the handle): the same results on consecutive calls, across problems that reuse the
one scratch array, and a clear rejection of problems above the scratch limit.

Collected last (file name) so that it also runs after everything else in the process."""
import ctypes as C

import pytest

from paper_2510_20499_gb300 import synth
from tests.gpu_helpers import assert_bounds_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu tests need a CUDA device")
    import paper_2510_20499_gb300 as pkg
    return pkg


def problems():
    return [
        synth.random_milp(31, 2000, 3000, len_lo=1, len_hi=400, inf_fraction=0.05, eq_fraction=0.2),
        synth.random_milp(32, 60, 6000, len_lo=500, len_hi=5000, integer_coefs=True),   # piece rows
        synth.binary_knapsack(),
    ]


def run(prob, p, fn):
    import torch
    gl = torch.tensor(p.lb, device="cuda")
    gu = torch.tensor(p.ub, device="cuda")
    r = getattr(prob, fn)(gl, gu)
    return gl.cpu().numpy(), gu.cpu().numpy(), r


def same(p, a, b):
    gl, gu, gr = a
    hl, hu, hr = b
    assert gr["error"] == 0 and hr["error"] == 0
    assert gr == hr, (gr, hr)
    assert_bounds_match(p, hl, hu, gl, gu)


def test_noalloc_matches_propagate_on_consecutive_calls(pkg):
    ps = problems()
    probs = [pkg.Problem(p) for p in ps]
    ref = [run(q, p, "propagate") for q, p in zip(probs, ps)]
    # two calls in a row on each problem
    for q, p, r in zip(probs, ps, ref):
        same(p, r, run(q, p, "propagate_noalloc"))
        same(p, r, run(q, p, "propagate_noalloc"))
    # the scratch passes from problem to problem and back
    for i in (0, 2, 1, 0, 1, 2):
        same(ps[i], ref[i], run(probs[i], ps[i], "propagate_noalloc"))
    # the handle's own buffers are untouched by the static-scratch calls
    for q, p, r in zip(probs, ps, ref):
        same(p, r, run(q, p, "propagate"))


def test_noalloc_leaves_free_device_memory_unchanged(pkg):
    """The entry point allocates nothing, not even on its first call for a new handle: the
    static scratch is reserved when the handle is created, so the device's free memory
    (cudaMemGetInfo) is the same before and after three calls."""
    import torch
    p = synth.random_milp(34, 3000, 4000, len_lo=1, len_hi=600, inf_fraction=0.05, eq_fraction=0.2)
    q = pkg.Problem(p)
    l0 = torch.tensor(p.lb, device="cuda")
    u0 = torch.tensor(p.ub, device="cuda")
    gl, gu = l0.clone(), u0.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rs = []
    for _ in range(3):
        gl.copy_(l0)
        gu.copy_(u0)
        rs.append(q.propagate_noalloc(gl, gu))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert rs[0] == rs[1] == rs[2] and rs[0]["error"] == 0
    same(p, run(q, p, "propagate"), (gl.cpu().numpy(), gu.cpu().numpy(), rs[2]))


def test_noalloc_full_size_workload(pkg):
    """The 200k x 500k, 5M-nonzero power-law instance fits the scratch (about 24.5 MB)."""
    p = synth.mixed_powerlaw()
    q = pkg.Problem(p)
    r = run(q, p, "propagate")
    same(p, r, run(q, p, "propagate_noalloc"))
    same(p, r, run(q, p, "propagate_noalloc"))


def test_noalloc_rejects_oversize_and_host_bounds(pkg):
    import torch
    big = synth.random_milp(33, 1000, 800_000, len_lo=1, len_hi=8)   # 44 B x 800k vars > 32 MiB
    q = pkg.Problem(big)
    gl = torch.tensor(big.lb, device="cuda")
    gu = torch.tensor(big.ub, device="cuda")
    with pytest.raises(pkg.GpuBpError) as e:
        q.propagate_noalloc(gl, gu)
    assert e.value.code == pkg.BP_ERR_CAPACITY
    assert "bytes of scratch" in str(e.value)
    # host bounds are refused on the host, before anything is enqueued
    p = synth.binary_knapsack()
    small = pkg.Problem(p)
    prm = pkg.params(bounds_mem=pkg.MEM_HOST)
    res = pkg.BpResult()
    hl, hu = p.lb.copy(), p.ub.copy()
    code = pkg.lib().bp_propagate_noalloc(small.h, C.c_void_p(hl.ctypes.data), C.c_void_p(hu.ctypes.data),
                                          C.byref(prm), C.byref(res), None)
    assert code == pkg.BP_ERR_INVALID
    # the oversize handle still propagates through the handle-owned path
    r = q.propagate(gl, gu)
    assert r["error"] == 0 and r["status"] in (0, 1, 2)
