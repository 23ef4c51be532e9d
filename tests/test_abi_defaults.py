"""Host-only parts of the C ABI, without a GPU: the parameter defaults equal those the header
documents, and every compute entry point rejects a null handle with BP_ERR_INVALID and a
readable message before it touches a device."""
import ctypes as C
import math

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2510_20499_gb300 import build
    try:
        path = build.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"nvcc unavailable: {e}")
    L = C.CDLL(path)
    L.bp_last_error.restype = C.c_char_p
    return L


def test_documented_defaults(lib):
    import paper_2510_20499_gb300 as pkg
    b = pkg.BpParams()
    lib.bp_params_default(C.byref(b))
    assert (b.theta, b.max_rounds, b.bounds_mem, b.trace) == (1e-3, 10000, 1, None)
    f = pkg.FpParams()
    lib.fp_params_default(C.byref(f))
    assert (f.seed, f.bulk_rule, f.last_single, f.fraction) == (1, 0, 36, 0.01)
    assert (f.repair_max, f.repair_cycles, f.order_score, f.up_prob) == (0, 8, None, None)
    d = pkg.PdhgParams()
    lib.pdhg_params_default(C.byref(d))
    assert (d.iterations, d.restart_period, d.step, d.primal_weight, d.objective, d.scaling_iterations) == \
        (1000, 100, 0.0, 0.0, None, 0)
    e = pkg.EfpParams()
    lib.efp_params_default(C.byref(e))
    assert (e.rounds, e.lp_iterations, e.ls_iterations, e.cycle_window, e.seed, e.improve, e.polish) == \
        (20, 500, 200, 3, 1, 0, 0)
    assert math.isclose(e.cycle_ratio, 0.1)


def test_null_handle_is_invalid(lib):
    import paper_2510_20499_gb300 as pkg
    null = C.c_void_p(None)
    calls = {
        "pdhg_solve": lambda: lib.pdhg_solve(null, null, null, null, null, null, C.byref(pkg.PdhgResult()), null),
        "local_search_mtm": lambda: lib.local_search_mtm(null, null, null, null, null, C.byref(pkg.LsParams(1, 0)),
                                                         C.byref(pkg.LsResult()), null),
        "local_search_objective": lambda: lib.local_search_objective(
            null, null, null, null, null, null, C.byref(pkg.LsObjParams(1, 0, 1.0)), C.byref(pkg.LsObjResult()), null),
        "extended_fp": lambda: lib.extended_fp(null, null, null, null, null, C.byref(pkg.EfpResult()), null),
    }
    for name, call in calls.items():
        assert call() == pkg.BP_ERR_INVALID, name
        assert b"null" in lib.bp_last_error(), name
