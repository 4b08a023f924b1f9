"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and validates its arguments before touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1810_07806_gb300 import wcns

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(wcns_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert {"wcns_create", "wcns_rhs", "wcns_step_rk3", "wcns_destroy"} <= names
    lib = C.CDLL(wcns.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_are_the_papers():
    p = wcns.default_params()
    assert (p.C, p.eps, p.CT, p.q) == (1.0, 1e-40, 1e-5, 6)   # Eq. 16, Sec. 2.3
    assert p.characteristic == 1 and p.weights == 0 and p.diff == 0
    assert p.precision == wcns.FP64
    assert p.eps_js == 1e-6                                    # Eq. 14


def _create(grid, gamma=1.4, **kw):
    p = wcns.default_params(**kw)
    h = C.c_void_p()
    st = wcns.lib().wcns_create(C.byref(grid), gamma, C.byref(p), C.byref(h))
    return st, h


@pytest.mark.parametrize("bad", [
    dict(ndim=0), dict(ndim=4), dict(gamma=1.0), dict(q=0), dict(CT=0.5), dict(C=0.0),
    dict(flux=7), dict(characteristic=0), dict(entropy_fix=1), dict(precision=3), dict(cfl=0.0),
    dict(n=(1,)), dict(half_periodic=True), dict(weights=4), dict(weights=-1),
    dict(weights=wcns.W_JS, eps_js=0.0), dict(flux=3), dict(diff=3), dict(diff=-1)])
def test_create_rejects_bad_arguments_without_a_gpu(bad):
    ndim = bad.get("ndim", 1)
    n = bad.get("n", (16,))
    g = wcns.make_grid(max(1, min(ndim, 3)), n + (1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0))
    g.ndim = ndim
    if bad.get("half_periodic"):
        g.bc[0][0] = wcns.BC_PERIODIC
    kw = {k: v for k, v in bad.items() if k not in ("ndim", "n", "gamma", "half_periodic")}
    st, h = _create(g, bad.get("gamma", 1.4), **kw)
    assert st == wcns.ERR_INVALID
    assert h.value is None
    assert len(wcns.lib().wcns_last_error()) > 0


def test_null_arguments_are_rejected():
    L = wcns.lib()
    assert L.wcns_create(None, 1.4, None, None) == wcns.ERR_INVALID
    assert L.wcns_rhs(None, None, None, None, None) == wcns.ERR_INVALID
    assert L.wcns_step_rk3(None, None, 0.0, None, None) == wcns.ERR_INVALID
    assert L.wcns_destroy(None) == wcns.OK


@pytest.mark.parametrize("bad", [
    dict(kind=2), dict(kind=-1), dict(n=0), dict(count=0), dict(ld=15), dict(h=0.0),
    dict(h=float("nan")), dict(precision=wcns.FP32), dict(weights=9), dict(q=0), dict(null=True)])
def test_scalar_entry_points_validate_before_touching_a_gpu(bad):
    L = wcns._scalar_fns()
    p = wcns.default_params(**{k: v for k, v in bad.items() if k in ("precision", "weights", "q")})
    kind, n, count = bad.get("kind", 0), bad.get("n", 16), bad.get("count", 1)
    ld, h = bad.get("ld", 16), bad.get("h", 1.0 / 16)
    ptr = None if bad.get("null") else C.c_void_p(16)   # never dereferenced: rejected first
    assert L.wcns_scalar_rhs(kind, C.byref(p), n, h, count, ptr, ld, ptr, None) == wcns.ERR_INVALID
    assert L.wcns_scalar_run(kind, C.byref(p), n, h, 1.0, 4, count, ptr, ld, None) == wcns.ERR_INVALID
    assert len(wcns.lib().wcns_last_error()) > 0


def test_scalar_run_rejects_bad_time_arguments():
    L = wcns._scalar_fns()
    p = wcns.default_params()
    ptr = C.c_void_p(16)
    assert L.wcns_scalar_run(0, C.byref(p), 16, 0.1, 1.0, -1, 1, ptr, 16, None) == wcns.ERR_INVALID
    assert L.wcns_scalar_run(0, C.byref(p), 16, 0.1, float("inf"), 4, 1, ptr, 16, None) == wcns.ERR_INVALID
    # zero steps is a no-op that touches nothing
    assert L.wcns_scalar_run(0, C.byref(p), 16, 0.1, 1.0, 0, 1, ptr, 16, None) == wcns.OK


def test_batch_create_rejects_bad_arguments_without_a_gpu():
    L = wcns.lib()
    L.wcns_batch_create.argtypes = [C.c_int, C.c_double, C.POINTER(wcns.SchemeParams), C.c_longlong, C.c_int,
                                    C.POINTER(C.c_void_p)]
    for nd, mx, ni, kw in ((4, 1000, 4, {}), (1, 0, 4, {}), (1, 1000, 0, {}), (1, 1000, 4, dict(weights=7)),
                           (1, 1000, 4, dict(precision=2))):
        p = wcns.default_params(**kw)
        h = C.c_void_p()
        assert L.wcns_batch_create(nd, 1.4, C.byref(p), mx, ni, C.byref(h)) == wcns.ERR_INVALID
        assert h.value is None


@pytest.mark.parametrize("case", ["reflect_short", "kind4", "fixed_bad_rho", "fixed_bad_p", "gravity_nan"])
def test_create_rejects_bad_boundaries_without_a_gpu(case):
    g = wcns.make_grid(2, (16, 16), (0, 0), (1, 1), (0, 0))
    if case == "reflect_short":
        g.n[0] = 4
        g.bc[0][0] = wcns.BC_REFLECTING
    elif case == "kind4":
        g.bc[1][1] = 4
    elif case in ("fixed_bad_rho", "fixed_bad_p"):
        g.bc[1][0] = wcns.BC_FIXED
        state = (0.0, 0.0, 0.0, 1.0) if case == "fixed_bad_rho" else (1.0, 0.0, 0.0, -1.0)
        for v in range(4):
            g.bc_state[1][0][v] = state[v]
    else:
        g.gravity[1] = float("nan")
    st, h = _create(g)
    assert st == wcns.ERR_INVALID and h.value is None
    assert len(wcns.lib().wcns_last_error()) > 0


def test_noalloc_step_rejects_single_grid_features_without_a_gpu():
    L = wcns.lib()
    fn = L.wcns_step_rk3_noalloc
    fn.argtypes = [C.POINTER(wcns.Grid), C.c_double, C.POINTER(wcns.SchemeParams), C.c_void_p, C.c_double,
                   C.POINTER(C.c_double), C.c_void_p]
    p = wcns.default_params()
    for kind in ("gravity", "reflect"):
        g = wcns.make_grid(2, (16, 16), (0, 0), (1, 1), (0, 0))
        if kind == "gravity":
            g.gravity[1] = 1.0
        else:
            g.bc[0][0] = g.bc[0][1] = wcns.BC_REFLECTING
        assert fn(C.byref(g), 1.4, C.byref(p), C.c_void_p(16), 0.0, None, None) == wcns.ERR_INVALID


def test_noalloc_step_rejects_oversized_grids_without_a_gpu():
    """The node count is checked axis by axis against the static buffer, so a
    grid whose byte count would wrap around 2^64 is rejected, as is one node
    more than fits (349,514 nodes in 1D, 262,136 in 2D, 209,708 in 3D)."""
    L = wcns.lib()
    fn = L.wcns_step_rk3_noalloc
    fn.argtypes = [C.POINTER(wcns.Grid), C.c_double, C.POINTER(wcns.SchemeParams), C.c_void_p, C.c_double,
                   C.POINTER(C.c_double), C.c_void_p]
    p = wcns.default_params()
    cases = [(2, (2 ** 30, 2 ** 29)), (3, (2 ** 21, 2 ** 21, 2 ** 21)), (3, (65536, 65536, 65536)),
             (1, (349515,)), (2, (262137, 1)), (3, (209709, 1, 1))]
    for nd, n in cases:
        g = wcns.make_grid(nd, n + (1,) * (3 - nd), (0, 0, 0), (1, 1, 1), (0, 0, 0))
        assert fn(C.byref(g), 1.4, C.byref(p), C.c_void_p(16), 0.0, None, None) == wcns.ERR_INVALID, n
        assert b"scratch" in wcns.lib().wcns_last_error()
