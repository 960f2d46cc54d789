"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point declared in include/gf.h; parameter validation,
the Wood-anomaly check (Sec. 1) and the resonance handling (Secs. 2.1, 3.1)
return their status codes before any device work."""
import ctypes
import os
import re

import pytest

from paper_1801_05977_gb300 import gf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gf.h")).read()
    return sorted(set(re.findall(r"\b(gf_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = gf.lib()
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(gf.EXPORTS)


def test_trunc_defaults():
    t = gf.trunc_default()
    assert (t.c, t.c_tilde, t.eps, t.quad_nodes) == (0.6, 1.0, 0.45, 0)
    assert (t.far_grid_M, t.far_grid_nz, t.far_grid_zmax) == (0, 0, 0.0)
    assert t.precision == gf.GF_FP64 and t.kind == gf.GF_HELMHOLTZ and t.k2 == 0.0


def _plan_status(dim, k, alpha, M, **kw):
    L = gf.lib()
    t = gf.trunc_default(**kw)
    al = (ctypes.c_double * 2)(*(list(alpha) + [0.0] * (2 - len(alpha))))
    mm = (ctypes.c_int * 3)(*(list(M) + [1] * (3 - len(M))))
    h = ctypes.c_void_p()
    st = L.gf_plan(dim, k, al, mm, ctypes.byref(t), None, ctypes.byref(h))
    return st, h, L.gf_last_error().decode()


@pytest.mark.parametrize("args,kw", [
    ((4, 1.0, (0.1, 0.2), (16, 16, 16)), {}),          # dim
    ((3, -1.0, (0.1, 0.2), (16, 16, 16)), {}),         # k <= 0
    ((3, float("nan"), (0.1, 0.2), (16, 16, 16)), {}),
    ((3, 1.0, (0.1, float("inf")), (16, 16, 16)), {}),
    ((3, 1.0, (0.1, 0.2), (12, 16, 16)), {}),          # not a power of two
    ((3, 1.0, (0.1, 0.2), (16, 16, 2048)), {}),        # too large (3D)
    ((2, 1.0, (0.1,), (16, 4096)), {}),                # too large (2D)
    ((3, 1.0, (0.1, 0.2), (4, 16, 16)), {}),           # too small
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"c": 1.2}),  # c >= c~
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"eps": 0.6}),  # 2 eps >= c~
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"quad_nodes": 4}),
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"quad_nodes": 2000}),
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"precision": 7}),
    ((2, 1.0, (0.1,), (16, 16)), {"kind": gf.GF_MAXWELL}),  # Maxwell is 3D only
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"far_grid_M": 100}),  # far grid: not a power of two
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"far_grid_M": 4096}),
    ((2, 1.0, (0.1,), (16, 16)), {"far_grid_M": 64}),     # far grid is 3D only
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"far_grid_M": 64, "far_grid_zmax": 0.5}),  # zmax <= c
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"far_grid_M": 64, "far_grid_nz": -1}),
    ((3, 1.0, (0.1, 0.2), (16, 16, 16)), {"kind": gf.GF_DERIV2D}),  # derivative fields are 2D only
    ((2, 1.0, (0.1,), (16, 16)), {"kind": 3}),                      # no such kind
    ((2, 1.0, (0.1,), (16, 16)), {"kind": gf.GF_DERIV2D, "k2": 1.0}),  # k2 = k: no difference
    ((2, 1.0, (0.1,), (16, 16)), {"kind": gf.GF_DERIV2D, "k2": -2.0}),
    ((2, 1.0, (0.1,), (16, 16)), {"kind": gf.GF_DERIV2D, "k2": float("inf")}),
    ((2, 1.0, (0.1,), (16, 16)), {"k2": 2.0}),                      # k2 without derivative fields
])
def test_plan_rejects_bad_arguments(args, kw):
    st, h, msg = _plan_status(*args, **kw)
    assert st == gf.GF_ERR_ARG and not h.value and msg


def test_plan_detects_wood_anomaly():
    # |alpha + n| = k exactly for n = (1, 0): beta vanishes
    st, h, msg = _plan_status(3, 1.1, (0.1, 0.0), (16, 16, 16))
    assert st == gf.GF_ERR_WOOD and "Wood" in msg
    st, h, msg = _plan_status(2, 1.3, (0.3,), (16, 16))
    assert st == gf.GF_ERR_WOOD
    # the second wave number of a derivative plan is checked too
    st, h, msg = _plan_status(2, 2.1, (0.3,), (16, 16), kind=gf.GF_DERIV2D, k2=1.3)
    assert st == gf.GF_ERR_WOOD and "Wood" in msg


def test_plan_resonance_policy_fail():
    # beta_{0,0} = sqrt(k^2 - |alpha|^2) = pi / c~ exactly: k^2 = pi^2 + |alpha|^2
    import math
    a = (0.1, 0.2)
    k = math.sqrt(math.pi**2 + a[0] ** 2 + a[1] ** 2)
    st, h, msg = _plan_status(3, k, a, (16, 16, 16), resonance_policy=gf.GF_FAIL)
    assert st == gf.GF_ERR_RESONANCE and "beta" in msg


def test_null_handles_are_rejected():
    L = gf.lib()
    assert L.gf_eval_points(None, None, 10, 1, None, None) == gf.GF_ERR_ARG
    assert L.gf_eval_grid(None, None, 0, None) == gf.GF_ERR_ARG
    assert L.gf_destroy(None) == gf.GF_OK
    assert L.gf_grid_bytes(None) == 0
    assert L.gf_status_string(gf.GF_ERR_WOOD).decode().startswith("Wood")


def test_batch_rejects_bad_arguments():
    L = gf.lib()
    t = gf.trunc_default()
    h = ctypes.c_void_p()
    k = (ctypes.c_double * 2)(2.5, 1.1)
    al = (ctypes.c_double * 4)(0.1, 0.3, 0.1, 0.0)
    M = (ctypes.c_int * 6)(16, 16, 16, 16, 16, 16)
    assert L.gf_plan_batch(0, k, al, M, ctypes.byref(t), None, ctypes.byref(h)) == gf.GF_ERR_ARG
    assert L.gf_plan_batch(2, None, al, M, ctypes.byref(t), None, ctypes.byref(h)) == gf.GF_ERR_ARG
    # the first pair is valid only on a GPU; put the Wood pair first so no device work happens
    k2 = (ctypes.c_double * 2)(1.1, 2.5)
    al2 = (ctypes.c_double * 4)(0.1, 0.0, 0.1, 0.3)
    st = L.gf_plan_batch(2, k2, al2, M, ctypes.byref(t), None, ctypes.byref(h))
    assert st == gf.GF_ERR_WOOD and "pair 0" in L.gf_last_error().decode()
    td = gf.trunc_default(kind=gf.GF_DERIV2D)
    assert L.gf_plan_batch(2, k, al, M, ctypes.byref(td), None, ctypes.byref(h)) == gf.GF_ERR_UNSUPPORTED
    assert L.gf_batch_destroy(None) == gf.GF_OK
    assert L.gf_batch_eval_points(None, None, None, 1, None, None) == gf.GF_ERR_ARG


@pytest.mark.parametrize("pipe,iters,sink", [(-1, 10, 8), (5, 10, 8), (gf.GF_PROBE_BOTH_HALVES, 0, 8),
                                             (gf.GF_PROBE_FP64_HALF, (1 << 20) + 1, 8), (gf.GF_PROBE_FP32, 10, 0)])
def test_peak_probe_rejects_bad_arguments(pipe, iters, sink):
    """The probe checks its arguments before any device work (no GPU needed)."""
    L = gf.lib()
    buf = (ctypes.c_double * 1)()
    ptr = ctypes.cast(buf, ctypes.c_void_p) if sink else None
    fl = ctypes.c_int64()
    assert L.gf_peak_probe(pipe, iters, ptr, ctypes.byref(fl), None) == gf.GF_ERR_ARG
