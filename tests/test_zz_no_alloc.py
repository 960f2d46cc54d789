"""gf_eval_points_noalloc: the allocation-free evaluation entry point.

Callers that must not allocate device memory while they evaluate (a solver
that reserved all free memory for its own pool, a latency-critical loop where
a synchronising cudaMalloc/cudaFree is not acceptable) use this variant, which
keeps its scratch in a fixed array compiled into the library.  Its results
must equal those of gf_eval_points on the same plan and targets; this is
checked on two calls in a row (the second call reuses the array the first one
left behind).  Kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1801_05977_gb300 import gf
from paper_1801_05977_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_err(got, ref, floor=1e-6):
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max())
    return float((np.abs(got - ref) / scale).max())


def norm_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def entry_norm_err(got, ref):
    return float((np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max())


# double plans: pointwise 1e-11 (the far targets are grouped into warps in
# atomic-append order, which moves the row-sum anchors and the warp's
# double/float split of the exponentially small series tail, so sums agree to
# rounding, not bitwise); the Maxwell entries weight that tail by b^2 and
# c^p c^q, and some of them pass near zero, so they are compared normwise per
# entry (1e-13; a pointwise floor of 1e-6 max|G| would magnify a 1e-16
# difference at such a point 1e6-fold); split plans: the normwise 2e-5 bound
# the split-precision parity test states, since float sums depend on that
# grouping
CASES = [
    # id, plan arguments, output kind, metric, tolerance
    ("3d-fp64", dict(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16), precision=gf.GF_FP64), gf.GF_OUT_GD,
     rel_err, 1e-11),
    ("3d-split", dict(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16), precision=gf.GF_FP32_SPLIT), gf.GF_OUT_GD,
     norm_err, 2e-5),
    ("2d-fp64", dict(dim=2, k=1.3, alpha=(0.2,), M=(64, 64), precision=gf.GF_FP64), gf.GF_OUT_G, rel_err, 1e-11),
    ("maxwell-fp64", dict(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16), precision=gf.GF_FP64,
                          kind=gf.GF_MAXWELL), gf.GF_OUT_MAXWELL7, entry_norm_err, 1e-13),
]


def _targets(dim, n, seed):
    return W.targets_3d(n, seed=seed) if dim == 3 else W.targets_2d(n, seed=seed)


def _compare(plan, dim, which, metric, tol, calls):
    for call, (n, seed) in enumerate(calls):
        x = torch.from_numpy(_targets(dim, n, seed)).cuda()
        ref = plan.eval_points(x, which)
        out = torch.full_like(ref, complex("nan"))
        plan.eval_points_noalloc_into(x, out, which)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all(), f"call {call}: unwritten outputs"
        assert metric(o, r) < tol, f"call {call}"


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_eval_points_twice(case):
    _, kw, which, metric, tol = case
    kw = dict(kw)
    dim, k, alpha, M = kw.pop("dim"), kw.pop("k"), kw.pop("alpha"), kw.pop("M")
    plan = gf.Plan(dim, k, alpha, M, **kw)
    _compare(plan, dim, which, metric, tol, [(20000, 1), (7001, 2)])
    plan.close()


def test_noalloc_at_the_size_limit():
    """Exactly GF_NOALLOC_MAX_TARGETS targets (the far lists fill the array to
    its end), then a smaller call that reuses what the first one left behind."""
    plan = gf.Plan(3, 2.5, (0.1, 0.3), (32, 32, 16))
    _compare(plan, 3, gf.GF_OUT_GD, rel_err, 1e-11, [(gf.NOALLOC_MAX_TARGETS, 3), (1001, 4)])
    plan.close()


def test_noalloc_rejects_oversize_and_bad_kind():
    plan = gf.Plan(3, 2.5, (0.1, 0.3), (16, 16, 16))
    L = gf.lib()
    n = gf.NOALLOC_MAX_TARGETS + 1
    st = L.gf_eval_points_noalloc(plan._h, ctypes.c_void_p(1), n, gf.GF_OUT_GD, ctypes.c_void_p(1), None)
    assert st == gf.GF_ERR_ARG
    assert "exceeds" in L.gf_last_error().decode()
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((4, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(gf.GfError):
        plan.eval_points_noalloc_into(x, out, gf.GF_OUT_G)
    plan.close()
