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


# double plans: pointwise 1e-11 (the far targets are grouped into warps in
# atomic-append order, which moves the row-sum anchors and the warp's
# double/float split of the exponentially small series tail, so sums agree to
# rounding, not bitwise); split plans:
# the normwise 2e-5 bound the split-precision parity test states, since float
# sums depend on that grouping
@pytest.mark.parametrize("precision,metric,tol", [(gf.GF_FP64, rel_err, 1e-11), (gf.GF_FP32_SPLIT, norm_err, 2e-5)])
def test_noalloc_matches_eval_points_twice(precision, metric, tol):
    plan = gf.Plan(3, 2.5, (0.1, 0.3), (32, 32, 16), precision=precision)
    for call, (n, seed) in enumerate([(20000, 1), (7001, 2)]):
        x = torch.from_numpy(W.targets_3d(n, seed=seed)).cuda()
        ref = plan.eval_points(x, gf.GF_OUT_GD)
        out = torch.full_like(ref, complex("nan"))
        plan.eval_points_noalloc_into(x, out, gf.GF_OUT_GD)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all(), f"call {call}: unwritten outputs"
        assert metric(o, r) < tol, f"call {call}"
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
