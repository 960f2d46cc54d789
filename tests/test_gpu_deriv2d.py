"""2D derivatives (Sec. 2.4) on the GPU against the oracle.

A GF_DERIV2D plan synthesises, beside L, the remainder fields K_1 - h_1, K_2 - h_2
(Sec. 2.4.1) and with k2 > 0 the fields T_pq - h_pq of the differences of second
derivatives for wave numbers k and k2 (Sec. 2.4.2); the evaluation interpolates
them, adds the singular parts back and lifts by e^{i alpha x1}, the far branch sums
the differentiated series.  The oracle (oracle/gf_oracle.c, pinned in
tests/test_oracle_deriv2d.py) does the same steps plainly; double-precision plans
must match it to 1e-10 pointwise, grids included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1801_05977_gb300 import gf

pytestmark = pytest.mark.gpu

K, K2, AL, CT = 1.3, 2.1, 0.2, 1.4
TOL64 = 1e-10


def rel_err(got, ref, floor=1e-6):
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    return float((np.abs(got - ref) / scale).max())


def norm_err(got, ref):
    return float((np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max())


def make(M, k2=K2, precision=gf.GF_FP64):
    plan = gf.Plan(2, K, (AL,), (M, M), kind=gf.GF_DERIV2D, k2=k2, c_tilde=CT, precision=precision)
    i = plan.info
    pb = O.Problem(dim=2, k=K, alpha=(AL,), M=(M, M), c=i.c, ct=i.c_tilde, eps=i.eps, Q=i.quad_nodes)
    return plan, pb


def targets(n, seed):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(-12, 12, n), rng.uniform(-1.5, 1.5, n)])
    # the cell seams, the branch boundary and one ulp beyond, the singular zone's edge,
    # next to the singularity, far copies
    extra = [[np.pi, 0.3], [-np.pi, -0.2], [0.4, 0.6], [0.4, np.nextafter(0.6, 1.0)], [-1.0, -0.6],
             [0.9, 0.0], [0.0, 0.9 - 1e-12], [1e-3, 2e-3], [-2e-3, -1e-3], [2 * np.pi * 1000 + 0.1, 0.05],
             [-777 * 2 * np.pi, 0.3], [0.25, 5.0]]
    return np.concatenate([x, extra])


def oracle_values(pb, x, k2):
    g = O.grid_deriv2(pb, k2)
    G = O.evaluate(pb, O.grid(pb), x, O.OUT_G)
    grad = np.concatenate([G, O.evaluate_deriv2(pb, k2, g, x, O.DERIV_GRAD)], axis=1)
    hess = O.evaluate_deriv2(pb, k2, g, x, O.DERIV_HYPER) if k2 > 0 else None
    return g, grad, hess


@pytest.mark.parametrize("M", [32, 64])
def test_deriv2d_fp64_matches_oracle(M):
    plan, pb = make(M)
    x = targets(4000, seed=81 + M)
    g, grad, hess = oracle_values(pb, x, K2)
    xd = torch.from_numpy(x).cuda()
    got = plan.eval_points(xd, gf.GF_OUT_GRAD).cpu().numpy()
    e = [rel_err(got[:, j], grad[:, j]) for j in range(3)]
    print(f"M={M} grad vs oracle pointwise: G {e[0]:.2e}, dG/dx1 {e[1]:.2e}, dG/dx2 {e[2]:.2e}")
    assert max(e) < TOL64
    got = plan.eval_points(xd, gf.GF_OUT_HESSDIFF).cpu().numpy()
    e = [rel_err(got[:, j], hess[:, j]) for j in range(3)]
    print(f"M={M} T vs oracle pointwise: T11 {e[0]:.2e}, T12 {e[1]:.2e}, T22 {e[2]:.2e}")
    assert max(e) < TOL64
    # the grids: L, then the five derivative fields, node by node
    grid = plan.eval_grid().cpu().numpy()
    assert grid.shape == (6, M, M)
    ref = np.concatenate([O.grid(pb), g])
    for f in range(6):
        assert norm_err(grid[f].ravel(), ref[f].ravel()) < 1e-12, f
    plan.close()


def test_gradient_only_plan_and_plain_g():
    """k2 = 0 stores three fields and refuses the second-derivative output; its G is
    the plain plan's G (the same coefficients for field 0)."""
    plan, pb = make(64, k2=0.0)
    assert plan.info.nfields == 3
    x = torch.from_numpy(targets(3000, seed=90)).cuda()
    got = plan.eval_points(x, gf.GF_OUT_GRAD).cpu().numpy()
    plain = gf.Plan(2, K, (AL,), (64, 64), c_tilde=CT)
    g0 = plain.eval_points(x, gf.GF_OUT_G).cpu().numpy()[:, 0]
    assert np.abs(got[:, 0] - g0).max() <= 1e-14 * np.abs(g0).max()
    assert np.abs(plan.eval_points(x, gf.GF_OUT_G).cpu().numpy()[:, 0] - g0).max() <= 1e-14 * np.abs(g0).max()
    with pytest.raises(gf.GfError):
        plan.eval_points(x, gf.GF_OUT_HESSDIFF)
    _, grad, _ = oracle_values(pb, x.cpu().numpy(), 0.0)
    assert max(rel_err(got[:, j], grad[:, j]) for j in range(3)) < TOL64
    # the allocation-free entry point serves the same outputs
    out = torch.empty_like(torch.from_numpy(got)).cuda()
    plan.eval_points_noalloc_into(x, out, gf.GF_OUT_GRAD)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), got)
    plain.close()
    plan.close()


def test_deriv2d_against_the_exact_series():
    """Method accuracy at 256^2 (c~ = 1.4): against the derivatives of (ei) summed term
    by term, next to the singularity included (measured 4.5e-5 for the gradient, 1.3e-4
    for the differences, normwise; the oracle pins the convergence at 64^2 and 128^2);
    the values at |x2| > c are that series itself."""
    plan, pb = make(256)
    rng = np.random.default_rng(92)
    x = np.column_stack([rng.uniform(-np.pi, np.pi, 400), rng.uniform(-0.6, 0.6, 400)])
    x = x[np.abs(x[:, 1]) > 0.02]
    x = np.concatenate([x, [[0.05, 0.03], [-0.02, -0.04], [0.3, 0.02]]])
    xd = torch.from_numpy(x).cuda()
    grad = plan.eval_points(xd, gf.GF_OUT_GRAD).cpu().numpy()[:, 1:]
    hess = plan.eval_points(xd, gf.GF_OUT_HESSDIFF).cpu().numpy()
    eg = norm_err(grad, O.series_deriv2(pb, 0.0, x, O.DERIV_GRAD))
    eh = norm_err(hess, O.series_deriv2(pb, K2, x, O.DERIV_HYPER))
    print(f"256^2 vs the exact series: gradient {eg:.2e}, second-derivative differences {eh:.2e}")
    assert eg < 1e-4 and eh < 5e-4
    xf = np.column_stack([rng.uniform(-9, 9, 200), rng.choice([-1, 1], 200) * rng.uniform(0.61, 4.0, 200)])
    xfd = torch.from_numpy(xf).cuda()
    assert rel_err(plan.eval_points(xfd, gf.GF_OUT_GRAD).cpu().numpy()[:, 1:], O.series_deriv2(pb, 0.0, xf, 0)) < 1e-12
    assert rel_err(plan.eval_points(xfd, gf.GF_OUT_HESSDIFF).cpu().numpy(), O.series_deriv2(pb, K2, xf, 1)) < 1e-12
    plan.close()


def test_deriv2d_split_precision():
    plan, pb = make(64, precision=gf.GF_FP32_SPLIT)
    x = targets(3000, seed=93)
    _, grad, hess = oracle_values(pb, x, K2)
    xd = torch.from_numpy(x).cuda()
    eg = norm_err(plan.eval_points(xd, gf.GF_OUT_GRAD).cpu().numpy().astype(np.complex128), grad)
    eh = norm_err(plan.eval_points(xd, gf.GF_OUT_HESSDIFF).cpu().numpy().astype(np.complex128), hess)
    print(f"split precision vs the oracle: gradient normwise {eg:.2e}, T normwise {eh:.2e}")
    assert eg < 2e-6 and eh < 2e-6
    plan.close()
