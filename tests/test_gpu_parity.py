"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bar (double-precision plans): grid values within 1e-12 of max|grid| and point
values within 1e-10 relative (pointwise, with a floor of 1e-6 max|G| for
near-zeros of G), on the same seeded inputs.  Split-precision plans (float
grid, interpolation and series; double coefficients, singular part,
reduction and phase) are checked against the same oracle at their stated
error bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1801_05977_gb300 import gf
from paper_1801_05977_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def rel_err(got, ref, floor=1e-6):
    got = np.asarray(got)
    ref = np.asarray(ref)
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max())
    return float((np.abs(got - ref) / scale).max())


def norm_err(got, ref):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / np.abs(ref).max())


def gpu_plan(pb: O.Problem, precision=gf.GF_FP64, series_tol=None):
    kw = dict(c=pb.c, c_tilde=pb.ct, eps=pb.eps, quad_nodes=pb.Q, precision=precision,
              kind=gf.GF_MAXWELL if pb.maxwell else gf.GF_HELMHOLTZ)
    if series_tol is not None:
        kw["series_tol"] = series_tol
    elif precision == gf.GF_FP64:
        kw["series_tol"] = pb.tau
    return gf.Plan(pb.dim, pb.k, pb.alpha, pb.M, **kw)


def gpu_eval(plan, x, which):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.eval_points(xd, which)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def edge_targets(dim, pb):
    """Reduction seams, branch boundary, grid nodes, far copies of the cell."""
    pi = np.pi
    if dim == 3:
        h3 = 2 * pb.ct / pb.M[2]
        pts = [[-pi, -pi, 0.3], [pi, pi, -0.3], [np.nextafter(pi, 0), 0.0, 0.2], [0.0, 0.0, pb.c],
               [0.1, 0.2, -pb.c], [0.1, 0.2, np.nextafter(pb.c, 2)], [2 * pi / pb.M[0] * 3, 2 * pi / pb.M[1] * 5, h3 * 4],
               [1000.0, -777.0, 0.15], [0.0, 0.0, 1e-3], [1e-3, 0, 0], [3.0, -3.0, 5.0], [0.0, 0.0, -0.95]]
    else:
        h2 = 2 * pb.ct / pb.M[1]
        pts = [[-pi, 0.3], [pi, -0.3], [np.nextafter(pi, 0), 0.2], [0.0, pb.c], [0.1, -pb.c],
               [0.1, np.nextafter(pb.c, 2)], [2 * pi / pb.M[0] * 3, h2 * 4], [1000.0, 0.15], [1e-3, 0.0],
               [0.0, 1e-3], [3.0, 5.0], [0.0, -0.95]]
    return np.array(pts, dtype=np.float64)


# ----------------------------------------------------------------------------- 3D Helmholtz
CASES3 = [((32, 32, 16), 2.5, (0.1, 0.3)), ((16, 64, 32), 1.7, (-0.35, 0.05)), ((64, 32, 8), 4.2, (0.45, -0.2))]


@pytest.fixture(scope="module", params=CASES3, ids=lambda c: "x".join(map(str, c[0])))
def case3(request):
    M, k, al = request.param
    pb = O.Problem(dim=3, k=k, alpha=al, M=M)
    g = O.grid(pb)
    return pb, g


def test_grid_parity_3d(case3):
    pb, g = case3
    plan = gpu_plan(pb)
    got = plan.eval_grid().cpu().numpy()
    torch.cuda.synchronize()
    assert got.shape == g.shape
    assert norm_err(got, g) < 1e-12
    # the synthesis passes' staged copies (TMA) all completed within their bounded waits
    assert plan.status() == gf.GF_OK


@pytest.mark.parametrize("n", [1, 31, 33, 1017, 3000])
def test_points_parity_3d(case3, n):
    pb, g = case3
    plan = gpu_plan(pb)
    x = W.targets_3d(n, seed=n)
    ref = O.evaluate(pb, g, x, O.OUT_GD)
    got = gpu_eval(plan, x, gf.GF_OUT_GD)
    assert rel_err(got, ref) < TOL64


def test_edge_targets_3d(case3):
    pb, g = case3
    plan = gpu_plan(pb)
    x = edge_targets(3, pb)
    ref = O.evaluate(pb, g, x, O.OUT_GD)
    got = gpu_eval(plan, x, gf.GF_OUT_GD)
    assert rel_err(got, ref) < TOL64


def test_nonfinite_and_empty():
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(16, 16, 16))
    plan = gpu_plan(pb)
    x = np.array([[np.nan, 0.0, 0.1], [0.0, np.inf, 0.0], [0.1, 0.2, 0.3]])
    got = gpu_eval(plan, x, gf.GF_OUT_GD)
    assert np.isnan(got[0, 0]) and np.isnan(got[1, 0]) and np.isfinite(got[2, 0])
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    assert plan.eval_points(empty, gf.GF_OUT_GD).shape == (0, 1)
    with pytest.raises(gf.GfError):
        plan.eval_points(torch.zeros((4, 3), dtype=torch.float64, device="cuda"), gf.GF_OUT_G)


def test_host_entry_point_matches_device():
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16))
    plan = gpu_plan(pb)
    x = W.targets_3d(4097, seed=7)
    dev = gpu_eval(plan, x, gf.GF_OUT_GD)
    host = np.zeros((x.shape[0], 1), dtype=np.complex128)
    plan.eval_points_host(x, host, gf.GF_OUT_GD)
    # the host entry point runs the same evaluation: the far list is a stable sort
    # and slab partials are added in slab order, so the results agree bit for bit
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("k,al", [(2.5, (0.1, 0.3)), (1.0, (0.002, 0.0)), (4.7, (-0.45, 0.25))],
                         ids=["config2", "near-wood", "k4.7"])
def test_far_series_tiers(k, al):
    """Far targets only (|x3| from just above c to 2): the series summed in its
    double, float-float and float tiers against the oracle's plain double sums
    of the same truncated series.  (1.0, (0.002, 0)) puts |alpha_(1,0)| within
    2e-3 of k: the smallest evanescent b is 0.063, so ln b and 1/b are far from
    the other cases."""
    pb = O.Problem(dim=3, k=k, alpha=al, M=(16, 16, 8))
    plan = gpu_plan(pb)
    rng = np.random.default_rng(17)
    n = 6000
    z = rng.uniform(pb.c * (1 + 1e-9), 2.0, n) * rng.choice([-1.0, 1.0], n)
    x = np.column_stack([rng.uniform(-7, 7, n), rng.uniform(-7, 7, n), z])
    ref = O.series(pb, x, O.OUT_GD)
    got = gpu_eval(plan, x, gf.GF_OUT_GD)
    e_nw, e_pt = norm_err(got, ref), rel_err(got, ref)
    print(f"far series k={k}: normwise {e_nw:.2e}, pointwise {e_pt:.2e} vs the oracle's double sums")
    assert e_nw < 1e-13  # measured 5e-15 .. 1.4e-14
    assert e_pt < TOL64


# ----------------------------------------------------------------------------- 2D (config: k = 1.3, alpha = 0.2, 64 x 64, 10^4 targets)
def test_parity_2d_config():
    pb = O.Problem(dim=2, k=1.3, alpha=(0.2,), M=(64, 64))
    g = O.grid(pb)
    plan = gpu_plan(pb)
    got_g = plan.eval_grid().cpu().numpy()
    assert norm_err(got_g, g) < 1e-12
    x = W.targets_2d(10_000, seed=0)
    ref = O.evaluate(pb, g, x, O.OUT_G)
    got = gpu_eval(plan, x, gf.GF_OUT_G)
    assert rel_err(got, ref) < TOL64
    x = edge_targets(2, pb)
    assert rel_err(gpu_eval(plan, x, gf.GF_OUT_G), O.evaluate(pb, g, x, O.OUT_G)) < TOL64


@pytest.mark.parametrize("M,k,al", [((32, 16), 3.3, (-0.4,)), ((16, 128), 0.7, (0.05,))])
def test_parity_2d_shapes(M, k, al):
    pb = O.Problem(dim=2, k=k, alpha=al, M=M)
    g = O.grid(pb)
    plan = gpu_plan(pb)
    assert norm_err(plan.eval_grid().cpu().numpy(), g) < 1e-12
    x = W.targets_2d(2049, seed=3)
    assert rel_err(gpu_eval(plan, x, gf.GF_OUT_G), O.evaluate(pb, g, x, O.OUT_G)) < TOL64


# ----------------------------------------------------------------------------- Maxwell
def test_parity_maxwell():
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16), maxwell=True)
    g = O.grid(pb)
    plan = gpu_plan(pb)
    x = np.concatenate([W.targets_3d(1500, seed=5), W.targets_3d_clustered(500, seed=6, frac=1.0)])
    ref = O.evaluate(pb, g, x, O.OUT_MAXWELL7)
    got = gpu_eval(plan, x, gf.GF_OUT_MAXWELL7)
    assert rel_err(got, ref) < TOL64
    got6 = gpu_eval(plan, x, gf.GF_OUT_MAXWELL6)
    assert rel_err(got6, got[:, :6]) < 1e-11  # same grouping caveat as the host-entry test
    # combined grids: (delta_pq - c^p c^q/k^2) L_d vs the oracle's L_d, L^{pq}
    gg = plan.eval_grid().cpu().numpy()
    for e, (p, q) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        want = (g[0] if p == q else 0) + g[1 + e] / pb.k**2
        assert norm_err(gg[e], want) < 1e-12
    assert norm_err(gg[6], g[0]) < 1e-12


# ----------------------------------------------------------------------------- split precision
def test_split_precision_error_statement():
    """Float grid/interpolation/series with double singular part and phase:
    error vs the FP64 oracle stays below 2e-5 normwise (config-2 parameters)."""
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(64, 64, 32))
    g = O.grid(pb)
    plan = gpu_plan(pb, precision=gf.GF_FP32_SPLIT)
    gg = plan.eval_grid().cpu().numpy()
    assert norm_err(gg, g) < 2e-6
    x = W.targets_3d(3000, seed=11)
    ref = O.evaluate(pb, g, x, O.OUT_GD)
    got = gpu_eval(plan, x, gf.GF_OUT_GD)
    e = norm_err(got, ref)
    print(f"split-precision normwise error vs FP64 oracle: {e:.3e}")
    assert e < 2e-5


# ----------------------------------------------------------------------------- full size (config 2: 128 x 128 x 64)
def test_full_size_config2_sampled():
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(128, 128, 64))
    plan = gpu_plan(pb)
    x_all = W.targets_3d(1_000_000, seed=0)
    xd = torch.from_numpy(x_all).cuda()
    out = plan.eval_points(xd, gf.GF_OUT_GD)
    torch.cuda.synchronize()
    got_all = out.cpu().numpy()
    # sampled grid nodes straight from the truncated series
    C = O.coef(pb)
    rng = np.random.default_rng(0)
    nodes = np.stack([rng.integers(0, m, 6) for m in pb.M], axis=1)
    gg = plan.eval_grid().cpu().numpy()[0]
    assert plan.status() == gf.GF_OK
    ref_nodes = O.grid_nodes(pb, C, nodes)
    got_nodes = np.array([gg[n[2], n[1], n[0]] for n in nodes])
    assert np.abs(got_nodes - ref_nodes).max() < 1e-12 * np.abs(gg).max()
    # sampled targets through the oracle's whole path
    g = O.grid(pb, C)
    sel = rng.choice(x_all.shape[0], 1500, replace=False)
    ref = O.evaluate(pb, g, x_all[sel], O.OUT_GD)
    e_pt, e_nw = rel_err(got_all[sel], ref), norm_err(got_all[sel], ref)
    print(f"config-2 full size: pointwise {e_pt:.2e}, normwise {e_nw:.2e} vs the FP64 oracle")
    assert e_pt < TOL64
    assert np.isfinite(got_all).all()


def test_host_entry_right_after_plan_on_a_side_stream():
    """The host-buffer entry point uploads on the library's copy stream while the
    plan's synthesis may still be running on the caller's stream (no synchronisation
    in between, a non-default stream): the result equals the device entry's bit for
    bit."""
    x = W.targets_3d(50_001, seed=9)
    s = torch.cuda.Stream()
    xp = torch.from_numpy(x).pin_memory()
    host = torch.empty((x.shape[0], 1), dtype=torch.complex128).pin_memory()
    plan = gf.Plan(3, 2.5, (0.1, 0.3), (64, 64, 32), stream=s)
    plan.eval_points_host(xp, host, gf.GF_OUT_GD, stream=s)
    ref = gpu_eval(plan, x, gf.GF_OUT_GD)
    assert np.array_equal(host.numpy(), ref)
    plan.close()
