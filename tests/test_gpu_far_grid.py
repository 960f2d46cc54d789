"""The far-region grid on the GPU against the oracle's mirror of it.

Plans with far_grid_M > 0 evaluate far targets with c < |x3| <= far_grid_zmax
from planes of F = e^{-i alpha.t} G_d synthesised by inverse FFT and read by
tensor cubics; the oracle builds the same planes by a naive DFT
(oracle/gf_oracle.c or_far_grid) and interpolates them the same way, so a
double-precision plan must match it to 1e-10 pointwise like the near branch.
Targets beyond far_grid_zmax keep the eigen-series, near targets the
remainder grid.  The split precision is checked at its stated bound, and at
the workload size against the plan without the far grid (the series).
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
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    return float((np.abs(got - ref) / scale).max())


def norm_err(got, ref):
    return float((np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max())


def oracle_with_far_grid(pb, Mf, Nz, zmax, x, which):
    """Near targets by Algorithm 2/3, c < |x3| <= zmax by the far grid, beyond by the series."""
    z = np.abs(x[:, 2])
    near, fg = z <= pb.c, (z > pb.c) & (z <= zmax)
    out = np.empty((x.shape[0], O.N_ENTRIES[which]), dtype=np.complex128)
    out[near] = O.evaluate(pb, O.grid(pb), x[near], which)
    out[fg] = O.far_grid_evaluate(pb, O.far_grid(pb, Mf, Nz, zmax), Nz, zmax, x[fg], which)
    rest = ~(near | fg)
    if rest.any():
        out[rest] = O.series(pb, x[rest], which)
    return out


def targets(n, seed):
    # the workload cloud (|x3| <= 1) plus a few beyond zmax = 0.9 and at its edge
    x = W.targets_3d(n, seed=seed)
    extra = np.array([[0.3, 0.2, 0.9], [-1.0, 2.0, -0.9], [0.5, 0.5, 1.3], [4.0, -2.0, -2.5],
                      [0.0, 0.0, np.nextafter(0.6, 1.0)], [7.0, 7.0, -0.61]])
    return np.concatenate([x, extra])


@pytest.mark.parametrize("maxwell", [False, True], ids=["helmholtz", "maxwell"])
def test_far_grid_fp64_matches_oracle(maxwell):
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(32, 32, 16), maxwell=maxwell)
    Mf, Nz, zmax = 64, 8, 0.9
    plan = gf.Plan(3, pb.k, pb.alpha, pb.M, series_tol=pb.tau, kind=gf.GF_MAXWELL if maxwell else gf.GF_HELMHOLTZ,
                   far_grid_M=Mf, far_grid_nz=Nz, far_grid_zmax=zmax)
    info = plan.info
    assert (info.far_grid_M, info.far_grid_nz, info.far_grid_zmax) == (Mf, Nz, zmax)
    x = targets(3000, seed=71)
    which, owhich = (gf.GF_OUT_MAXWELL7, O.OUT_MAXWELL7) if maxwell else (gf.GF_OUT_GD, O.OUT_GD)
    ref = oracle_with_far_grid(pb, Mf, Nz, zmax, x, owhich)
    got = plan.eval_points(torch.from_numpy(x).cuda(), which).cpu().numpy()
    e = rel_err(got, ref)
    print(f"far grid FP64 ({'Maxwell' if maxwell else 'Helmholtz'}): pointwise {e:.2e} vs the oracle's far grid")
    assert e < TOL64
    # the allocation-free entry point classifies in place and gathers there
    out = torch.empty_like(torch.from_numpy(got)).cuda()
    plan.eval_points_noalloc_into(torch.from_numpy(x).cuda(), out, which)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref) < TOL64
    plan.close()


def test_far_grid_split_matches_oracle():
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(64, 64, 32))
    Mf, Nz, zmax = 128, 16, 1.0
    plan = gf.Plan(3, pb.k, pb.alpha, pb.M, precision=gf.GF_FP32_SPLIT, far_grid_M=Mf, far_grid_nz=Nz)
    x = targets(4000, seed=72)
    ref = oracle_with_far_grid(pb, Mf, Nz, zmax, x, O.OUT_GD)
    got = plan.eval_points(torch.from_numpy(x).cuda(), gf.GF_OUT_GD).cpu().numpy()
    e = norm_err(got, ref)
    print(f"far grid split: normwise {e:.2e} vs the oracle's far grid")
    assert e < 1e-6
    plan.close()


def test_far_grid_split_workload_accuracy():
    """Config-2 parameters and 1e6 targets: the split plan with a 512 x 512 far
    grid against the double-precision plan (series): the far grid's h^4 error
    (about 5e-8 of max|G| at 512 points) stays inside the split bound."""
    x = torch.from_numpy(W.targets_3d(1_000_000, seed=0)).cuda()
    ref = gf.Plan(3, 2.5, (0.1, 0.3), (128, 128, 64)).eval_points(x, gf.GF_OUT_GD)
    plan = gf.Plan(3, 2.5, (0.1, 0.3), (128, 128, 64), precision=gf.GF_FP32_SPLIT, far_grid_M=512)
    got = plan.eval_points(x, gf.GF_OUT_GD)
    torch.cuda.synchronize()
    far = (x[:, 2].abs() > 0.6).cpu().numpy()
    g, r = got.cpu().numpy().astype(np.complex128), ref.cpu().numpy()
    e_all, e_far = norm_err(g, r), float(np.abs(g[far] - r[far]).max() / np.abs(r).max())
    print(f"split + 512^2 far grid vs the FP64 series path: normwise {e_all:.2e} (far targets {e_far:.2e})")
    assert e_all < 2e-7
    plan.close()
