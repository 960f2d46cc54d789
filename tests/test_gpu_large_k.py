"""Large wave numbers and large grids (the paper's Tables 3-4, 8.5-8.6 and
10.5-10.6) on the GPU.

- Against the paper's accuracy: at the grids of the paper's large-k examples
  (up to 2048 x 2048 in 2D and 1024^3 in 3D) the GPU path is compared with the
  eigen-series (ei)/(he) at the paper's points off the periodic plane; the
  relative error the paper prints for its own runs bounds ours (its eps,
  cut-offs and FFT-computed coefficient integrals are not all stated, so its
  digits cannot be reproduced; our coefficients come from exact quadrature).
  The Maxwell error is the largest over the tensor entries.
- Against the oracle: k = 50 on grids the oracle synthesises in seconds,
  element by element at 1e-10 (many propagating terms in the far series,
  many propagating columns in the coefficients).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1801_05977_gb300 import gf
from paper_1801_05977_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
P2 = np.array([[0.01 * np.pi, 0.01], [0.5 * np.pi, 0.01]])
P3 = np.array([[0.0, 1.5, 0.1], [0.03, 0.03, 0.1]])


def rows():
    out = []
    with open(os.path.join(HERE, "golden", "paper_tables_large_k_rerr.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, tab, k, a1, a2, n, e1, e2 = line.split()
                out.append((kind, tab, float(k), float(a1), float(a2), int(n), float(e1), float(e2)))
    return out


def rel_err(got, ref, floor=1e-6):
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    return float((np.abs(got - ref) / scale).max())


@pytest.mark.parametrize("row", rows(), ids=lambda r: f"{r[0]}-table{r[1]}-N{r[5]}")
def test_large_k_within_paper_tables(row):
    kind, _, k, a1, a2, N, e1, e2 = row
    M = 2 * N
    if kind == "2d":
        pb = O.Problem(dim=2, k=k, alpha=(a1,), M=(M, M))
        pts, which, owhich = P2, gf.GF_OUT_G, O.OUT_G
        plan = gf.Plan(2, k, (a1,), (M, M))
    else:
        maxwell = kind == "maxwell"
        pb = O.Problem(dim=3, k=k, alpha=(a1, a2), M=(M, M, M), maxwell=maxwell)
        pts = P3
        which, owhich = (gf.GF_OUT_MAXWELL6, O.OUT_MAXWELL6) if maxwell else (gf.GF_OUT_GD, O.OUT_GD)
        # double-precision Maxwell synthesis at 1024 points per axis needs more shared
        # memory than a CTA has: that grid runs in the split precision (float grid,
        # about 1e-7 relative, far below the errors compared here)
        prec = gf.GF_FP32_SPLIT if (maxwell and M > 512) else gf.GF_FP64
        plan = gf.Plan(3, k, (a1, a2), (M, M, M), precision=prec,
                       kind=gf.GF_MAXWELL if maxwell else gf.GF_HELMHOLTZ)
    exact = O.series(pb, pts, owhich)
    got = plan.eval_points(torch.from_numpy(pts).cuda(), which).cpu().numpy().astype(np.complex128)
    plan.close()
    err = (np.abs(got - exact) / np.abs(exact)).max(axis=1)  # max over tensor entries
    print(f"{kind} k={k} N={N}: rel. error {err[0]:.2e}, {err[1]:.2e} (paper {e1:.2e}, {e2:.2e})")
    assert err[0] <= e1 and err[1] <= e2, (err, (e1, e2))


@pytest.mark.parametrize("kind", ["2d", "3d", "maxwell"])
def test_large_k_matches_oracle(kind):
    k = 50.0
    if kind == "2d":
        pb = O.Problem(dim=2, k=k, alpha=(2 ** 0.5,), M=(128, 128))
        x = W.targets_2d(2000, seed=81)
        which, owhich = gf.GF_OUT_G, O.OUT_G
    else:
        pb = O.Problem(dim=3, k=k, alpha=(3 ** 0.5, 0.5), M=(64, 64, 32), maxwell=(kind == "maxwell"))
        x = np.concatenate([W.targets_3d(1500, seed=82), W.targets_3d_clustered(300, seed=83, frac=1.0)])
        which, owhich = (gf.GF_OUT_MAXWELL7, O.OUT_MAXWELL7) if pb.maxwell else (gf.GF_OUT_GD, O.OUT_GD)
    plan = gf.Plan(pb.dim, k, pb.alpha, pb.M, series_tol=pb.tau,
                   kind=gf.GF_MAXWELL if pb.maxwell else gf.GF_HELMHOLTZ)
    ref = O.evaluate(pb, O.grid(pb), x, owhich)
    got = plan.eval_points(torch.from_numpy(x).cuda(), which).cpu().numpy()
    plan.close()
    e = rel_err(got, ref)
    print(f"k = 50 {kind}: pointwise {e:.2e} vs the oracle")
    assert e < 1e-10
