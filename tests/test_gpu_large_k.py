"""Large wave numbers and large grids (the paper's Tables 3-4, 8.5-8.6 and
10.5-10.6) on the GPU.

- Against the paper's accuracy: at the grids of the paper's large-k examples
  (up to 2048 x 2048 in 2D and 1024^3 in 3D) the GPU path is compared with the
  eigen-series (ei)/(he) at the paper's points off the periodic plane.  The
  paper's eps, cut-offs and FFT-computed coefficient integrals are not all
  stated, so its digits cannot be reproduced: its printed relative error sets
  the scale (ours within 20x of it; a wrong term or sign would be O(1)), and
  the error must fall as the grid is refined, as the paper's does.  The
  Maxwell error is the largest over the tensor entries (the paper's r-error).
- Against the oracle: k = 50 on grids the oracle synthesises in seconds,
  element by element.  Near the resonance sphere the coefficients carry
  1/(|xi_j|^2 - k^2), which the resonance rule keeps above 1e-6 k^2 only, so
  rounding-order differences between the two programs grow up to 1e6-fold
  there: the bar is 1e-12 normwise per entry (measured 2.6e-14) and 1e-10
  pointwise where |G| is above 1e-2 of its maximum (measured 2.2e-12).
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
        plan = gf.Plan(3, k, (a1, a2), (M, M, M), kind=gf.GF_MAXWELL if maxwell else gf.GF_HELMHOLTZ)
    exact = O.series(pb, pts, owhich)
    got = plan.eval_points(torch.from_numpy(pts).cuda(), which).cpu().numpy().astype(np.complex128)
    plan.close()
    err = (np.abs(got - exact) / np.abs(exact)).max(axis=1)  # max over tensor entries
    print(f"{kind} k={k} N={N}: rel. error {err[0]:.2e}, {err[1]:.2e} (paper {e1:.2e}, {e2:.2e})")
    MEASURED[(kind, k, N)] = err
    assert err[0] <= 20 * e1 and err[1] <= 20 * e2, (err, (e1, e2))


MEASURED = {}


def test_large_k_errors_fall_with_the_grid():
    """Within each of the paper's tables, the error at the first point falls as
    N doubles (second-order and better convergence, Thms 2.2 and 3.2)."""
    if not MEASURED:
        pytest.skip("needs the table rows above in the same session")
    for kind, k in {(kd, kk) for kd, kk, _ in MEASURED}:
        ns = sorted(n for kd, kk, n in MEASURED if (kd, kk) == (kind, k))
        e = [MEASURED[(kind, k, n)][0] for n in ns]
        assert all(b < a for a, b in zip(e, e[1:])), (kind, k, ns, e)


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
    plan = gf.Plan(pb.dim, k, pb.alpha, pb.M, series_tol=pb.tau, quad_nodes=pb.Q,
                   kind=gf.GF_MAXWELL if pb.maxwell else gf.GF_HELMHOLTZ)
    pb.ct = plan.info.c_tilde  # (a resonance perturbation would show here)
    ref = O.evaluate(pb, O.grid(pb), x, owhich)
    got = plan.eval_points(torch.from_numpy(x).cuda(), which).cpu().numpy()
    plan.close()
    e_nw = float((np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max())
    e_pt = rel_err(got, ref, floor=1e-2)
    print(f"k = 50 {kind}: normwise {e_nw:.2e}, pointwise (floor 1e-2 max|G|) {e_pt:.2e} vs the oracle")
    assert e_nw < 1e-12 and e_pt < 1e-10
