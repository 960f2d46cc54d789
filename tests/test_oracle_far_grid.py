"""Pins of the oracle's far-region grid (the far branch |x3| > c on a grid of
planes instead of the eigen-series (he), as the near branch does with the
remainder).

- node values against the definition: the planes' naive inverse DFT against
  numpy's FFT of the same coefficients, and against the eigen-series (he) at
  the nodes (the coefficients decay like e^{-|n| z}, so at z >= c = 0.6 and
  128 in-plane points the aliasing is below 1e-16);
- interpolation: the error against the series falls like h^4 as the in-plane
  spacing halves (tensor cubics), and the z spacing does not limit it;
- Maxwell (Sec. 4): the seven fields against the series' second derivatives,
  with the sign change of the xz and yz entries across x3 = 0.
"""
import numpy as np
import pytest

from oracle import oracle as O

K3, AL3 = 2.5, (0.1, 0.3)
ZMAX = 1.0


def beta_of(k, a2):
    return np.where(a2 <= k * k, np.sqrt(np.abs(k * k - a2)) + 0j, 1j * np.sqrt(np.abs(a2 - k * k)))


def norm_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def far_targets(n, seed, zmax=ZMAX, c=0.6):
    rng = np.random.default_rng(seed)
    z = rng.uniform(c * (1 + 1e-9), zmax, n) * rng.choice([-1.0, 1.0], n)
    return np.column_stack([rng.uniform(-9, 9, n), rng.uniform(-9, 9, n), z])


def test_far_grid_planes_match_numpy_fft():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(16, 16, 16))
    Mf, Nz = 32, 4
    fg = O.far_grid(pb, Mf, Nz, ZMAX)
    assert fg.shape == (1, Nz + 3, Mf, Mf)
    hz = (ZMAX - pb.c) / Nz
    j = np.fft.fftfreq(Mf, 1.0 / Mf)
    c1, c2 = AL3[0] + j[None, :], AL3[1] + j[:, None]          # [n2][n1]
    beta = beta_of(K3, c1 * c1 + c2 * c2)
    for m in range(Nz + 3):
        a = 1j / (8 * np.pi**2) * np.exp(1j * beta * (pb.c + (m - 1) * hz)) / beta
        ref = np.fft.ifft2(a) * Mf * Mf                            # sum_n a_n e^{2 pi i n.l/Mf}
        assert norm_err(fg[0, m], ref) < 1e-14


def test_far_grid_nodes_are_the_series():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(16, 16, 16))
    Mf, Nz = 128, 4
    fg = O.far_grid(pb, Mf, Nz, ZMAX)
    hz = (ZMAX - pb.c) / Nz
    rng = np.random.default_rng(1)
    l = rng.integers(0, Mf, (40, 2))
    m = rng.integers(1, Nz + 2, 40)
    t = l * (2 * np.pi / Mf)
    t = np.where(t >= np.pi, t - 2 * np.pi, t)                  # node l at x = l h (mod 2 pi)
    x = np.column_stack([t[:, 0], t[:, 1], pb.c + (m - 1) * hz])
    ref = O.series(pb, x, O.OUT_GD)[:, 0] * np.exp(-1j * (AL3[0] * x[:, 0] + AL3[1] * x[:, 1]))
    got = fg[0, m, l[:, 1], l[:, 0]]
    assert norm_err(got, ref) < 1e-13


def test_far_grid_interpolation_order_h4():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(16, 16, 16))
    x = far_targets(400, seed=2)
    ref = O.series(pb, x, O.OUT_GD)
    errs = []
    for Mf in (64, 128, 256):
        fg = O.far_grid(pb, Mf, 16, ZMAX)
        errs.append(norm_err(O.far_grid_evaluate(pb, fg, 16, ZMAX, x, O.OUT_GD), ref))
    # cubic interpolation: h^4, i.e. 16x per halving (measured 12x .. 17x on this cloud)
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8, errs
    assert errs[2] < 2e-6, errs
    # the z spacing is not the limit: 8 or 32 intervals give the same error at Mf = 128
    e8 = norm_err(O.far_grid_evaluate(pb, O.far_grid(pb, 128, 8, ZMAX), 8, ZMAX, x, O.OUT_GD), ref)
    e32 = norm_err(O.far_grid_evaluate(pb, O.far_grid(pb, 128, 32, ZMAX), 32, ZMAX, x, O.OUT_GD), ref)
    assert e8 < 1.5 * errs[1] and e32 < 1.5 * errs[1], (e8, e32, errs[1])


def test_far_grid_edges_and_quasi_periodicity():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(16, 16, 16))
    Nz = 8
    fg = O.far_grid(pb, 128, Nz, ZMAX)
    # z at the slab's ends (c just above, zmax exactly: the clamped last interval)
    x = np.array([[0.3, -1.2, pb.c * (1 + 1e-12)], [2.0, 0.5, ZMAX], [-3.1, 3.1, -ZMAX], [1.0, 1.0, 0.8]])
    ref = O.series(pb, x, O.OUT_GD)
    assert norm_err(O.far_grid_evaluate(pb, fg, Nz, ZMAX, x, O.OUT_GD), ref) < 1e-4
    # G(x + 2 pi e_i) = e^{i 2 pi alpha_i} G(x)
    g0 = O.far_grid_evaluate(pb, fg, Nz, ZMAX, x, O.OUT_GD)[:, 0]
    for i in range(2):
        xs = x.copy()
        xs[:, i] += 2 * np.pi
        g1 = O.far_grid_evaluate(pb, fg, Nz, ZMAX, xs, O.OUT_GD)[:, 0]
        assert np.abs(g1 - np.exp(2j * np.pi * AL3[i]) * g0).max() < 1e-13 * np.abs(g0).max()


def test_far_grid_maxwell_fields_and_sign():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(16, 16, 16), maxwell=True)
    Nz = 8
    fg = O.far_grid(pb, 128, Nz, ZMAX)
    assert fg.shape[0] == 7
    x = far_targets(300, seed=3)
    ref = O.series(pb, x, O.OUT_MAXWELL7)
    got = O.far_grid_evaluate(pb, fg, Nz, ZMAX, x, O.OUT_MAXWELL7)
    # interpolation error of second derivatives (terms weighted by b^2, c^p c^q):
    # measured 5.4e-5 at 128 points; a wrong factor or sign would be O(1)
    for e in range(7):
        assert norm_err(got[:, e], ref[:, e]) < 2e-4, e
    # the xz and yz entries are odd in x3, the others even
    xm = x.copy()
    xm[:, 2] = -xm[:, 2]
    gm = O.far_grid_evaluate(pb, fg, Nz, ZMAX, xm, O.OUT_MAXWELL7)
    sign = np.array([1, 1, 1, 1, -1, -1, 1])
    assert np.abs(gm - sign * got).max() == 0.0
