"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself:
library routines for special cases (Gauss-Legendre, Bessel, Hankel, FFT),
independent quadratures of the Fourier-coefficient DEFINITIONS (the paper's
closed forms (fck-coef), (kdj1), (fj), (fcf1-coef), (fcf2-coef) are derived from
those by integration by parts / Green's identity), the eigenfunction
expansions (ei)/(he) that define G and G_d (Sec. 1), and invariants
(quasi-periodicity, the trace identity of the Maxwell tensor, the free-space
singularity).  All run on the CPU in seconds.
"""
import numpy as np
import pytest
from scipy import special
from scipy.integrate import quad

from oracle import oracle as O

K3, AL3 = 2.5, (0.1, 0.3)


def cquad(f, a, b):
    kw = dict(limit=500, epsabs=1e-15, epsrel=1e-13)
    return quad(lambda t: f(t).real, a, b, **kw)[0] + 1j * quad(lambda t: f(t).imag, a, b, **kw)[0]


# --------------------------------------------------------------------------- building blocks
def test_gauss_legendre_matches_numpy_and_is_exact():
    for Q in (4, 17, 64, 96):
        x, w = O.gauss_legendre(Q)
        xr, wr = np.polynomial.legendre.leggauss(Q)
        assert np.allclose(x, xr, atol=1e-14, rtol=0)
        assert np.allclose(w, wr, atol=1e-14, rtol=0)
        for p in range(0, 2 * Q, 7):  # exact up to degree 2Q-1
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs(np.dot(w, x**p) - exact) < 1e-13


def test_smoothstep_is_c8_step():
    # S8'(s) = 17!/(8! 8!) s^8 (1-s)^8 (the derivative of the order-8 smoothstep)
    coef = special.factorial(17) / special.factorial(8) ** 2
    for s in np.linspace(0.01, 0.99, 23):
        assert abs(O.smooth8(s, 1) - coef * s**8 * (1 - s) ** 8) < 1e-11
        assert abs(O.smooth8(s) + O.smooth8(1 - s) - 1.0) < 1e-14
        assert abs(O.smooth8(s) - special.betainc(9, 9, s)) < 1e-14
        h = 1e-6
        fd2 = (O.smooth8(s + h, 1) - O.smooth8(s - h, 1)) / (2 * h)
        assert abs(fd2 - O.smooth8(s, 2)) < 1e-5 * max(1, abs(fd2))
    assert O.smooth8(0.0) == 0.0 and O.smooth8(1.0) == 1.0 and abs(O.smooth8(0.5) - 0.5) < 1e-15
    # flat to 8th order at both ends
    assert O.smooth8(1e-3) < 1e-21 and 1 - O.smooth8(1 - 1e-3) < 1e-21


def test_cutoffs_shape():
    c, ct, eps = 0.6, 1.0, 0.45
    assert O.chi(0.3, c, ct) == 1.0 and O.chi(0.6, c, ct) == 1.0 and O.chi(0.8, c, ct) == 0.0
    assert abs(O.chi(0.7, c, ct) - 0.5) < 1e-14
    assert O.yps(0.2, eps) == 1.0 and O.yps(0.9, eps) == 0.0
    # derivatives integrate to the jumps
    assert abs(quad(lambda t: O.chi(t, c, ct, 1), c, 0.8, epsabs=1e-14)[0] + 1.0) < 1e-12
    assert abs(quad(lambda r: O.yps(r, eps, 1), eps, 2 * eps, epsabs=1e-14)[0] + 1.0) < 1e-12
    assert abs(quad(lambda r: O.yps(r, eps, 2), eps, 2 * eps, epsabs=1e-14)[0]) < 1e-11


@pytest.mark.parametrize("z", [0.0, 0.3, 1.0, 5.5, 17.0, 63.0, 150.0])
def test_bessel_matches_scipy(z):
    j0, j1 = O.bessel_j01(z)
    assert abs(j0 - special.j0(z)) < 1e-14
    assert abs(j1 - special.j1(z)) < 1e-14


def test_beta_branch():
    k = 2.5
    for a2 in [0.0, 1.0, 6.0, 6.25, 6.3, 50.0, 1e4]:
        b = O.beta(k, a2)
        assert b.imag >= 0 and b.real >= 0
        assert abs(b * b - (k * k - a2)) < 1e-12 * max(1, a2)
        if a2 < k * k:
            assert b.imag == 0
        elif a2 > k * k:
            assert b.real == 0


# --------------------------------------------------------------------------- coefficient definitions
@pytest.mark.parametrize("j", [(0, 0, 0), (1, 0, 0), (-2, 1, 0), (0, 0, 5), (3, -2, 7), (20, 5, -9), (-31, 0, 3)])
def test_3d_coefficients_match_definition(j):
    """(kdj1) vs the un-integrated (kdj) (corrected exponent), and (fj) vs the
    direct radial Fourier integral of F = Phi_0 Y_eps, both by adaptive quadrature."""
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(8, 8, 8))
    a1, a2, q = AL3[0] + j[0], AL3[1] + j[1], j[2] * np.pi / pb.ct
    A2 = a1 * a1 + a2 * a2
    b = O.beta(pb.k, A2)
    s = np.sqrt(A2 + q * q)
    cm = 0.5 * (pb.c + pb.ct)
    # int_0^{c~} e^{i g t} X dt = int_0^c e^{igt} dt + int_c^{cm} e^{igt} X dt
    def E(g):
        head = pb.c if g == 0 else (np.exp(1j * g * pb.c) - 1) / (1j * g)
        return head + cquad(lambda t: np.exp(1j * g * t) * O.chi(t, pb.c, pb.ct), pb.c, cm)
    K_def = (1j / (2 * b)) * (E(b - q) + E(b + q))
    F_def = cquad(lambda r: np.exp(1j * pb.k * r) * O.yps(r, pb.eps) * (np.sin(s * r) / s if s else r), 0, 2 * pb.eps)
    K, F = O.coef_parts(pb, *j)
    assert abs(K - K_def) <= 1e-11 * max(abs(K_def), 1e-3)
    assert abs(F - F_def) <= 1e-11 * max(abs(F_def), 1e-3)


@pytest.mark.parametrize("j", [(0, 0), (1, 0), (0, 1), (-3, 2), (7, -5), (25, 11)])
def test_2d_coefficients_match_definition(j):
    """(fck-coef) vs the direct x2 integral; (fcf1-coef)/(fcf2-coef) vs the
    planar Fourier transforms of f1 = -(1/2pi) ln|x| Y and f2 = x1 f1."""
    pb = O.Problem(dim=2, k=1.3, alpha=(0.2,), M=(8, 8))
    a, q = 0.2 + j[0], j[1] * np.pi / pb.ct
    b = O.beta(pb.k, a * a)
    cm = 0.5 * (pb.c + pb.ct)
    def E(g):
        head = pb.c if g == 0 else (np.exp(1j * g * pb.c) - 1) / (1j * g)
        return head + cquad(lambda t: np.exp(1j * g * t) * O.chi(t, pb.c, pb.ct), pb.c, cm)
    K_def = (1j / (2 * b)) * (E(b - q) + E(b + q))
    eta = np.hypot(j[0], q)
    lnY = lambda r: np.log(r) * O.yps(r, pb.eps) if r > 0 else 0.0
    if eta == 0:
        F1_def = -quad(lambda r: r * lnY(r), 0, 2 * pb.eps, epsabs=1e-15, limit=400)[0]
        F2_def = 0.0
    else:
        F1_def = -quad(lambda r: lnY(r) * special.j0(eta * r) * r, 0, 2 * pb.eps, epsabs=1e-15, limit=400)[0]
        F2_def = 1j * (j[0] / eta) * quad(lambda r: lnY(r) * special.j1(eta * r) * r * r, 0, 2 * pb.eps,
                                          epsabs=1e-15, limit=400)[0]
    K, F1, F2 = O.coef_parts(pb, j[0], j[1])
    assert abs(K - K_def) <= 1e-11 * max(abs(K_def), 1e-3)
    assert abs(F1 - F1_def) <= 1e-10 * max(abs(F1_def), 1e-3)
    assert abs(F2 - F2_def) <= 1e-10 * max(abs(F2_def), 1e-3)


def test_maxwell_coefficients_are_minus_cpcq():
    pb = O.Problem(dim=3, k=K3, alpha=AL3, M=(8, 8, 4), maxwell=True)
    C = O.coef(pb)
    j1 = np.fft.fftfreq(8, 1 / 8)
    j3 = np.fft.fftfreq(4, 1 / 4)
    c1 = (AL3[0] + j1)[None, None, :]
    c2 = (AL3[1] + j1)[None, :, None]
    c3 = (j3 * np.pi)[:, None, None]
    cv = [c1, c2, c3]
    for e, (p, q) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        assert np.allclose(C[1 + e], -cv[p] * cv[q] * C[0], rtol=1e-15, atol=0)


# --------------------------------------------------------------------------- grid synthesis
@pytest.mark.parametrize("dim,M", [(2, (8, 16)), (3, (8, 4, 16)), (3, (16, 16, 8))])
def test_naive_dft_matches_numpy_fft(dim, M):
    rng = np.random.default_rng(1)
    pb = O.Problem(dim=dim, k=1.0, alpha=(0.1, 0.2)[: dim - 1], M=M)
    C = rng.standard_normal((1,) + pb.shape) + 1j * rng.standard_normal((1,) + pb.shape)
    g = O.grid(pb, C)
    V = 8 * np.pi**2 * pb.ct if dim == 3 else 4 * np.pi * pb.ct
    ref = np.fft.ifftn(C[0]) * np.prod(M) / V
    assert np.allclose(g[0], ref, atol=1e-13 * np.abs(ref).max(), rtol=0)
    nodes = np.array([[0, 0, 0], [3, 1, 2], [7, 3, 15]] if dim == 3 else [[0, 0], [5, 9], [7, 15]])
    nodes = nodes % np.array(M)
    direct = O.grid_nodes(pb, C, nodes)
    ref_n = np.array([ref[tuple(n[::-1])] for n in nodes])
    assert np.allclose(direct, ref_n, atol=1e-13 * np.abs(ref).max(), rtol=0)


def test_interpolation_reproduces_cubics_and_nodes():
    pb = O.Problem(dim=3, k=1.0, alpha=(0.0, 0.0), M=(16, 8, 16))
    M1, M2, M3 = pb.M
    h = np.array([2 * np.pi / M1, 2 * np.pi / M2, 2 * pb.ct / M3])
    # node index l stands for x = l h (mod period); fill with a tensor cubic of x
    x1 = np.arange(M1) * h[0]
    x2 = np.arange(M2) * h[1]
    x3 = np.arange(M3) * h[2]
    x1 = np.where(x1 >= np.pi, x1 - 2 * np.pi, x1)
    x2 = np.where(x2 >= np.pi, x2 - 2 * np.pi, x2)
    x3 = np.where(x3 >= pb.ct, x3 - 2 * pb.ct, x3)
    f = lambda a, b, c: (1 + 2 * a - a**3 / 3) * (0.5 - b + b**2) * (c**3 - c + 2) * (1 + 0.5j)
    g = f(x1[None, None, :], x2[None, :, None], x3[:, None, None])
    rng = np.random.default_rng(0)
    # stay two cells away from the wrap so that the stencil does not see the period seam
    y = np.stack([rng.uniform(-np.pi + 2 * h[0], np.pi - 3 * h[0], 50),
                  rng.uniform(-np.pi + 2 * h[1], np.pi - 3 * h[1], 50),
                  rng.uniform(-pb.ct + 2 * h[2], pb.ct - 3 * h[2], 50)], axis=1)
    got = O.interp(pb, g, y)
    assert np.allclose(got, f(y[:, 0], y[:, 1], y[:, 2]), rtol=1e-12, atol=1e-12)
    # exactly on a node
    y = np.array([[x1[3], x2[5], x3[2]], [x1[12], x2[1], x3[9]]])
    got = O.interp(pb, g, y)
    assert np.allclose(got, [g[2, 5, 3], g[9, 1, 12]], rtol=1e-14)


# --------------------------------------------------------------------------- whole algorithm vs the definition of G
@pytest.fixture(scope="module")
def grids3d():
    out = {}
    for M in [(32, 32, 32), (64, 64, 64)]:
        pb = O.Problem(dim=3, k=K3, alpha=AL3, M=M)
        out[M] = (pb, O.grid(pb))
    return out


PTS3 = np.array([[0.3, -1.0, 0.3], [0.1, 0.2, 0.1], [2.0, 1.0, -0.45], [0.03, 0.03, 0.1],
                 [0.0, 1.5, 0.1], [-2.9, 3.0, 0.2], [0.03, 0.03, 0.05], [0.4, -0.3, -0.25]])


def test_3d_algorithm_converges_to_eigen_series(grids3d):
    """Algorithm 2 vs the eigenfunction expansion (he), which converges at
    |x3| >= 0.05; the error must fall with the grid (Thm 3.1/3.2)."""
    exact = O.series(grids3d[(32, 32, 32)][0], PTS3, O.OUT_GD)[:, 0]
    errs = []
    for M in [(32, 32, 32), (64, 64, 64)]:
        pb, g = grids3d[M]
        v = O.evaluate(pb, g, PTS3, O.OUT_GD)[:, 0]
        errs.append(np.abs(v - exact).max() / np.abs(exact).max())
    assert errs[1] < 1e-3, errs
    assert errs[1] < errs[0] / 5, errs


def test_3d_far_branch_is_series_and_continuous(grids3d):
    pb, g = grids3d[(64, 64, 64)]
    x = np.array([[0.5, 0.7, 0.61], [1.0, -2.0, -0.9], [7.0, -8.0, 0.75]])
    assert np.array_equal(O.evaluate(pb, g, x, O.OUT_GD), O.series(pb, x, O.OUT_GD))
    xc = np.array([[0.5, 0.7, 0.6], [2.0, -1.0, -0.6]])  # on the branch boundary: grid side
    v = O.evaluate(pb, g, xc, O.OUT_GD)[:, 0]
    s = O.series(pb, xc, O.OUT_GD)[:, 0]
    assert np.all(np.abs(v - s) / np.abs(s) < 2e-3)


def test_3d_quasi_periodicity(grids3d):
    pb, g = grids3d[(32, 32, 32)]
    rng = np.random.default_rng(3)
    x = np.stack([rng.uniform(0, 2 * np.pi, 40), rng.uniform(0, 2 * np.pi, 40), rng.uniform(-1, 1, 40)], axis=1)
    v0 = O.evaluate(pb, g, x, O.OUT_GD)[:, 0]
    for m1, m2 in [(1, 0), (0, 1), (-3, 2)]:
        xs = x + np.array([2 * np.pi * m1, 2 * np.pi * m2, 0.0])
        v1 = O.evaluate(pb, g, xs, O.OUT_GD)[:, 0]
        ph = np.exp(2j * np.pi * (AL3[0] * m1 + AL3[1] * m2))
        assert np.allclose(v1, ph * v0, rtol=1e-12, atol=0)


def test_3d_free_space_singularity(grids3d):
    """G_d - e^{ikr}/(4 pi r) is regular at the origin (Sec. 3.2): along a ray
    it is linear in r for small r, and its limit agrees with the regular part
    of the eigen-series (he) extrapolated from r = 0.05, 0.1."""
    pb, g = grids3d[(64, 64, 64)]
    d = np.array([0.48, -0.6, 0.64])
    d /= np.linalg.norm(d)
    rs = np.array([1e-3, 2e-3, 4e-3])
    v = O.evaluate(pb, g, rs[:, None] * d[None, :], O.OUT_GD)[:, 0]
    reg = v - np.exp(1j * pb.k * rs) / (4 * np.pi * rs)
    s1 = (reg[1] - reg[0]) / 1e-3
    s2 = (reg[2] - reg[1]) / 2e-3
    assert abs(s1 - s2) < 0.05 * abs(s1)
    rr = np.array([0.05, 0.1])
    s = O.series(pb, rr[:, None] * d[None, :], O.OUT_GD)[:, 0] - np.exp(1j * pb.k * rr) / (4 * np.pi * rr)
    extrap = 2 * s[0] - s[1]
    assert abs(reg[0] - extrap) < 0.1 * abs(extrap)
    # relative to G_d itself at r = 1e-3 the regular part is the method's error scale
    assert abs(reg[0] - extrap) < 1e-4 * abs(v[0])


def test_maxwell_trace_and_series():
    """Series side: Sum_p G_pp = 3 G_d + k^-2 Lap G_d = 2 G_d off the lattice
    (Eq. (me)) and the entries equal finite-difference second derivatives of
    (he).  Grid side (Algorithm 3): converges to the series with the grid, and
    near the lattice point it approaches the free-space dyadic Green's function
    (I + grad grad / k^2) e^{ikr}/(4 pi r), which pins the singular F^{pq}."""
    x = np.array([[0.3, -1.0, 0.3], [2.0, 1.0, -0.45], [0.1, 0.2, 0.2], [1.0, -2.0, 0.8]])
    errs = []
    for M in [(32, 32, 32), (64, 64, 64)]:
        pb = O.Problem(dim=3, k=K3, alpha=AL3, M=M, maxwell=True)
        g = O.grid(pb)
        v = O.evaluate(pb, g, x, O.OUT_MAXWELL7)
        s = O.series(pb, x, O.OUT_MAXWELL7)
        errs.append(np.abs(v - s).max() / np.abs(s).max())
    assert errs[1] < errs[0] / 1.8 and errs[1] < 0.2, errs
    strace = s[:, 0] + s[:, 1] + s[:, 2]
    assert np.allclose(strace, 2 * s[:, 6], rtol=1e-11)
    # free-space dyadic near the origin
    d = np.array([0.48, -0.6, 0.64])
    d /= np.linalg.norm(d)
    r = 0.01
    y = (r * d)[None, :]
    vm = O.evaluate(pb, g, y, O.OUT_MAXWELL6)[0]
    k = pb.k
    A = np.exp(1j * k * r) / (4 * np.pi * r)
    # textbook dyadic: A [(1 + i/(kr) - 1/(kr)^2) I + (-1 - 3i/(kr) + 3/(kr)^2) d d^T]
    a_ = 1 + 1j / (k * r) - 1 / (k * r) ** 2
    b_ = -1 - 3j / (k * r) + 3 / (k * r) ** 2
    Dy = A * (a_ * np.eye(3) + b_ * np.outer(d, d))
    want = [Dy[0, 0], Dy[1, 1], Dy[2, 2], Dy[0, 1], Dy[0, 2], Dy[1, 2]]
    assert np.allclose(vm, want, rtol=0, atol=2e-3 * np.abs(want).max())
    # series second derivatives vs finite differences of the series G_d
    h = 1e-4
    x0 = np.array([[0.7, -0.4, 0.8]])
    def gd(yv):
        return O.series(pb, yv, O.OUT_GD)[0, 0]
    e = np.eye(3)
    H = np.zeros((3, 3), complex)
    for p in range(3):
        for q in range(3):
            H[p, q] = (gd(x0 + h * (e[p] + e[q])) - gd(x0 + h * (e[p] - e[q])) - gd(x0 - h * (e[p] - e[q]))
                       + gd(x0 - h * (e[p] + e[q]))) / (4 * h * h)
    G0 = gd(x0)
    want = [G0 + H[0, 0] / k**2, G0 + H[1, 1] / k**2, G0 + H[2, 2] / k**2,
            H[0, 1] / k**2, H[0, 2] / k**2, H[1, 2] / k**2]
    got = O.series(pb, x0, O.OUT_MAXWELL6)[0]
    assert np.allclose(got, want, rtol=1e-5, atol=1e-7)


# --------------------------------------------------------------------------- 2D
def test_2d_algorithm_vs_series_and_hankel():
    errs = []
    pts = np.array([[0.5 * np.pi, 0.1], [0.01 * np.pi, 0.05], [-2.0, -0.3], [1.0, 0.55], [3.0, 0.2]])
    for M in [(64, 64), (256, 256)]:
        pb = O.Problem(dim=2, k=1.3, alpha=(0.2,), M=M)
        g = O.grid(pb)
        v = O.evaluate(pb, g, pts, O.OUT_G)[:, 0]
        s = O.series(pb, pts, O.OUT_G)[:, 0]
        errs.append(np.abs(v - s).max() / np.abs(s).max())
    assert errs[1] < 1e-4 and errs[1] < errs[0] / 4, errs  # O(N^-2), Thm 2.1/2.2
    # near the origin: G - (i/4) H0(kr) is regular (Sec. 2.2, image expansion (ii))
    d = np.array([0.6, 0.8])
    rs = np.array([1e-3, 2e-3, 4e-3])
    v = O.evaluate(pb, g, rs[:, None] * d[None, :], O.OUT_G)[:, 0]
    reg = v - 0.25j * special.hankel1(0, pb.k * rs)
    assert abs(reg[1] - reg[0]) < 0.02 * abs(reg[0]) and abs(reg[2] - reg[1]) < 0.02 * abs(reg[0])
    # quasi-periodicity in x1
    x = np.array([[0.3, 0.1], [2.0, -0.7], [-1.0, 0.4]])
    v0 = O.evaluate(pb, g, x, O.OUT_G)[:, 0]
    v1 = O.evaluate(pb, g, x + np.array([4 * np.pi, 0]), O.OUT_G)[:, 0]
    assert np.allclose(v1, np.exp(4j * np.pi * 0.2) * v0, rtol=1e-12)


def test_2d_image_expansion_far_point():
    """(ei) vs the image expansion (ii) summed with a Kummer-free check at a
    point where both converge to the same value: compare against a direct
    numerical sum of (ii) with many images and a smooth window."""
    pb = O.Problem(dim=2, k=1.3, alpha=(0.2,), M=(16, 16))
    x = np.array([[0.7, 0.9]])
    s = O.series(pb, x, O.OUT_G)[0, 0]
    # (ii) converges slowly; accelerate with the alpha-weighted Cesaro-free trick:
    # sum over |n| <= Nn of e^{i 2 pi alpha n} H0(k r_n) with a smooth taper
    Nn = 40000
    n = np.arange(-Nn, Nn + 1)
    rn = np.hypot(x[0, 0] - 2 * np.pi * n, x[0, 1])
    taper = np.exp(-(n / (0.35 * Nn)) ** 2)
    ii = 0.25j * np.sum(np.exp(2j * np.pi * 0.2 * n) * special.hankel1(0, pb.k * rn) * taper)
    assert abs(ii - s) < 2e-3 * abs(s)
