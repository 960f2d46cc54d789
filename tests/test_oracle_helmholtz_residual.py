"""Finite-difference Helmholtz residual of the oracle's G (2D) and G_d (3D), far branch.

Away from the lattice points G solves Delta G + k^2 G = 0 (the problem statement of
Sec. 1; the quasi-periodic Green's functions of Secs. 2 and 3).  The oracle's far branch
(|x_last| > c, the eigen-series (ei)/(he) truncated as the plan states) is checked
against that equation, which none of its parts assumes: the residual, by the
fourth-order Richardson combination of central differences with steps h and h/2, sits at
the level of the differencing error.  A term whose beta does not satisfy
beta^2 = k^2 - |alpha_n|^2 with the alpha_n of its own phase (a wrong index, alpha or k)
leaves a residual of the size of that term; the branch of beta and the 1/beta factor,
which each term's equation leaves free, are pinned by the image expansion and the
singularity tests instead.  (The near branch is pinned by its values
against the exact series instead: its values converge to the series, but its second
derivatives converge slowly, being those of a cubic gather of a periodised remainder
that carries the slab's cutoff; measured residual ~0.1 of k^2 max|G| at 64^2 in 2D.)
"""
import numpy as np
import pytest

from oracle import oracle as O


def laplacian_residual(f, x, k, h):
    """(sum_i central second difference along axis i) + k^2 f, at the rows of x."""
    f0 = f(x)
    lap = np.zeros_like(f0)
    for ax in range(x.shape[1]):
        e = np.zeros(x.shape[1])
        e[ax] = h
        lap += (f(x + e) - 2.0 * f0 + f(x - e)) / (h * h)
    return lap + k * k * f0, f0


def richardson_residual(f, x, k, h):
    r1, f0 = laplacian_residual(f, x, k, h)
    r2, _ = laplacian_residual(f, x, k, h / 2)
    return (4.0 * r2 - r1) / 3.0, f0


def scale(f0, k):
    return k * k * np.abs(f0).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_far_branch_solves_helmholtz(dim):
    if dim == 3:
        pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(16, 16, 16))
        lo, hi = np.array([-3.0, -3.0, 0.7]), np.array([3.0, 3.0, 1.6])
        which = O.OUT_GD
    else:
        pb = O.Problem(dim=2, k=1.3, alpha=(0.2,), M=(16, 16))
        lo, hi = np.array([-3.0, 0.7]), np.array([3.0, 1.6])
        which = O.OUT_G
    g = O.grid(pb)
    rng = np.random.default_rng(11 + dim)
    x = rng.uniform(lo, hi, (24, dim))
    x[::2, -1] *= -1.0
    f = lambda y: O.evaluate(pb, g, y, which)[:, 0]
    r, f0 = richardson_residual(f, x, pb.k, 2e-2)
    rel = np.abs(r).max() / scale(f0, pb.k)
    print(f"{dim}D far branch: Helmholtz residual {rel:.2e} of k^2 max|G|")
    assert rel < 1e-7
