"""The host-side counts behind bench.py's roofline, against brute force.

The far series of a 3D target runs over the lattice points n in Z^2 with
|alpha + n|^2 <= k^2 + (T/|x3|)^2 (Eq. (he), truncated); bench.py counts them,
and the core and double-band subsets, row by row to turn kernel time into
algorithmic work.  Here each count is compared with plain enumeration of the
lattice on small cases, so a wrong row range or rounding in the counting
cannot pass unseen into the reported flops.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def brute_disk(R2, alpha):
    """Lattice points with |alpha + n|^2 <= R2, summed over the entries of R2, by enumeration."""
    R = np.sqrt(max(float(np.max(R2)), 0.0))
    n = np.arange(-int(R) - 3, int(R) + 4)
    c1 = alpha[0] + n[:, None]
    c2 = alpha[1] + n[None, :]
    a2 = (c1 * c1 + c2 * c2).ravel()
    return int(sum(np.count_nonzero(a2 <= r2) for r2 in np.atleast_1d(R2)))


@pytest.mark.parametrize("alpha", [(0.1, 0.3), (-0.37, 0.0123), (0.5, -0.5)])
def test_disk_count_matches_enumeration(alpha):
    rng = np.random.default_rng(5)
    R2 = rng.uniform(0.0, 400.0, 60)
    assert bench.disk_count(R2, alpha) == brute_disk(R2, alpha)
    # radii below the nearest lattice point: no terms
    a = np.array(alpha)
    nearest = min(float(np.sum((a + np.array(m)) ** 2)) for m in [(0, 0), (-1, 0), (0, -1), (-1, -1), (1, 0), (0, 1)])
    assert bench.disk_count(np.array([0.5 * nearest]), alpha) == 0


@pytest.mark.parametrize("k,alpha", [(2.5, (0.1, 0.3)), (1.0, (0.002, 0.0)), (4.2, (-0.3, 0.45))])
def test_smallest_evanescent_beta_matches_enumeration(k, alpha):
    n = np.arange(-20, 21)
    c1 = alpha[0] + n[:, None]
    c2 = alpha[1] + n[None, :]
    a2 = (c1 * c1 + c2 * c2).ravel()
    ref = float(np.sqrt(a2[a2 > k * k] - k * k).min())
    assert bench.smallest_evanescent_beta(k, alpha) == pytest.approx(ref, rel=1e-15)


def test_far_terms_nested_and_counted_per_target():
    k, alpha, c, tol = 2.5, (0.1, 0.3), 0.6, 1e-16
    rng = np.random.default_rng(9)
    x = np.column_stack([rng.uniform(0, 6, 40), rng.uniform(0, 6, 40), rng.uniform(-2.0, 2.0, 40)])
    total, core, bands = bench.far_terms(x, k, alpha, c, tol)
    assert bands["double"] + bands["float-float"] == core
    assert 0 < bands["double"] <= core <= total
    # near targets (|x3| <= c) add nothing; far targets add their own disks
    z = np.abs(x[:, 2])
    far = z > c
    T = np.log(1.0 / tol) + 3.0
    assert total == sum(brute_disk(np.array([k * k + (T / zi) ** 2]), alpha) for zi in z[far])
    assert bench.far_terms(x[~far], k, alpha, c, tol)[0] == 0
