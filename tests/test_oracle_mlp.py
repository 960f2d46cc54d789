"""Pins of the FP64 reference MLP: analytic gradients vs central finite
differences of its loss, and the SiLU derivative vs finite differences."""
import numpy as np

from oracle import mlp as R


def test_silu_derivative():
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    fd = (R.silu(z + h) - R.silu(z - h)) / (2 * h)
    assert np.allclose(fd, R.dsilu(z), rtol=1e-7, atol=1e-9)


def test_features_layout():
    inp = np.array([[0.3, -1.2, 0.4, 0.1, -0.2, 3.0]])
    X = R.features(inp)
    fr = R.frequencies()
    assert fr.shape == (32, 3) and len({tuple(f) for f in fr}) == 32 and not (fr == 0).all(1).any()
    ph = fr[5, 0] * 0.3 + fr[5, 1] * -1.2 + fr[5, 2] * np.pi * 0.4
    assert abs(X[0, 10] - np.cos(ph)) < 1e-15 and abs(X[0, 11] - np.sin(ph)) < 1e-15
    assert X[0, 64] == 0.2 and X[0, 65] == -0.4 and abs(X[0, 66] - 1 / 3) < 1e-15
    r = np.sqrt(0.3**2 + 1.2**2 + 0.4**2)
    assert abs(X[0, 67] - r) < 1e-15 and abs(X[0, 68 + 8] - np.exp(-0.5 * ((r - 1.2) / 0.15) ** 2)) < 1e-15


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    npar = sum(R.DIMS[l + 1] * R.DIMS[l] + R.DIMS[l + 1] for l in range(5))
    p = rng.standard_normal(npar) * 0.05
    inp = np.column_stack([rng.uniform(-np.pi, np.pi, (8, 2)), rng.uniform(-0.6, 0.6, 8),
                           rng.uniform(-0.5, 0.5, (8, 2)), rng.uniform(1, 4, 8)])
    tgt = rng.standard_normal((8, 2))
    loss, g = R.loss_and_grad(p, inp, tgt)
    h = 1e-6
    for idx in rng.choice(npar, 40, replace=False):
        e = np.zeros(npar)
        e[idx] = h
        fd = (R.loss_and_grad(p + e, inp, tgt)[0] - R.loss_and_grad(p - e, inp, tgt)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), idx
