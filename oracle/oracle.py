"""ctypes front end of the FP64 CPU oracle (oracle/gf_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the library never imports it.  It
shares no code with the CUDA path.

The oracle follows Algorithms 1-3 of Zhang & Zhang (arXiv:1801.05977) step by
step in double precision, with a naive O(M^2)-per-line inverse DFT in place of
the FFT.  Parity of every function is pinned in ``tests/test_oracle_*.py``
against the problem's definitions (eigenfunction expansions (ei)/(he)),
independent quadratures of the Fourier-coefficient definitions, library
special functions and structural invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("M", ctypes.c_int * 3),
        ("Q", ctypes.c_int),
        ("maxwell", ctypes.c_int),
        ("k", ctypes.c_double),
        ("alpha", ctypes.c_double * 2),
        ("c", ctypes.c_double),
        ("ct", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("tau", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, p, l = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_long
        P = ctypes.POINTER(Params)
        _lib.or_smooth8.restype = d
        _lib.or_smooth8.argtypes = [d, i]
        _lib.or_chi.restype = d
        _lib.or_chi.argtypes = [d, d, d, i]
        _lib.or_yps.restype = d
        _lib.or_yps.argtypes = [d, d, i]
        _lib.or_gauss_legendre.argtypes = [i, p, p]
        _lib.or_beta.argtypes = [d, d, p, p]
        _lib.or_bessel_j01.argtypes = [d, p, p]
        _lib.or_coef.restype = i
        _lib.or_coef.argtypes = [P, p]
        _lib.or_coef_parts.argtypes = [P, i, i, i, p]
        _lib.or_grid.argtypes = [P, p, p]
        _lib.or_eval.argtypes = [P, p, p, l, i, p]
        _lib.or_series.argtypes = [P, p, l, i, p]
        _lib.or_interp.argtypes = [P, p, p, l, p]
        _lib.or_grid_nodes.argtypes = [P, p, i, p, l, p]
        _lib.or_far_grid.argtypes = [P, i, i, i, d, p]
        _lib.or_eval_far_grid.argtypes = [P, i, i, i, d, p, p, l, i, p]
        _lib.or_set_threads.restype = i
        _lib.or_set_threads.argtypes = [i]
        _lib.or_bessel_j0123.argtypes = [d, p]
        _lib.or_deriv2_singular_at.argtypes = [P, d, p, l, p]
        _lib.or_deriv2_parts.argtypes = [P, d, i, i, p]
        _lib.or_coef_deriv2.restype = i
        _lib.or_coef_deriv2.argtypes = [P, d, p]
        _lib.or_series_deriv2.argtypes = [P, d, p, l, i, p]
        _lib.or_eval_deriv2.argtypes = [P, d, p, p, l, i, p]
    return _lib


def set_threads(n: int = 0) -> int:
    """OpenMP threads of the oracle's loops (n > 0 sets them); returns the count in effect."""
    return int(lib().or_set_threads(int(n)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


OUT_G, OUT_GD, OUT_MAXWELL6, OUT_MAXWELL7, OUT_LD = 0, 1, 2, 3, 4
N_ENTRIES = {OUT_G: 1, OUT_GD: 1, OUT_MAXWELL6: 6, OUT_MAXWELL7: 7, OUT_LD: 1}


@dataclass
class Problem:
    """One (k, alpha, grid) problem.  M = grid points per axis (paper's 2N)."""

    dim: int
    k: float
    alpha: tuple
    M: tuple
    c: float = 0.6
    ct: float = 1.0
    eps: float = 0.45
    tau: float = 1e-16
    Q: int = 64
    maxwell: bool = False
    _c: Params = field(default=None, repr=False)

    def cstruct(self) -> Params:
        p = Params()
        p.dim = self.dim
        for a in range(3):
            p.M[a] = int(self.M[a]) if a < len(self.M) else 1
        p.Q = self.Q
        p.maxwell = int(self.maxwell)
        p.k = self.k
        al = list(self.alpha) + [0.0] * (2 - len(self.alpha))
        p.alpha[0], p.alpha[1] = al[0], al[1]
        p.c, p.ct, p.eps, p.tau = self.c, self.ct, self.eps, self.tau
        return p

    @property
    def nfields(self) -> int:
        return 7 if (self.dim == 3 and self.maxwell) else 1

    @property
    def shape(self) -> tuple:
        """Array shape of one field: (M3, M2, M1) in 3D, (M2, M1) in 2D."""
        return tuple(int(m) for m in reversed(self.M[: self.dim]))


def smooth8(s: float, d: int = 0) -> float:
    return lib().or_smooth8(float(s), int(d))


def chi(t: float, c: float, ct: float, d: int = 0) -> float:
    return lib().or_chi(float(t), float(c), float(ct), int(d))


def yps(r: float, eps: float, d: int = 0) -> float:
    return lib().or_yps(float(r), float(eps), int(d))


def gauss_legendre(Q: int):
    x = np.zeros(Q)
    w = np.zeros(Q)
    lib().or_gauss_legendre(Q, _ptr(x), _ptr(w))
    return x, w


def beta(k: float, a2: float) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_beta(float(k), float(a2), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def bessel_j01(z: float):
    j0, j1 = ctypes.c_double(), ctypes.c_double()
    lib().or_bessel_j01(float(z), ctypes.byref(j0), ctypes.byref(j1))
    return j0.value, j1.value


def coef(pb: Problem) -> np.ndarray:
    """sqrt(V) L-hat_j in FFT order, shape (nfields, *pb.shape), complex128."""
    out = np.zeros((pb.nfields,) + pb.shape, dtype=np.complex128)
    p = pb.cstruct()
    rc = lib().or_coef(ctypes.byref(p), _ptr(out))
    if rc != 0:
        raise ValueError("Wood anomaly or resonance in the coefficient set")
    return out


def coef_parts(pb: Problem, j1: int, j2: int, j3: int = 0) -> np.ndarray:
    out = np.zeros(3, dtype=np.complex128)
    p = pb.cstruct()
    lib().or_coef_parts(ctypes.byref(p), int(j1), int(j2), int(j3), _ptr(out))
    return out[:2] if pb.dim == 3 else out


def grid(pb: Problem, C: np.ndarray | None = None) -> np.ndarray:
    """Remainder grid L_N at the nodes (naive inverse DFT), shape (nfields, *shape)."""
    if C is None:
        C = coef(pb)
    C = np.ascontiguousarray(C, dtype=np.complex128)
    out = np.zeros_like(C)
    p = pb.cstruct()
    lib().or_grid(ctypes.byref(p), _ptr(C), _ptr(out))
    return out


def grid_nodes(pb: Problem, C: np.ndarray, nodes: np.ndarray, field: int = 0) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.complex128)
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    out = np.zeros(nodes.shape[0], dtype=np.complex128)
    p = pb.cstruct()
    lib().or_grid_nodes(ctypes.byref(p), _ptr(C), int(field), _ptr(nodes), nodes.shape[0], _ptr(out))
    return out


def evaluate(pb: Problem, g: np.ndarray, x: np.ndarray, which: int) -> np.ndarray:
    """Algorithms 1-3, calculation step, at the points x (n, dim)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    ne = N_ENTRIES[which]
    out = np.zeros((x.shape[0], ne), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_eval(ctypes.byref(p), _ptr(g), _ptr(x), x.shape[0], int(which), _ptr(out))
    return out


def series(pb: Problem, x: np.ndarray, which: int) -> np.ndarray:
    """Eigenfunction expansion (ei)/(he) (and its second derivatives) at x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    ne = N_ENTRIES[which]
    out = np.zeros((x.shape[0], ne), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_series(ctypes.byref(p), _ptr(x), x.shape[0], int(which), _ptr(out))
    return out


def interp(pb: Problem, g: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Tensor cubic interpolation of one field at coordinates y (n, dim)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    out = np.zeros(y.shape[0], dtype=np.complex128)
    p = pb.cstruct()
    lib().or_interp(ctypes.byref(p), _ptr(g), _ptr(y), y.shape[0], _ptr(out))
    return out


def run(pb: Problem, x: np.ndarray, which: int) -> np.ndarray:
    """Whole path: coefficients, grid, point values."""
    return evaluate(pb, grid(pb), x, which)


def far_grid(pb: Problem, Mf, Nz: int, zmax: float) -> np.ndarray:
    """Far-region grid: F = e^{-i alpha.t} G_d on planes z_m = c + (m - 1) hz,
    m = 0 .. Nz + 2, by a naive inverse DFT of the series terms over n in S_Mf;
    shape (nfields, Nz + 3, Mf2, Mf1)."""
    Mf1, Mf2 = (Mf, Mf) if np.isscalar(Mf) else Mf
    out = np.zeros((pb.nfields, Nz + 3, Mf2, Mf1), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_far_grid(ctypes.byref(p), int(Mf1), int(Mf2), int(Nz), float(zmax), _ptr(out))
    return out


def far_grid_evaluate(pb: Problem, fg: np.ndarray, Nz: int, zmax: float, x: np.ndarray, which: int) -> np.ndarray:
    """Targets with c < |x3| <= zmax from the far-region grid (tensor cubics + phase)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    fg = np.ascontiguousarray(fg, dtype=np.complex128)
    ne = N_ENTRIES[which]
    out = np.zeros((x.shape[0], ne), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_eval_far_grid(ctypes.byref(p), int(fg.shape[3]), int(fg.shape[2]), int(Nz), float(zmax), _ptr(fg),
                           _ptr(x), x.shape[0], int(which), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# 2D derivatives (Sec. 2.4): gradient (Sec. 2.4.1) and the differences of
# second derivatives for two wave numbers (Sec. 2.4.2).
# ---------------------------------------------------------------------------
DERIV_GRAD, DERIV_HYPER = 0, 1
DERIV_FIELDS = ("K1-h1", "K2-h2", "T11-h11", "T12-h12", "T22-h22")


def bessel_j0123(z: float) -> np.ndarray:
    """J_0 .. J_3 at z from one trapezoidal sum of Bessel's integral (the transforms' routine)."""
    out = np.zeros(4)
    lib().or_bessel_j0123(float(z), _ptr(out))
    return out


def deriv2_parts(pb: Problem, k2: float, j1: int, j2: int) -> tuple[np.ndarray, np.ndarray]:
    """(twelve plane transforms of the singular functions, the five sqrt(V) H-hat) of index j."""
    out = np.zeros(17, dtype=np.complex128)
    p = pb.cstruct()
    lib().or_deriv2_parts(ctypes.byref(p), float(k2), int(j1), int(j2), _ptr(out))
    return out[:12], out[12:]


def deriv2_singular_at(pb: Problem, k2: float, x: np.ndarray) -> np.ndarray:
    """The singular parts h_1, h_2, h_11, h_12, h_22 at in-cell points x (n, 2)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], 5), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_deriv2_singular_at(ctypes.byref(p), float(k2), _ptr(x), x.shape[0], _ptr(out))
    return out


def coef_deriv2(pb: Problem, k2: float = 0.0) -> np.ndarray:
    """sqrt(V) coefficients of K1-h1, K2-h2 (and T11-h11, T12-h12, T22-h22 when k2 > 0),
    FFT order, shape (nf, M2, M1)."""
    nf = 5 if k2 > 0 else 2
    out = np.zeros((nf,) + pb.shape, dtype=np.complex128)
    p = pb.cstruct()
    if lib().or_coef_deriv2(ctypes.byref(p), float(k2), _ptr(out)) != 0:
        raise ValueError("Wood anomaly or resonance in the coefficient set")
    return out


def grid_deriv2(pb: Problem, k2: float = 0.0) -> np.ndarray:
    """The derivative remainder fields at the nodes (naive inverse DFT per field)."""
    C = coef_deriv2(pb, k2)
    return np.stack([grid(pb, C[f:f + 1])[0] for f in range(C.shape[0])])


def series_deriv2(pb: Problem, k2: float, x: np.ndarray, which: int) -> np.ndarray:
    """Term-by-term derivatives of (ei): which 0 -> (dG/dx1, dG/dx2), 1 -> (T11, T12, T22)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], 2 if which == 0 else 3), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_series_deriv2(ctypes.byref(p), float(k2), _ptr(x), x.shape[0], int(which), _ptr(out))
    return out


def evaluate_deriv2(pb: Problem, k2: float, g: np.ndarray, x: np.ndarray, which: int) -> np.ndarray:
    """Algorithm 1's calculation step for the derivative fields at the points x (n, 2)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    if which == 1 and g.shape[0] < 5:
        raise ValueError("T fields need k2 > 0")
    out = np.zeros((x.shape[0], 2 if which == 0 else 3), dtype=np.complex128)
    p = pb.cstruct()
    lib().or_eval_deriv2(ctypes.byref(p), float(k2), _ptr(g), _ptr(x), x.shape[0], int(which), _ptr(out))
    return out
