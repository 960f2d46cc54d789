"""FP64 NumPy reference of the surrogate network (test infrastructure only).

Plain double-precision forward and backward passes of the 5-layer MLP the
library trains on the tensor cores: features cos/sin(n1 t1 + n2 t2 + m3 pi x3/c~)
for 32 integer vectors (n1, n2, m3), 2 alpha1, 2 alpha2, (k - 2.5)/1.5, the
in-cell distance r and 12 Gaussian shells exp(-((r - 0.15 j)/0.15)^2/2); layers 80 -> 256 -> 256 -> 256 -> 256 -> 2 with SiLU between
them; loss sum (Y - T)^2 / (2n).  Parameters are flattened layer by layer as
W [out][in] then b [out].  Written from the layer equations; shares no code
with the CUDA library.  Its gradients are pinned against finite differences.
"""
from __future__ import annotations

import numpy as np

DIMS = [80, 256, 256, 256, 256, 2]


def frequencies():
    """The 32 feature vectors (n1, n2, m3): the 17 non-zero ones with n1, n2 in
    {-1, 0, 1} and m3 in {0, 1} (m3 slowest, then n1, then n2), then 15 higher ones."""
    fr = []
    for m3 in range(2):
        for n1 in (-1, 0, 1):
            for n2 in (-1, 0, 1):
                if n1 or n2 or m3:
                    fr.append((n1, n2, m3))
    fr += [(0, 0, 2), (0, 0, 3), (2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (2, 0, 1), (0, 2, 1),
           (3, 0, 0), (0, 3, 0), (-3, 0, 0), (0, -3, 0), (1, 1, 2), (-1, 1, 2), (2, 2, 0)]
    return np.array(fr, dtype=np.float64)


def features(inp: np.ndarray, c_tilde: float = 1.0) -> np.ndarray:
    inp = np.asarray(inp, dtype=np.float64)
    t1, t2, x3, a1, a2, k = inp.T
    fr = frequencies()
    ph = np.outer(t1, fr[:, 0]) + np.outer(t2, fr[:, 1]) + np.outer(np.pi / c_tilde * x3, fr[:, 2])
    X = np.zeros((inp.shape[0], DIMS[0]))
    X[:, 0:64:2] = np.cos(ph)
    X[:, 1:64:2] = np.sin(ph)
    X[:, 64] = 2 * a1
    X[:, 65] = 2 * a2
    X[:, 66] = (k - 2.5) / 1.5
    r = np.sqrt(t1 * t1 + t2 * t2 + x3 * x3)
    X[:, 67] = r
    for j in range(12):
        X[:, 68 + j] = np.exp(-0.5 * ((r - 0.15 * j) / 0.15) ** 2)
    return X


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    Ws, bs, off = [], [], 0
    for l in range(5):
        o, i = DIMS[l + 1], DIMS[l]
        Ws.append(p[off:off + o * i].reshape(o, i))
        off += o * i
        bs.append(p[off:off + o])
        off += o
    return Ws, bs


def pack(Ws, bs) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, inp, c_tilde=1.0):
    Ws, bs = unpack(p)
    h = features(inp, c_tilde)
    for l in range(4):
        h = silu(h @ Ws[l].T + bs[l])
    return h @ Ws[4].T + bs[4]


def loss_and_grad(p, inp, target, c_tilde=1.0):
    """Loss sum (Y - T)^2 / (2n) and its gradient (flattened like p)."""
    Ws, bs = unpack(p)
    n = inp.shape[0]
    acts, pre = [features(inp, c_tilde)], []
    for l in range(4):
        z = acts[-1] @ Ws[l].T + bs[l]
        pre.append(z)
        acts.append(silu(z))
    Y = acts[-1] @ Ws[4].T + bs[4]
    d = Y - np.asarray(target, dtype=np.float64)
    loss = 0.5 * np.sum(d * d) / n
    gW, gb = [None] * 5, [None] * 5
    dz = d / n
    gW[4] = dz.T @ acts[4]
    gb[4] = dz.sum(0)
    dh = dz @ Ws[4]
    for l in range(3, -1, -1):
        dz = dh * dsilu(pre[l])
        gW[l] = dz.T @ acts[l]
        gb[l] = dz.sum(0)
        dh = dz @ Ws[l]
    return loss, pack(gW, gb)
