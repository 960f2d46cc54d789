"""Training and use of the learned surrogate of the smooth remainder L_d.

Data: the FFT path itself.  For P (alpha, k) pairs (k in [1, 4], alpha in
[-1/2, 1/2]^2, pairs within `wood_gap` of a Wood anomaly redrawn) a batched
sweep (gf_plan_batch, split precision) evaluates the interpolated remainder
L_dN (GF_OUT_LD) at `per_pair` near-region points (x1, x2 ~ U[-pi, pi),
x3 ~ U[-c, c]).  Samples are (t1, t2, x3, alpha1, alpha2, k) -> L_d / scale,
shuffled once on the host.  Training runs the library's own tensor-core
forward/backward kernels and Adam (gf_mlp_train_step) over mini-batches.

Residual form: the network learns L_d minus the remainder of a coarse plan
(COARSE points per axis), which a coarse batched sweep supplies again at
inference (gf_surrogate_eval_residual adds it back); the network then only
has to carry the difference between the two grids.
"""
from __future__ import annotations

import math

import numpy as np

from . import gf
from . import workloads as W


# grid of the coarse plans of the residual form (points per axis)
COARSE = (32, 32, 32)


def grid_for(k: float) -> tuple:
    m = int(min(256, max(32, 2 ** math.ceil(math.log2(math.ceil(32 * k))))))
    return (m, m, 64)


def near_points(n: int, seed: int, c: float = 0.6) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((n, 3))
    x[:, 0] = rng.uniform(-np.pi, np.pi, n)
    x[:, 1] = rng.uniform(-np.pi, np.pi, n)
    x[:, 2] = rng.uniform(-c, c, n)
    return x


def remainder_values(pairs, xd, off, M=None, precision=gf.GF_FP32_SPLIT):
    """L_d of one plan per pair (grid grid_for(k), or M for every pair) at the
    rows of xd (pair p owns rows off[p] .. off[p+1]-1): complex CUDA tensor [N]."""
    import torch

    k = np.ascontiguousarray(pairs[:, 2])
    al = np.ascontiguousarray(pairs[:, :2])
    Mm = np.array([M if M is not None else grid_for(v) for v in k], dtype=np.int32)
    batch = gf.Batch(k, al, Mm, precision=precision)
    out = torch.empty((xd.shape[0], 1), dtype=batch.complex_dtype, device=xd.device)
    batch.eval_points_into(xd, off, out, gf.GF_OUT_LD)
    torch.cuda.synchronize()
    batch.close()
    return out[:, 0]


def make_dataset(n_pairs: int, per_pair: int, seed: int = 0, wood_gap: float = 1e-2, kmin=1.0, kmax=4.0,
                 residual: bool = False):
    """Returns (inputs float32 [N][6], targets complex64 [N], pairs [P][3] (a1, a2, k)).
    residual: the targets are L_d minus the coarse plans' L_d (COARSE points per axis)."""
    import torch

    pairs = W.sweep_pairs(n_pairs, seed=seed, kmin=kmin, kmax=kmax, wood_gap=wood_gap)
    k = pairs[:, 2].copy()
    al = pairs[:, :2].copy()
    xs = [near_points(per_pair, seed=10_000 * (seed + 1) + i) for i in range(n_pairs)]
    x = np.concatenate(xs)
    off = np.arange(n_pairs + 1, dtype=np.int64) * per_pair
    xd = torch.from_numpy(x).cuda()
    Lt = remainder_values(pairs, xd, off)
    if residual:
        Lt = Lt - remainder_values(pairs, xd, off, M=COARSE)
    L = Lt.cpu().numpy()
    inp = np.empty((x.shape[0], 6), dtype=np.float32)
    inp[:, :3] = x
    rep = np.repeat(np.arange(n_pairs), per_pair)
    inp[:, 3:5] = al[rep]
    inp[:, 5] = k[rep]
    return inp, L, pairs


def train(mlp: "gf.MLP", inp: np.ndarray, L: np.ndarray, epochs: int = 8, batch: int = 8192, lr: float = 2e-3,
          seed: int = 0, log=None, min_steps: int = 0):
    """Adam on mean-squared error of L / scale; cosine learning-rate decay.
    At least `min_steps` optimizer steps are taken (epochs are extended)."""
    import torch

    scale = float(np.sqrt(np.mean(np.abs(L) ** 2)))
    mlp.set_scale(scale)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(inp.shape[0])
    xin = torch.from_numpy(np.ascontiguousarray(inp[perm])).cuda()
    tg = np.empty((inp.shape[0], 2), dtype=np.float32)
    tg[:, 0] = L.real / scale
    tg[:, 1] = L.imag / scale
    tgt = torch.from_numpy(tg[perm]).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    nb = inp.shape[0] // batch
    epochs = max(epochs, -(-min_steps // nb))
    total = epochs * nb
    it = 0
    hist = []
    for ep in range(epochs):
        for b in range(nb):
            lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * it / total)) + 1e-5
            mlp.train_step(xin[b * batch:(b + 1) * batch], tgt[b * batch:(b + 1) * batch], lr_t, loss)
            it += 1
        torch.cuda.synchronize()
        hist.append(float(loss.item()))
        if log:
            log(f"epoch {ep}: last-batch loss {hist[-1]:.3e}")
    return hist
