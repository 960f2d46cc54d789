"""Batched (alpha, k) sweeps: the batched persistent launches and the CUDA
graph must reproduce, pair by pair, what each pair's plan gives alone, and the
oracle."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1801_05977_gb300 import gf
from paper_1801_05977_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAIRS = [  # k, alpha, M (uneven grids)
    (2.5, (0.1, 0.3), (32, 32, 16)),
    (0.9, (-0.35, 0.2), (16, 16, 16)),
    (4.4, (0.45, -0.1), (64, 32, 16)),
    (1.7, (0.0, 0.25), (16, 32, 8)),
    (3.1, (-0.2, -0.4), (32, 16, 32)),
]
COUNTS = [1000, 0, 2500, 31, 777]


def rel_err(got, ref, floor=1e-6):
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max())
    return float((np.abs(got - ref) / scale).max())


def norm_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def make(precision):
    k = np.array([p[0] for p in PAIRS])
    al = np.array([p[1] for p in PAIRS])
    M = np.array([p[2] for p in PAIRS])
    b = gf.Batch(k, al, M, precision=precision)
    xs = [W.targets_3d(n, seed=10 + i) if n else np.zeros((0, 3)) for i, n in enumerate(COUNTS)]
    off = np.concatenate([[0], np.cumsum(COUNTS)]).astype(np.int64)
    x = torch.from_numpy(np.concatenate(xs)).cuda()
    return b, xs, off, x


@pytest.mark.parametrize("precision", [gf.GF_FP64, gf.GF_FP32_SPLIT])
def test_batch_matches_single_plans(precision):
    b, xs, off, x = make(precision)
    out = torch.empty((int(off[-1]), 1), dtype=b.complex_dtype, device="cuda")
    b.eval_points_into(x, off, out, gf.GF_OUT_GD)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, (k, al, M) in enumerate(PAIRS):
        if COUNTS[i] == 0:
            continue
        p = gf.Plan(3, k, al, M, precision=precision)
        ref = p.eval_points(torch.from_numpy(xs[i]).cuda(), gf.GF_OUT_GD).cpu().numpy()
        g = got[off[i]:off[i + 1]]
        if precision == gf.GF_FP64:
            assert rel_err(g, ref) < 1e-11, i
        else:
            assert norm_err(g, ref) < 2e-5, i
        p.close()
    b.close()


def test_batch_vs_oracle_and_resynthesis():
    b, xs, off, x = make(gf.GF_FP64)
    b.synthesize()  # re-run all pairs' synthesis as batched launches
    out = torch.empty((int(off[-1]), 1), dtype=torch.complex128, device="cuda")
    b.eval_points_into(x, off, out, gf.GF_OUT_GD)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in (0, 2, 4):
        k, al, M = PAIRS[i]
        pb = O.Problem(dim=3, k=k, alpha=al, M=M)
        ref = O.evaluate(pb, O.grid(pb), xs[i], O.OUT_GD)
        assert rel_err(got[off[i]:off[i + 1]], ref) < 1e-10, i
    b.close()


def test_batch_graph_and_autotune():
    b, xs, off, x = make(gf.GF_FP64)
    ref = torch.empty((int(off[-1]), 1), dtype=torch.complex128, device="cuda")
    b.eval_points_into(x, off, ref, gf.GF_OUT_GD)
    tune = b.autotune(x, off, torch.empty_like(ref), gf.GF_OUT_GD)
    assert tune[0] in (2, 4, 8, 16) and tune[1] in (64, 128, 256) and tune[2] in (4, 8, 16)
    s = torch.cuda.Stream()
    out = torch.zeros_like(ref)
    with torch.cuda.stream(s):
        for _ in range(2):  # capture, then replay
            out.zero_()
            b.run_graph(x, off, out, gf.GF_OUT_GD, stream=s)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-11
    b.close()
