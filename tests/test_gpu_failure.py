"""Failure detection on the GPU without a fault: the bounded device waits.

The tensor-core kernels of the surrogate wait on mbarriers with a poll limit
and, when it runs out, record an error word and unwind, so that the host gets
GF_ERR_TIMEOUT instead of a hung GPU.  gf_wait_selftest runs that same wait on
a barrier nothing arrives at (short limit), so the limit is the only way out:
the status must say so, and the context must stay usable afterwards.  A
control run arrives on the barrier first and must complete.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1801_05977_gb300 import gf
from paper_1801_05977_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_survives():
    assert gf.wait_selftest(2000, arrive=False) == gf.GF_ERR_TIMEOUT
    assert "ran out" in gf.lib().gf_last_error().decode()
    assert gf.wait_selftest(2000, arrive=True) == gf.GF_OK
    # an evaluation after the timed-out wait still matches the oracle
    pb = O.Problem(dim=3, k=2.5, alpha=(0.1, 0.3), M=(16, 16, 16))
    plan = gf.Plan(3, pb.k, pb.alpha, pb.M, series_tol=pb.tau, quad_nodes=pb.Q)
    x = W.targets_3d(500, seed=91)
    got = plan.eval_points(torch.from_numpy(x).cuda(), gf.GF_OUT_GD).cpu().numpy()
    ref = O.evaluate(pb, O.grid(pb), x, O.OUT_GD)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
    plan.close()
    assert gf.lib().gf_wait_selftest(0, 0, None) == gf.GF_ERR_ARG
