"""The arithmetic peak probe's overlap modes (diagnostic): FP64 chains on half
the warps, FP32 chains on the other half, each alone and together.  Together
they can take no less than the longer half and no more than the two halves'
sum (plus launch noise); the bench reports where between the two they fall."""
import pytest

torch = pytest.importorskip("torch")

from paper_1801_05977_gb300 import gf

pytestmark = pytest.mark.gpu


def _time(pipe, iters, sink):
    best = None
    for i in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = gf.peak_probe(pipe, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        if i > 0:
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
    return fl, best


def test_probe_halves_and_both():
    sink = torch.zeros(2, dtype=torch.float64, device="cuda")
    f64, t64 = _time(gf.GF_PROBE_FP64_HALF, 200, sink)
    f32, t32 = _time(gf.GF_PROBE_FP32_HALF, 200, sink)
    fb, tb = _time(gf.GF_PROBE_BOTH_HALVES, 200, sink)
    assert f64 > 0 and f32 == f64 * gf.GF_PROBE_FP32_PER_FP64 and fb == f64 + f32
    print(f"probe halves: FP64 {t64:.3f} ms, FP32 {t32:.3f} ms, both {tb:.3f} ms")
    assert 0.9 * max(t64, t32) <= tb <= 1.1 * (t64 + t32)
