"""The Python binding has no CPU fallback.

Every step of the method runs in the CUDA library; when the library is
absent and cannot be built (no nvcc), each public entry point must raise
rather than return anything computed another way.  The library is made
absent by pointing the build module at an empty directory and refusing the
build, as on a machine without the CUDA toolkit.
"""
import numpy as np
import pytest

from paper_1801_05977_gb300 import build as _build
from paper_1801_05977_gb300 import gf


@pytest.fixture
def no_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gf, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libgf.so"))
    monkeypatch.setattr(_build, "up_to_date", lambda: False)

    def refuse(*args, **kwargs):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")

    monkeypatch.setattr(_build, "build", refuse)


def test_library_load_raises(no_library):
    with pytest.raises(RuntimeError, match="not found"):
        gf.lib(build_if_missing=False)
    with pytest.raises(RuntimeError, match="nvcc"):
        gf.lib()


@pytest.mark.parametrize("call", [
    lambda: gf.trunc_default(),
    lambda: gf.launch_count(),
    lambda: gf.set_phase_timing(True),
    lambda: gf.release_memory(),
    lambda: gf.Plan(3, 2.5, (0.1, 0.3), (16, 16, 8)),
    lambda: gf.Plan(2, 1.3, (0.2,), (64, 64)),
    lambda: gf.Batch(np.array([2.5]), np.array([[0.1, 0.3]]), np.array([[16, 16, 8]])),
    lambda: gf.MLP(seed=0),
    lambda: gf.MLP.param_count(),
], ids=["trunc_default", "launch_count", "set_phase_timing", "release_memory", "plan_3d", "plan_2d",
        "batch", "mlp", "mlp_param_count"])
def test_every_entry_point_raises(no_library, call):
    with pytest.raises(RuntimeError):
        call()
