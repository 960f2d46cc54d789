"""Thin ctypes binding of the C ABI in include/gf.h (argument marshalling only).

Every step of the method runs in the CUDA library (_build/libgf.so); torch is
used for device memory and streams.  There is no CPU fallback: if the library
is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GF_OK, GF_ERR_ARG, GF_ERR_WOOD, GF_ERR_RESONANCE, GF_ERR_NOMEM, GF_ERR_CUDA, GF_ERR_TIMEOUT, GF_ERR_UNSUPPORTED = range(8)
GF_FP64, GF_FP32_SPLIT = 0, 1
GF_HELMHOLTZ, GF_MAXWELL, GF_DERIV2D = 0, 1, 2
GF_PERTURB_CTILDE, GF_FAIL = 0, 1
GF_OUT_G, GF_OUT_GD, GF_OUT_MAXWELL6, GF_OUT_MAXWELL7, GF_OUT_LD, GF_OUT_GRAD, GF_OUT_HESSDIFF = 0, 1, 2, 3, 4, 5, 6
N_ENTRIES = {GF_OUT_G: 1, GF_OUT_GD: 1, GF_OUT_MAXWELL6: 6, GF_OUT_MAXWELL7: 7, GF_OUT_LD: 1, GF_OUT_GRAD: 3,
             GF_OUT_HESSDIFF: 3}


class GfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class Trunc(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("c_tilde", ctypes.c_double), ("eps", ctypes.c_double),
                ("series_tol", ctypes.c_double), ("quad_nodes", ctypes.c_int), ("precision", ctypes.c_int),
                ("kind", ctypes.c_int), ("resonance_policy", ctypes.c_int), ("far_grid_M", ctypes.c_int),
                ("far_grid_nz", ctypes.c_int), ("far_grid_zmax", ctypes.c_double), ("k2", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("M", ctypes.c_int * 3), ("nfields", ctypes.c_int),
                ("precision", ctypes.c_int), ("kind", ctypes.c_int), ("k", ctypes.c_double),
                ("alpha", ctypes.c_double * 2), ("c", ctypes.c_double), ("c_tilde", ctypes.c_double),
                ("eps", ctypes.c_double), ("series_tol", ctypes.c_double), ("quad_nodes", ctypes.c_int),
                ("series_n1_lo", ctypes.c_int), ("series_n1_hi", ctypes.c_int), ("series_n2_lo", ctypes.c_int),
                ("series_n2_hi", ctypes.c_int), ("grid_device_bytes", ctypes.c_size_t),
                ("far_grid_M", ctypes.c_int), ("far_grid_nz", ctypes.c_int), ("far_grid_zmax", ctypes.c_double),
                ("far_grid_device_bytes", ctypes.c_size_t), ("k2", ctypes.c_double)]


EXPORTS = ["gf_trunc_default", "gf_plan", "gf_eval_grid", "gf_grid_bytes", "gf_eval_points",
           "gf_eval_points_host", "gf_plan_get_info", "gf_destroy", "gf_status_string", "gf_last_error",
           "gf_launch_count", "gf_set_phase_timing", "gf_plan_phase_ms", "gf_eval_points_noalloc",
           "gf_plan_batch", "gf_batch_synthesize", "gf_batch_eval_points", "gf_batch_autotune",
           "gf_batch_get_tuning", "gf_batch_run_graph", "gf_batch_get_plan", "gf_batch_destroy",
           "gf_gemm_bf16", "gf_mlp_create", "gf_mlp_param_count", "gf_mlp_params", "gf_mlp_set_scale",
           "gf_mlp_forward", "gf_mlp_train_step", "gf_mlp_gradients", "gf_mlp_error_word", "gf_surrogate_eval",
           "gf_mlp_destroy", "gf_release_memory", "gf_peak_probe", "gf_surrogate_eval_residual",
           "gf_wait_selftest", "gf_plan_status"]

NOALLOC_MAX_TARGETS = 1 << 18

_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgf.so (building it first if needed and possible)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not found at {_build.LIB}; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    L.gf_trunc_default.argtypes = [ctypes.POINTER(Trunc)]
    L.gf_plan.argtypes = [i32, d, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(Trunc), vp, ctypes.POINTER(vp)]
    L.gf_eval_grid.argtypes = [vp, vp, sz, vp]
    L.gf_grid_bytes.argtypes = [vp]
    L.gf_grid_bytes.restype = sz
    L.gf_eval_points.argtypes = [vp, vp, i64, i32, vp, vp]
    L.gf_eval_points_host.argtypes = [vp, vp, i64, i32, vp, vp]
    L.gf_eval_points_noalloc.argtypes = [vp, vp, i64, i32, vp, vp]
    P = ctypes.POINTER
    L.gf_plan_batch.argtypes = [i32, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int), P(Trunc), vp, P(vp)]
    L.gf_batch_synthesize.argtypes = [vp, vp]
    for nm in ("gf_batch_eval_points", "gf_batch_autotune", "gf_batch_run_graph"):
        getattr(L, nm).argtypes = [vp, vp, P(ctypes.c_int64), i32, vp, vp]
    L.gf_batch_get_tuning.argtypes = [vp, P(ctypes.c_int)]
    L.gf_batch_get_plan.argtypes = [vp, i32, P(vp)]
    L.gf_batch_destroy.argtypes = [vp]
    L.gf_gemm_bf16.argtypes = [vp, i64, i32, vp, i64, i32, i32, i32, i32, vp, i64, i32, vp]
    L.gf_mlp_create.argtypes = [ctypes.c_uint64, d, P(vp)]
    L.gf_mlp_param_count.restype = i64
    L.gf_mlp_params.argtypes = [vp, vp, i64, i32]
    L.gf_mlp_set_scale.argtypes = [vp, d]
    L.gf_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    L.gf_mlp_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp]
    L.gf_mlp_gradients.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.gf_mlp_error_word.argtypes = [vp, P(ctypes.c_int)]
    L.gf_surrogate_eval.argtypes = [vp, i32, P(d), P(d), P(ctypes.c_int64), vp, vp, d, P(Trunc), P(ctypes.c_int), vp]
    L.gf_surrogate_eval_residual.argtypes = [vp, i32, P(d), P(d), P(ctypes.c_int64), vp, vp, vp, d, P(Trunc),
                                             P(ctypes.c_int), vp]
    L.gf_mlp_destroy.argtypes = [vp]
    L.gf_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.gf_destroy.argtypes = [vp]
    L.gf_status_string.argtypes = [i32]
    L.gf_status_string.restype = ctypes.c_char_p
    L.gf_last_error.restype = ctypes.c_char_p
    L.gf_launch_count.restype = i64
    L.gf_set_phase_timing.argtypes = [i32]
    L.gf_plan_phase_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.gf_release_memory.argtypes = []
    L.gf_peak_probe.argtypes = [i32, i64, vp, P(ctypes.c_int64), vp]
    L.gf_wait_selftest.argtypes = [i64, i32, vp]
    L.gf_plan_status.argtypes = [vp, vp]
    for name in ("gf_trunc_default", "gf_plan", "gf_eval_grid", "gf_eval_points", "gf_eval_points_host",
                 "gf_eval_points_noalloc", "gf_plan_batch", "gf_batch_synthesize", "gf_batch_eval_points",
                 "gf_batch_autotune", "gf_batch_get_tuning", "gf_batch_run_graph", "gf_batch_get_plan",
                 "gf_batch_destroy", "gf_gemm_bf16", "gf_mlp_create", "gf_mlp_params", "gf_mlp_set_scale",
                 "gf_mlp_forward", "gf_mlp_train_step", "gf_mlp_gradients", "gf_mlp_error_word",
                 "gf_surrogate_eval", "gf_mlp_destroy",
                 "gf_plan_get_info", "gf_destroy", "gf_set_phase_timing", "gf_plan_phase_ms", "gf_release_memory",
                 "gf_peak_probe", "gf_surrogate_eval_residual", "gf_wait_selftest", "gf_plan_status"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != GF_OK:
        L = lib(False)
        raise GfError(status, f"{L.gf_status_string(status).decode()}: {L.gf_last_error().decode()}")


def trunc_default(**kw) -> Trunc:
    t = Trunc()
    _check(lib().gf_trunc_default(ctypes.byref(t)))
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def launch_count() -> int:
    return int(lib().gf_launch_count())


def set_phase_timing(on: bool):
    _check(lib().gf_set_phase_timing(1 if on else 0))


GF_PROBE_FP64, GF_PROBE_FP32, GF_PROBE_FP64_HALF, GF_PROBE_FP32_HALF, GF_PROBE_BOTH_HALVES = 0, 1, 2, 3, 4
GF_PROBE_FP32_PER_FP64 = 64  # FP32 trips per FP64 trip in the overlap modes (gf.h)


def peak_probe(pipe: int, iters: int, sink, stream=None) -> int:
    """gf_peak_probe: enqueue one FMA-chain launch on the FP64 or FP32 pipe;
    returns its flop count (the caller times the launch)."""
    fl = ctypes.c_int64()
    _check(lib().gf_peak_probe(int(pipe), int(iters), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fl),
                               _stream_ptr(stream)))
    return int(fl.value)


def wait_selftest(polls: int, arrive: bool, stream=None) -> int:
    """gf_wait_selftest: the status of one bounded mbarrier wait (GF_ERR_TIMEOUT when
    nothing arrives and the poll limit runs out, GF_OK when it completes)."""
    return int(lib().gf_wait_selftest(int(polls), 1 if arrive else 0, _stream_ptr(stream)))


def release_memory():
    """gf_release_memory: hand the pool's unused device memory back to the driver."""
    _check(lib().gf_release_memory())


class Plan:
    """A prepared (k, alpha, grid) problem: gf_plan / gf_eval_grid / gf_eval_points."""

    def __init__(self, dim: int, k: float, alpha, M, trunc: Trunc | None = None, stream=None, **trunc_kw):
        L = lib()
        if trunc is None:
            trunc = trunc_default(**trunc_kw)
        al = (ctypes.c_double * 2)(*(list(alpha) + [0.0] * (2 - len(alpha))))
        mm = (ctypes.c_int * 3)(*(list(M) + [1] * (3 - len(M))))
        h = ctypes.c_void_p()
        _check(L.gf_plan(int(dim), float(k), al, mm, ctypes.byref(trunc), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.dim = dim
        self.info = self.get_info()

    def get_info(self) -> PlanInfo:
        info = PlanInfo()
        _check(lib().gf_plan_get_info(self._h, ctypes.byref(info)))
        return info

    @property
    def precision(self) -> int:
        return self.info.precision

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == GF_FP64 else torch.complex64

    def eval_grid(self, stream=None):
        """Remainder grid L_N in node order, shape (nfields, [M3,] M2, M1)."""
        import torch
        i = self.info
        shape = (i.nfields,) + tuple(int(m) for m in reversed(i.M[: self.dim]))
        out = torch.empty(shape, dtype=self.complex_dtype, device="cuda")
        nbytes = out.numel() * out.element_size()
        _check(lib().gf_eval_grid(self._h, ctypes.c_void_p(out.data_ptr()), nbytes, _stream_ptr(stream)))
        return out

    def _check_io(self, x, out, which: int):
        """The kernels write n * entries values of the plan's complex type into out
        and read n * dim doubles from x: refuse buffers that do not hold them."""
        import torch
        if which not in N_ENTRIES:
            raise GfError(GF_ERR_ARG, f"unknown output kind {which}")
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and x.dim() == 2
                and x.shape[1] == self.dim):
            raise GfError(GF_ERR_ARG, f"x must be a contiguous float64 CUDA tensor of shape (n, {self.dim})")
        if not (out.is_cuda and out.dtype == self.complex_dtype and out.is_contiguous()
                and tuple(out.shape) == (x.shape[0], N_ENTRIES[which]) and out.device == x.device):
            raise GfError(GF_ERR_ARG, f"out must be a contiguous {self.complex_dtype} tensor of shape "
                                      f"({x.shape[0]}, {N_ENTRIES[which]}) on {x.device}")

    def eval_points_into(self, x, out, which: int, stream=None):
        """x: float64 CUDA tensor (n, dim); out: complex CUDA tensor (n, entries)."""
        self._check_io(x, out, which)
        n = x.shape[0]
        _check(lib().gf_eval_points(self._h, ctypes.c_void_p(x.data_ptr()), n, int(which),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def eval_points_noalloc_into(self, x, out, which: int, stream=None):
        """gf_eval_points_noalloc: same result, fixed library scratch, no allocation."""
        self._check_io(x, out, which)
        n = x.shape[0]
        _check(lib().gf_eval_points_noalloc(self._h, ctypes.c_void_p(x.data_ptr()), n, int(which),
                                            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def eval_points(self, x, which: int, stream=None):
        import torch
        if which not in N_ENTRIES:
            raise GfError(GF_ERR_ARG, f"unknown output kind {which}")
        out = torch.empty((x.shape[0], N_ENTRIES[which]), dtype=self.complex_dtype, device=x.device)
        return self.eval_points_into(x, out, which, stream)

    def eval_points_host(self, x: np.ndarray, out: np.ndarray, which: int, stream=None):
        """Host buffers in and out (numpy or pinned torch CPU tensors)."""
        if which not in N_ENTRIES:
            raise GfError(GF_ERR_ARG, f"unknown output kind {which}")
        item = 16 if self.precision == GF_FP64 else 8
        if isinstance(x, np.ndarray):
            ok_x = x.dtype == np.float64 and x.flags.c_contiguous
        else:
            import torch
            ok_x = (not x.is_cuda) and x.dtype == torch.float64 and x.is_contiguous()
        if not (ok_x and x.ndim == 2 and x.shape[1] == self.dim):
            raise GfError(GF_ERR_ARG, f"x must be a contiguous float64 host array of shape (n, {self.dim})")
        obytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        ocont = out.flags.c_contiguous if isinstance(out, np.ndarray) else (out.is_contiguous() and not out.is_cuda)
        if not (ocont and obytes >= x.shape[0] * N_ENTRIES[which] * item):
            raise GfError(GF_ERR_ARG, "out must be a contiguous host buffer of n * entries complex values")
        xp = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
        op = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        n = x.shape[0]
        _check(lib().gf_eval_points_host(self._h, ctypes.c_void_p(xp), n, int(which), ctypes.c_void_p(op),
                                         _stream_ptr(stream)))
        return out

    def status(self, stream=None) -> int:
        """gf_plan_status: GF_OK, or GF_ERR_TIMEOUT if a bounded wait of the synthesis ran out."""
        return int(lib().gf_plan_status(self._h, _stream_ptr(stream)))

    def phase_ms(self):
        """(synthesis, far table, near kernel, far kernel) device ms of the latest run."""
        ms = (ctypes.c_float * 4)()
        _check(lib().gf_plan_phase_ms(self._h, ms))
        return tuple(float(v) for v in ms)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A sweep of 3D plans run as batched persistent launches (gf_plan_batch ...)."""

    def __init__(self, k, alpha, M, trunc: Trunc | None = None, stream=None, **trunc_kw):
        L = lib()
        if trunc is None:
            trunc = trunc_default(**trunc_kw)
        k = np.ascontiguousarray(k, dtype=np.float64)
        alpha = np.ascontiguousarray(alpha, dtype=np.float64).reshape(-1, 2)
        M = np.ascontiguousarray(M, dtype=np.int32).reshape(-1, 3)
        self.np = k.shape[0]
        assert alpha.shape[0] == self.np and M.shape[0] == self.np
        h = ctypes.c_void_p()
        _check(L.gf_plan_batch(self.np, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               M.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(trunc),
                               _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.precision = trunc.precision

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == GF_FP64 else torch.complex64

    def _off(self, offsets):
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        assert off.shape[0] == self.np + 1
        self._off_keep = off
        return off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def synthesize(self, stream=None):
        _check(lib().gf_batch_synthesize(self._h, _stream_ptr(stream)))

    def eval_points_into(self, x, offsets, out, which: int, stream=None):
        _check(lib().gf_batch_eval_points(self._h, ctypes.c_void_p(x.data_ptr()), self._off(offsets), int(which),
                                          ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def autotune(self, x, offsets, out, which: int, stream=None):
        _check(lib().gf_batch_autotune(self._h, ctypes.c_void_p(x.data_ptr()), self._off(offsets), int(which),
                                       ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        t = (ctypes.c_int * 3)()
        _check(lib().gf_batch_get_tuning(self._h, t))
        return tuple(t)

    def run_graph(self, x, offsets, out, which: int, stream=None):
        _check(lib().gf_batch_run_graph(self._h, ctypes.c_void_p(x.data_ptr()), self._off(offsets), int(which),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def plan_handle(self, i: int):
        h = ctypes.c_void_p()
        _check(lib().gf_batch_get_plan(self._h, int(i), ctypes.byref(h)))
        return h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_bf16(A, B, a_trans=False, b_trans=False, ksplit=1, stream=None):
    """C = A . B^T on the tensor cores: A (M, K) or its transpose (K, M), B (N, K)
    or its transpose (K, N), bf16 CUDA tensors; returns fp32 (M, N)."""
    import torch
    M = A.shape[1] if a_trans else A.shape[0]
    K = A.shape[0] if a_trans else A.shape[1]
    N = B.shape[1] if b_trans else B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().gf_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), int(a_trans), ctypes.c_void_p(B.data_ptr()),
                              B.stride(0), int(b_trans), M, N, K, ctypes.c_void_p(C.data_ptr()), C.stride(0),
                              int(ksplit), _stream_ptr(stream)))
    return C


class MLP:
    """The surrogate network (gf_mlp_*)."""

    def __init__(self, seed: int = 0, c_tilde: float = 1.0):
        h = ctypes.c_void_p()
        _check(lib().gf_mlp_create(ctypes.c_uint64(seed), float(c_tilde), ctypes.byref(h)))
        self._h = h
        self.scale = 1.0

    @staticmethod
    def param_count() -> int:
        return int(lib().gf_mlp_param_count())

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.param_count(), dtype=np.float32)
        _check(lib().gf_mlp_params(self._h, p.ctypes.data, p.size, 0))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().gf_mlp_params(self._h, p.ctypes.data, p.size, 1))

    def set_scale(self, s: float):
        _check(lib().gf_mlp_set_scale(self._h, float(s)))
        self.scale = s

    def forward(self, inp, stream=None):
        import torch
        out = torch.empty((inp.shape[0], 2), dtype=torch.float32, device=inp.device)
        _check(lib().gf_mlp_forward(self._h, ctypes.c_void_p(inp.data_ptr()), inp.shape[0],
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def train_step(self, inp, target, lr: float, loss=None, stream=None):
        _check(lib().gf_mlp_train_step(self._h, ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                       inp.shape[0], ctypes.c_float(lr),
                                       ctypes.c_void_p(loss.data_ptr()) if loss is not None else None,
                                       _stream_ptr(stream)))

    def gradients(self, inp, target, stream=None):
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().gf_mlp_gradients(self._h, ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                      inp.shape[0], g.ctypes.data, ctypes.byref(loss), _stream_ptr(stream)))
        return g, loss.value

    def error_word(self) -> int:
        v = ctypes.c_int()
        lib().gf_mlp_error_word(self._h, ctypes.byref(v))
        return v.value

    def surrogate_eval(self, k, alpha, offsets, x, wood_delta=1e-2, trunc=None, stream=None, base=None):
        """gf_surrogate_eval, or gf_surrogate_eval_residual when `base` (complex128 CUDA
        tensor of the coarse remainder at the targets) is given."""
        import torch
        k = np.ascontiguousarray(k, dtype=np.float64)
        alpha = np.ascontiguousarray(alpha, dtype=np.float64).reshape(-1, 2)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if off.shape[0] != k.shape[0] + 1 or alpha.shape[0] != k.shape[0] or off[-1] != x.shape[0]:
            raise GfError(GF_ERR_ARG, "k, alpha and offsets must describe the rows of x")
        out = torch.empty((x.shape[0],), dtype=torch.complex128, device=x.device)
        nfb = ctypes.c_int()
        if trunc is None:
            trunc = trunc_default()
        args = (self._h, k.shape[0], k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.c_void_p(x.data_ptr()))
        tail = (ctypes.c_void_p(out.data_ptr()), float(wood_delta), ctypes.byref(trunc), ctypes.byref(nfb),
                _stream_ptr(stream))
        if base is None:
            _check(lib().gf_surrogate_eval(*args, *tail))
        else:
            if not (base.is_cuda and base.dtype == torch.complex128 and base.is_contiguous()
                    and base.numel() == x.shape[0]):
                raise GfError(GF_ERR_ARG, "base must be a contiguous complex128 CUDA tensor with one value per target")
            _check(lib().gf_surrogate_eval_residual(*args, ctypes.c_void_p(base.data_ptr()), *tail))
        return out, nfb.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
