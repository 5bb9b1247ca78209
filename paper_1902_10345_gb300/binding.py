"""Thin ctypes binding over libsdfgjacobi.so.

Every function here only marshals arguments: the work happens in the
library's CUDA kernels.  The functions named ``sdfg_*`` mirror the C ABI in
``include/sdfg_jacobi.h`` one to one (raw integers for pointers and streams);
the short helpers below them accept torch tensors and pass their data
pointers, shapes and the current CUDA stream.

``lib()`` raises if the shared library has not been built: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

# ---- constants mirrored from the header --------------------------------------
SDFG_F32, SDFG_BF16, SDFG_F64 = 0, 1, 2
SDFG_OK, SDFG_PENDING, SDFG_PAUSED = 0, 1, 2
SDFG_ERR_INVAL, SDFG_ERR_NOMEM, SDFG_ERR_CUDA, SDFG_ERR_TIMEOUT, SDFG_ERR_BUSY, SDFG_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
SDFG_KERNEL_AUTO, SDFG_KERNEL_NAIVE, SDFG_KERNEL_TEMPORAL, SDFG_KERNEL_PERSISTENT, SDFG_KERNEL_RESIDENT = 0, 1, 2, 3, 4
SDFG_KERNEL_SKEWED = 5

STATUS_NAMES = {0: "OK", 1: "PENDING", 2: "PAUSED", -1: "ERR_INVAL", -2: "ERR_NOMEM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT",
                -5: "ERR_BUSY", -6: "ERR_UNSUPPORTED"}


class SdfgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class sdfg_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("k", ctypes.c_int), ("seg_rows", ctypes.c_int), ("warps", ctypes.c_int)]


class sdfg_desc(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("ld", ctypes.c_int), ("T", ctypes.c_int), ("tol", ctypes.c_double), ("dtype", ctypes.c_int),
                ("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("t_start", ctypes.c_int), ("priority", ctypes.c_int), ("r_first2", ctypes.c_double)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_PROTOS = {
    "sdfg_jacobi2d": (_I, [_VP, _VP, _I, _I, _I, _VP]),
    "sdfg_jacobi2d_ex": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _VP]),
    "sdfg_jacobi2d_cfg": (_I, [_VP, _VP, _I, _I, _I, _I, _I, ctypes.POINTER(sdfg_config), _VP]),
    "sdfg_jacobi2d_host": (_I, [_VP, _VP, _I, _I, _I, _I, _VP]),
    "sdfg_jacobi2d_host_many": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _VP]),
    "sdfg_jacobi2d_noalloc": (_I, [_VP, _VP, _I, _I, _I, _VP]),
    "sdfg_jacobi2d_solve": (_I, [ctypes.POINTER(sdfg_desc), _I, ctypes.POINTER(sdfg_config), _VP]),
    "sdfg_jacobi2d_batch": (_I, [ctypes.POINTER(sdfg_desc), _I, _I, _VP]),
    "sdfg_batch_plan_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(sdfg_desc), _I, _I,
                                    ctypes.POINTER(sdfg_config), _VP]),
    "sdfg_batch_plan_run": (_I, [_VP, _VP]),
    "sdfg_batch_plan_results": (_I, [_VP, ctypes.POINTER(sdfg_desc), _I]),
    "sdfg_batch_plan_destroy": (_I, [_VP]),
    "sdfg_server_create": (_I, [ctypes.POINTER(_VP), ctypes.c_size_t, _I, _I, _I, _I]),
    "sdfg_server_set_config": (_I, [_VP, ctypes.POINTER(sdfg_config)]),
    "sdfg_server_submit": (_I, [_VP, ctypes.POINTER(sdfg_desc), ctypes.POINTER(ctypes.c_uint64)]),
    "sdfg_server_poll": (_I, [_VP, ctypes.c_uint64, ctypes.POINTER(sdfg_desc)]),
    "sdfg_server_drain": (_I, [_VP, _I]),
    "sdfg_server_snapshot": (_I, [_VP, ctypes.c_uint64]),
    "sdfg_server_destroy": (_I, [_VP]),
    "sdfg_laplace1d": (_I, [_VP, _I, _I, _VP]),
    "sdfg_jacobi3d": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _I, _VP]),
    "sdfg_sor2d": (_I, [_VP, _VP, _I, _I, _I, _I, ctypes.c_double, _I, _VP]),
    "sdfg_autotune": (_I, [_I, _I, _I, _I, ctypes.POINTER(sdfg_config), _VP]),
    "sdfg_autotune_batch": (_I, [ctypes.POINTER(sdfg_desc), _I, _I, ctypes.POINTER(sdfg_config), _VP]),
    "sdfg_stats_enable": (_I, [_I]),
    "sdfg_stats_reset": (_I, []),
    "sdfg_stats_get": (_I, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    "sdfg_device_error": (_I, [_I]),
    "sdfg_last_error": (ctypes.c_char_p, []),
    "sdfg_version": (_I, []),
    "sdfg_test_hook": (_I, [_I, ctypes.c_longlong]),
    "sdfg_plan_geometry": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_int)]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libsdfgjacobi.so (it must have been built: see ``build.build``)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                path = library_path()
                if not os.path.exists(path):
                    raise ImportError(f"libsdfgjacobi.so is not built ({path}); run paper_1902_10345_gb300.build.build()")
                L = ctypes.CDLL(path)
                for name, (res, args) in _PROTOS.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = L
    return _lib


def last_error() -> str:
    m = lib().sdfg_last_error()
    return m.decode() if m else ""


def check(rc: int) -> int:
    if rc < 0:
        raise SdfgError(rc, last_error())
    return rc


# ---- raw C-ABI mirrors ---------------------------------------------------------
def sdfg_jacobi2d(inp: int, out: int, rows: int, cols: int, T: int, stream: int = 0) -> int:
    return lib().sdfg_jacobi2d(inp, out, rows, cols, T, stream)


def sdfg_jacobi2d_ex(inp, out, rows, cols, ld, T, dtype, stream=0) -> int:
    return lib().sdfg_jacobi2d_ex(inp, out, rows, cols, ld, T, dtype, stream)


def sdfg_jacobi2d_cfg(inp, out, rows, cols, ld, T, dtype, cfg: sdfg_config | None, stream=0) -> int:
    return lib().sdfg_jacobi2d_cfg(inp, out, rows, cols, ld, T, dtype, ctypes.byref(cfg) if cfg else None, stream)


def sdfg_jacobi2d_noalloc(inp: int, out: int, rows: int, cols: int, T: int, stream: int = 0) -> int:
    return lib().sdfg_jacobi2d_noalloc(inp, out, rows, cols, T, stream)


def sdfg_jacobi2d_host(h_in, h_out, rows, cols, T, dtype, stream=0) -> int:
    return lib().sdfg_jacobi2d_host(h_in, h_out, rows, cols, T, dtype, stream)


def sdfg_jacobi2d_host_many(h_ins, h_outs, rows, cols, T, dtype, stream=0) -> int:
    """h_ins, h_outs: sequences of host addresses (ints) of equal length."""
    n = len(h_ins)
    if len(h_outs) != n:
        raise ValueError("h_ins and h_outs differ in length")
    ins = (ctypes.c_void_p * max(n, 1))(*h_ins)
    outs = (ctypes.c_void_p * max(n, 1))(*h_outs)
    return lib().sdfg_jacobi2d_host_many(ctypes.cast(ins, ctypes.c_void_p), ctypes.cast(outs, ctypes.c_void_p), n,
                                         rows, cols, T, dtype, stream)


def sdfg_jacobi2d_solve(desc: sdfg_desc, check_stride: int, cfg: sdfg_config | None = None, stream=0) -> int:
    return lib().sdfg_jacobi2d_solve(ctypes.byref(desc), check_stride, ctypes.byref(cfg) if cfg else None, stream)


def _write_back(descs, arr):
    """Copy the output fields of `arr` into the caller's descriptor objects."""
    for d, r in zip(descs, arr):
        d.status, d.steps_done, d.rel_residual, d.r_first2 = r.status, r.steps_done, r.rel_residual, r.r_first2


def sdfg_jacobi2d_batch(descs, check_stride: int, stream=0) -> int:
    arr = (sdfg_desc * len(descs))(*descs)
    rc = lib().sdfg_jacobi2d_batch(arr, len(descs), check_stride, stream)
    _write_back(descs, arr)
    return rc


def sdfg_laplace1d(A: int, N: int, T: int, stream: int = 0) -> int:
    return lib().sdfg_laplace1d(A, N, T, stream)


def sdfg_jacobi3d(inp: int, out: int, D: int, R: int, C: int, ld: int, T: int, dtype: int, stream: int = 0) -> int:
    return lib().sdfg_jacobi3d(inp, out, D, R, C, ld, T, dtype, stream)


def sdfg_autotune(rows, cols, T, dtype, stream=0) -> sdfg_config:
    c = sdfg_config()
    check(lib().sdfg_autotune(rows, cols, T, dtype, ctypes.byref(c), stream))
    return c


def sdfg_autotune_batch(descs, check_stride: int, stream=0) -> sdfg_config:
    arr = (sdfg_desc * len(descs))(*descs)
    c = sdfg_config()
    check(lib().sdfg_autotune_batch(arr, len(descs), check_stride, ctypes.byref(c), stream))
    return c


def sdfg_stats_enable(on: bool) -> int:
    return lib().sdfg_stats_enable(1 if on else 0)


def sdfg_stats_reset() -> int:
    return lib().sdfg_stats_reset()


def sdfg_stats_get(name: str):
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    check(lib().sdfg_stats_get(name.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def sdfg_device_error(clear: bool = True) -> int:
    return lib().sdfg_device_error(1 if clear else 0)


def sdfg_test_hook(hook: int, value: int) -> int:
    return lib().sdfg_test_hook(hook, value)


def sdfg_version() -> int:
    return lib().sdfg_version()


def sdfg_plan_geometry(rows, cols, dtype, k, seg_rows=0):
    info = (ctypes.c_int * 8)()
    check(lib().sdfg_plan_geometry(rows, cols, dtype, k, seg_rows, info))
    keys = ["halo_cols", "warp_cols", "out_cols_per_strip", "n_strips", "seg_rows", "n_segs", "chunk_rows", "stages"]
    return dict(zip(keys, list(info)))


# ---- torch helpers ----------------------------------------------------------------
def dtype_code(t) -> int:
    import torch
    return {torch.float32: SDFG_F32, torch.bfloat16: SDFG_BF16, torch.float64: SDFG_F64}[t.dtype]


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _grid_args(t):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("grid must be a 2-D tensor with unit column stride")
    return t.data_ptr(), t.shape[0], t.shape[1], t.stride(0)


def config(kernel=SDFG_KERNEL_AUTO, k=0, seg_rows=0, warps=0) -> sdfg_config:
    return sdfg_config(kernel, k, seg_rows, warps)


def jacobi2d(inp, out, T: int, cfg: sdfg_config | None = None, stream=None) -> None:
    """out <- inp after T timesteps (device tensors of equal shape/dtype; may be the same)."""
    pi, R, C, ld = _grid_args(inp)
    po, R2, C2, ld2 = _grid_args(out)
    if (R, C, ld) != (R2, C2, ld2) or inp.dtype != out.dtype:
        raise ValueError("in and out must have the same shape, pitch and dtype")
    check(sdfg_jacobi2d_cfg(pi, po, R, C, ld, T, dtype_code(inp), cfg, _stream(stream)))


def _box_args(t):
    """(pointer, depth, rows, cols, ld) of a 3-D tensor whose planes are rows * ld apart."""
    if t.dim() != 3 or t.stride(2) != 1 or t.stride(0) != t.shape[1] * t.stride(1):
        raise ValueError("box must be a 3-D tensor with unit column stride and planes rows * ld apart")
    return t.data_ptr(), t.shape[0], t.shape[1], t.shape[2], t.stride(1)


def jacobi3d(inp, out, T: int, stream=None) -> None:
    """out <- inp after T timesteps of the 7-point stencil (device tensors of
    equal shape, pitch and dtype; may be the same)."""
    pi, D, R, C, ld = _box_args(inp)
    po, D2, R2, C2, ld2 = _box_args(out)
    if (D, R, C, ld) != (D2, R2, C2, ld2) or inp.dtype != out.dtype:
        raise ValueError("in and out must have the same shape, pitch and dtype")
    check(sdfg_jacobi3d(pi, po, D, R, C, ld, T, dtype_code(inp), _stream(stream)))


def sor2d(inp, out, T: int, omega: float, stream=None) -> None:
    """out <- inp after T red-black SOR iterations with relaxation omega
    (device tensors of equal shape, pitch and dtype; may be the same)."""
    pi, R, C, ld = _grid_args(inp)
    po, R2, C2, ld2 = _grid_args(out)
    if (R, C, ld) != (R2, C2, ld2) or inp.dtype != out.dtype:
        raise ValueError("in and out must have the same shape, pitch and dtype")
    check(lib().sdfg_sor2d(pi, po, R, C, ld, T, float(omega), dtype_code(inp), _stream(stream)))


def desc_for(inp, out, T: int, tol: float = 0.0, t_start: int = 0, r_first2: float = 0.0,
             priority: int = 0) -> sdfg_desc:
    pi, R, C, ld = _grid_args(inp)
    po, _, _, _ = _grid_args(out)
    return sdfg_desc(pi, po, R, C, ld, T, tol, dtype_code(inp), 0, 0, 0.0, t_start, priority, r_first2)
