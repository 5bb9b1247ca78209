"""FP64 CPU oracles for the iterated Jacobi stencils (2-D 5-point, 3-D 7-point)
and the 1-D Laplace program of the paper's Fig. 1.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  The CUDA library never calls it, and the two share no code:
this wrapper loads ``jacobi2d_oracle.c``, ``jacobi3d_oracle.c`` and
``sor2d_oracle.c``, each
compiled by gcc with ``-O2 -ffp-contract=off`` (no fast-math), nothing else.

``laplace1d`` is the 1-D Laplace program printed in the paper's Fig. 1.
``sor2d`` is the in-place, ordered counterpart: red-black successive
over-relaxation of the same 2-D Laplace problem (``sor2d_oracle.c``).
``jacobi3d`` is the same method as the 2-D Jacobi stencil one dimension up
(7 points, weight 1/7 each, fixed one-cell shell); the C file's header gives
the formula and its readings.

What it computes is the plain definition (paper Sec. 6.1, Jacobi stencil;
Fig. 1 for the ping-pong state loop; Sec. 3 "State" for the data-dependent
stop condition); the C file's header spells out the formula and each reading
of a point the paper leaves open.

``jacobi2d_window`` adds one more exact use of the definition: one timestep
moves information by one cell, so the grid after T steps inside a window
depends only on the input within distance T of it.  Running the definition on
a crop that extends T+1 cells past the window (clamped to the grid) therefore
gives the window's values exactly, whatever the crop's artificial edge does.

Parity status: the 2-D functions are pinned by ``tests/test_oracle_pins.py``
(hand-computed 4x4 fixtures, exact rational brute force, closed-form
eigenmodes, harmonic fixed points, maximum principle, symmetries, semigroup,
thread-count invariance, closed-form stopping step), ``laplace1d`` by
``tests/test_oracle_laplace1d.py`` and ``jacobi3d`` by
``tests/test_oracle_jacobi3d.py`` (hand-computed 4x4x4 fixtures, closed-form
eigenmodes, harmonic fixed points, maximum principle, symmetries, semigroup,
thread-count invariance) and ``sor2d`` by ``tests/test_oracle_sor2d.py``
(hand-computed sweeps, Young's convergence rates for red-black ordering,
harmonic fixed points, exact rationals, symmetry); mutation tests plant
mistakes in a copy of each C source and check that the pins catch them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi2d_oracle.c")
_SRC3D = os.path.join(_HERE, "jacobi3d_oracle.c")
_SRCSOR = os.path.join(_HERE, "sor2d_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_LIB3D_PATH = os.path.join(_BUILD_DIR, "liboracle3d.so")
_LIBSOR_PATH = os.path.join(_BUILD_DIR, "liboraclesor.so")
_lock = threading.Lock()
_lib = None
_lib3d = None
_libsor = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c99"]


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source file to a shared object with the oracle's flags."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build liboracle.so, liboracle3d.so and liboraclesor.so (each only if
    missing or older than its source); returns the 2-D library's path."""
    with _lock:
        for src, lib in ((_SRC, _LIB_PATH), (_SRC3D, _LIB3D_PATH), (_SRCSOR, _LIBSOR_PATH)):
            if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
                compile_source(src, lib)
    return _LIB_PATH


def load_library3d(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_jacobi3d.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_int]
    lib.oracle_jacobi3d.restype = ctypes.c_int
    return lib


def load_library(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_long)
    lib.oracle_jacobi2d.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_int]
    lib.oracle_jacobi2d.restype = ctypes.c_int
    lib.oracle_jacobi2d_tol.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double,
                                        ctypes.c_long, ctypes.c_int, lp, dp, dp]
    lib.oracle_jacobi2d_tol.restype = ctypes.c_int
    lib.oracle_laplace1d.argtypes = [dp, ctypes.c_long, ctypes.c_long]
    lib.oracle_laplace1d.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _get():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def load_library_sor(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_sor2d.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double]
    lib.oracle_sor2d.restype = ctypes.c_int
    return lib


def _getsor():
    global _libsor
    if _libsor is None:
        build()
        _libsor = load_library_sor(_LIBSOR_PATH)
    return _libsor


def _get3d():
    global _lib3d
    if _lib3d is None:
        build()
        _lib3d = load_library3d(_LIB3D_PATH)
    return _lib3d


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_f64(grid) -> np.ndarray:
    g = np.ascontiguousarray(np.asarray(grid, dtype=np.float64))
    if g.ndim != 2:
        raise ValueError("grid must be 2-D")
    return g


def num_threads(threads: int = 0, lib=None) -> int:
    """Threads the oracle uses for ``threads`` (0 = OpenMP default)."""
    return int((lib or _get()).oracle_num_threads(int(threads)))


def jacobi2d(grid, T: int, threads: int = 1, lib=None) -> np.ndarray:
    """Grid after T timesteps (FP64; the input is converted to FP64 exactly)."""
    lib = lib or _get()
    a = _as_f64(grid)
    out = np.empty_like(a)
    rc = lib.oracle_jacobi2d(_dptr(a), _dptr(out), a.shape[0], a.shape[1], int(T), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_jacobi2d failed with status {rc}")
    return out


def jacobi2d_tol(grid, T_cap: int, tol: float, check_stride: int, threads: int = 1, lib=None):
    """Tolerance mode.  Returns (grid, steps_done, rel_residual, r_first)."""
    lib = lib or _get()
    a = _as_f64(grid)
    out = np.empty_like(a)
    steps = ctypes.c_long(0)
    rel = ctypes.c_double(0.0)
    r1 = ctypes.c_double(0.0)
    rc = lib.oracle_jacobi2d_tol(_dptr(a), _dptr(out), a.shape[0], a.shape[1], int(T_cap), float(tol),
                                 int(check_stride), int(threads), ctypes.byref(steps), ctypes.byref(rel),
                                 ctypes.byref(r1))
    if rc != 0:
        raise ValueError(f"oracle_jacobi2d_tol failed with status {rc}")
    return out, int(steps.value), float(rel.value), float(r1.value)


def laplace1d(A2, T: int, lib=None) -> np.ndarray:
    """The paper's Fig. 1 program on a copy of the float64[2, N] array A2:
    returns the array as the program leaves it after T steps."""
    lib = lib or _get()
    a = np.array(A2, dtype=np.float64, copy=True, order="C")
    if a.ndim != 2 or a.shape[0] != 2:
        raise ValueError("A must have shape (2, N)")
    rc = lib.oracle_laplace1d(_dptr(a), a.shape[1], int(T))
    if rc != 0:
        raise ValueError(f"oracle_laplace1d failed with status {rc}")
    return a


def jacobi2d_window(grid, T: int, r0: int, r1: int, c0: int, c1: int, threads: int = 1, lib=None) -> np.ndarray:
    """Rows r0:r1, cols c0:c1 of the grid after T steps, from a light-cone crop.

    A window cell at distance > T from the crop's artificial edge cannot be
    reached by anything the crop gets wrong, so the result is exact.
    """
    a = np.asarray(grid)
    R, C = a.shape
    if not (0 <= r0 <= r1 <= R and 0 <= c0 <= c1 <= C):
        raise ValueError("window out of range")
    m = int(T) + 1
    cr0, cr1 = max(0, r0 - m), min(R, r1 + m)
    cc0, cc1 = max(0, c0 - m), min(C, c1 + m)
    crop = jacobi2d(a[cr0:cr1, cc0:cc1], T, threads=threads, lib=lib)
    return crop[r0 - cr0:r1 - cr0, c0 - cc0:c1 - cc0]


def jacobi3d(box, T: int, threads: int = 1, lib=None) -> np.ndarray:
    """D x R x C box after T timesteps of the 7-point stencil (FP64; the input
    is converted to FP64 exactly).  threads 0 = the OpenMP default."""
    lib = lib or _get3d()
    a = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    if a.ndim != 3:
        raise ValueError("box must be 3-D")
    out = np.empty_like(a)
    rc = lib.oracle_jacobi3d(_dptr(a), _dptr(out), a.shape[0], a.shape[1], a.shape[2], int(T), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_jacobi3d failed with status {rc}")
    return out


def jacobi3d_window(box, T: int, lo, hi, threads: int = 1, lib=None) -> np.ndarray:
    """box[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] after T steps, from a
    light-cone crop that extends T+1 cells past the window along each axis
    (clamped to the box): exact, as in ``jacobi2d_window``."""
    a = np.asarray(box)
    m = int(T) + 1
    cl = [max(0, int(l) - m) for l in lo]
    ch = [min(n, int(h) + m) for n, h in zip(a.shape, hi)]
    for l, h, n in zip(lo, hi, a.shape):
        if not 0 <= l <= h <= n:
            raise ValueError("window out of range")
    crop = jacobi3d(a[cl[0]:ch[0], cl[1]:ch[1], cl[2]:ch[2]], T, threads=threads, lib=lib)
    return crop[lo[0] - cl[0]:hi[0] - cl[0], lo[1] - cl[1]:hi[1] - cl[1], lo[2] - cl[2]:hi[2] - cl[2]]


def sor2d(grid, T: int, omega: float, lib=None) -> np.ndarray:
    """Grid after T red-black SOR iterations with relaxation omega (FP64; the
    input is converted to FP64 exactly): red points (i + j even) first, then
    black, each updated in place from its four neighbours."""
    lib = lib or _getsor()
    a = _as_f64(grid)
    out = np.empty_like(a)
    rc = lib.oracle_sor2d(_dptr(a), _dptr(out), a.shape[0], a.shape[1], int(T), float(omega))
    if rc != 0:
        raise ValueError(f"oracle_sor2d failed with status {rc}")
    return out
