"""Pins of the FP64 3-D oracle (7-point Jacobi stencil, weight 1/7, fixed
one-cell shell) to facts that do not come from the oracle itself:

* hand-computed 4x4x4 / 3x3x3 fixtures in exact rationals
  (tests/golden/hand_4x4x4.json);
* closed-form eigenmodes of the zero-shell problem on boxes with three
  different extents, so that a mixed-up axis or stride changes the answer;
* discrete-harmonic fixed points in index coordinates;
* the discrete maximum principle (positive weights summing to one);
* symmetries: reflecting any axis and transposing rows with columns commute
  with a step bit for bit (the summation order pairs n+s, w+e, u+d);
* semigroup (run T1 then T2 equals run T1+T2, bit for bit), thread-count
  invariance, the light-cone window, degenerate boxes.

Every pin takes the oracle library as an argument so that the mutation tests
can run it against a copy with a planted mistake.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def lib():
    oracle.build()
    return oracle._get3d()


def run(lib, box, T, threads=1):
    return oracle.jacobi3d(box, T, threads=threads, lib=lib)


# ------------------------------------------------------------------ pins -----
def pin_hand_fixtures(lib):
    with open(os.path.join(HERE, "golden", "hand_4x4x4.json")) as f:
        doc = json.load(f)
    for case in doc["cases"]:
        box = np.array(case["box"], dtype=np.float64)
        for e in case["expect"]:
            got = run(lib, box, e["T"])
            want = np.array([[[float(Fraction(v)) for v in row] for row in plane] for plane in e["interior"]])
            n = box.shape[0]
            inner = got[1:n - 1, 1:n - 1, 1:n - 1]
            assert inner.shape == want.shape
            assert np.abs(inner - want).max() <= 8 * e["T"] * EPS, (case["name"], e["T"])
            # the shell is never written
            shell = np.ones(box.shape, bool)
            shell[1:n - 1, 1:n - 1, 1:n - 1] = False
            assert np.array_equal(got[shell], box[shell]), case["name"]


def _mode(shape, a, b, c):
    D, R, C = shape
    z = np.arange(D)[:, None, None]
    i = np.arange(R)[None, :, None]
    j = np.arange(C)[None, None, :]
    u = np.sin(a * np.pi * z / (D - 1)) * np.sin(b * np.pi * i / (R - 1)) * np.sin(c * np.pi * j / (C - 1))
    lam = (1 + 2 * np.cos(a * np.pi / (D - 1)) + 2 * np.cos(b * np.pi / (R - 1)) + 2 * np.cos(c * np.pi / (C - 1))) / 7
    # the shell of a sine mode is zero up to rounding; make it exactly zero
    u[0], u[-1], u[:, 0], u[:, -1], u[:, :, 0], u[:, :, -1] = 0, 0, 0, 0, 0, 0
    return u, lam


def pin_eigenmodes(lib):
    for shape, modes in [((7, 9, 12), [(1, 1, 1), (2, 3, 1), (5, 1, 7)]),
                         ((5, 16, 6), [(1, 2, 3), (3, 14, 4)]),
                         ((12, 5, 9), [(10, 3, 2)])]:
        for a, b, c in modes:
            u, lam = _mode(shape, a, b, c)
            for T in (1, 5, 23):
                got = run(lib, u, T)
                want = lam ** T * u
                assert np.abs(got - want).max() <= 16 * (T + 1) * EPS, (shape, (a, b, c), T)


def pin_harmonic_fixed_points(lib):
    D, R, C = 6, 7, 9
    z, i, j = np.meshgrid(np.arange(D, dtype=float), np.arange(R, dtype=float), np.arange(C, dtype=float),
                          indexing="ij")
    fields = {"const": np.full((D, R, C), 0.75), "linear": 0.5 + 0.25 * z - 0.125 * i + 0.0625 * j,
              "i2-j2": i * i - j * j, "i2+j2-2z2": i * i + j * j - 2 * z * z, "ij": i * j, "iz": i * z,
              "jz": j * z, "ijz": i * j * z}
    for name, f in fields.items():
        got = run(lib, f, 12)
        scale = max(1.0, np.abs(f).max())
        assert np.abs(got - f).max() <= 64 * EPS * scale, name


def pin_maximum_principle(lib):
    rng = np.random.default_rng(3)
    box = rng.random((9, 10, 11))
    lo, hi = box.min(), box.max()
    for T in (1, 7, 40):
        got = run(lib, box, T)
        assert got.min() >= lo - 8 * EPS and got.max() <= hi + 8 * EPS, T
        # strictly inside after a step: interior values average positive weights
        assert np.all(got[1:-1, 1:-1, 1:-1] > lo) and np.all(got[1:-1, 1:-1, 1:-1] < hi)


def pin_symmetries(lib):
    rng = np.random.default_rng(5)
    box = rng.random((8, 11, 11))
    T = 9
    ref = run(lib, box, T)
    for ax in range(3):
        flipped = run(lib, np.flip(box, axis=ax).copy(), T)
        assert np.array_equal(np.flip(flipped, axis=ax), ref), f"reflection of axis {ax}"
    tr = run(lib, np.ascontiguousarray(box.transpose(0, 2, 1)), T)
    assert np.array_equal(tr.transpose(0, 2, 1), ref), "transpose rows/cols"
    cube = rng.random((9, 9, 9))
    refc = run(lib, cube, T)
    perm = run(lib, np.ascontiguousarray(cube.transpose(1, 0, 2)), T)
    assert np.abs(perm.transpose(1, 0, 2) - refc).max() <= 16 * T * EPS, "planes/rows permutation"


def pin_semigroup(lib):
    rng = np.random.default_rng(7)
    box = rng.random((6, 13, 10))
    a = run(lib, run(lib, box, 5), 8)
    b = run(lib, box, 13)
    assert np.array_equal(a, b)


def pin_exact_rational_bruteforce(lib):
    """Exact rational evaluation of the definition on a tiny random box; the
    FP64 oracle must agree to a few ulps per step."""
    rng = np.random.default_rng(9)
    box = rng.integers(0, 16, size=(4, 5, 4)).astype(np.float64) / 16
    D, R, C = box.shape
    A = [[[Fraction(x).limit_denominator(1 << 20) for x in row] for row in plane] for plane in box]
    T = 4
    for _ in range(T):
        B = [[list(row) for row in plane] for plane in A]
        for z in range(1, D - 1):
            for i in range(1, R - 1):
                for j in range(1, C - 1):
                    s = A[z][i][j] + A[z][i - 1][j] + A[z][i + 1][j] + A[z][i][j - 1] + A[z][i][j + 1] + \
                        A[z - 1][i][j] + A[z + 1][i][j]
                    B[z][i][j] = s / 7
        A = B
    want = np.array([[[float(x) for x in row] for row in plane] for plane in A])
    got = run(lib, box, T)
    assert np.abs(got - want).max() <= 8 * T * EPS


ALL_PINS = [pin_hand_fixtures, pin_eigenmodes, pin_harmonic_fixed_points, pin_maximum_principle, pin_symmetries,
            pin_semigroup, pin_exact_rational_bruteforce]


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, lib):
    pin(lib)


# ------------------------------------------------------------ properties -----
def test_thread_count_invariance(lib):
    rng = np.random.default_rng(11)
    box = rng.random((20, 17, 15))
    one = run(lib, box, 6, threads=1)
    for th in (2, 3, 0):
        assert np.array_equal(run(lib, box, 6, threads=th), one)


def test_light_cone_window(lib):
    rng = np.random.default_rng(13)
    box = rng.random((16, 18, 20))
    T = 3
    full = run(lib, box, T)
    lo, hi = (5, 2, 9), (9, 7, 14)
    win = oracle.jacobi3d_window(box, T, lo, hi, lib=lib)
    assert np.array_equal(win, full[5:9, 2:7, 9:14])
    # a window touching the shell
    win = oracle.jacobi3d_window(box, T, (0, 0, 0), (4, 4, 4), lib=lib)
    assert np.array_equal(win, full[:4, :4, :4])


@pytest.mark.parametrize("shape", [(2, 5, 5), (5, 2, 5), (5, 5, 1), (0, 3, 3), (3, 3, 3)])
def test_degenerate_boxes(lib, shape):
    rng = np.random.default_rng(17)
    box = rng.random(shape)
    got = run(lib, box, 4)
    if min(shape) < 3:
        assert np.array_equal(got, box)
    else:
        assert got.shape == box.shape
    assert np.array_equal(run(lib, box, 0), box)


def test_invalid_arguments(lib):
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.oracle_jacobi3d(dp(), dp(), -1, 3, 3, 1, 1) != 0
    assert lib.oracle_jacobi3d(dp(), dp(), 3, 3, 3, -1, 1) != 0
    assert lib.oracle_jacobi3d(dp(), dp(), 3, 3, 3, 1, 1) != 0  # null arrays for a non-empty box
