"""Pins of the FP64 red-black SOR oracle to facts that do not come from the
oracle itself:

* hand-computed sweeps in exact rationals (tests/golden/hand_sor_4x4.json),
  which also tell red-black order from a lexicographic sweep;
* Young's theory for consistently ordered matrices (red-black ordering of the
  5-point Laplacian is one): with mu the Jacobi spectral radius
  0.5 (cos(pi/(R-1)) + cos(pi/(C-1))), Gauss-Seidel contracts the error by
  mu^2 per iteration, and SOR with 1 < omega < omega_opt by lambda, the largest
  root of (lambda + omega - 1)^2 = lambda omega^2 mu^2;
* discrete-harmonic fixed points, for any omega;
* exact rational brute force of the sweep on tiny grids;
* transposing rows and columns commutes with an iteration bit for bit (the
  colour of a point is kept, and (n + s) + (w + e) only swaps its addends);
* degenerate shapes and T = 0 copy.

Every pin takes the oracle library as an argument so that the mutation tests
can run it against a copy with a planted mistake.
"""
import json
import math
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
    return oracle._getsor()


def run(lib, g, T, omega):
    return oracle.sor2d(g, T, omega, lib=lib)


def pin_hand_fixtures(lib):
    with open(os.path.join(HERE, "golden", "hand_sor_4x4.json")) as f:
        doc = json.load(f)
    for case in doc["cases"]:
        g = np.array(case["grid"], dtype=np.float64)
        omega = float(Fraction(case["omega"]))
        for e in case["expect"]:
            got = run(lib, g, e["T"], omega)
            want = np.array([[float(Fraction(v)) for v in row] for row in e["interior"]])
            n = g.shape[0]
            assert np.abs(got[1:n - 1, 1:n - 1] - want).max() <= 8 * e["T"] * EPS, (case["name"], e["T"])
            ring = np.ones(g.shape, bool)
            ring[1:n - 1, 1:n - 1] = False
            assert np.array_equal(got[ring], g[ring]), case["name"]


def _young_rate(mu, omega):
    if omega == 1.0:
        return mu * mu
    s = (omega * mu + math.sqrt(omega * omega * mu * mu - 4 * (omega - 1))) / 2
    return s * s


def pin_young_rates(lib):
    for (R, C), omega in [((10, 12), 1.0), ((10, 12), 1.3), ((9, 15), 0.7), ((13, 11), 1.45)]:
        mu = 0.5 * (math.cos(math.pi / (R - 1)) + math.cos(math.pi / (C - 1)))
        omega_opt = 2 / (1 + math.sqrt(1 - mu * mu))
        assert omega < omega_opt
        rho = _young_rate(mu, omega)
        g = np.zeros((R, C))
        g[1:-1, 1:-1] = np.random.default_rng(R * C).random((R - 2, C - 2)) + 0.5
        # iterate until the slowest mode dominates, then compare successive
        # error norms (the exact solution is zero)
        t0 = 300
        a = run(lib, g, t0, omega)
        b = run(lib, a, 1, omega)
        c = run(lib, b, 1, omega)
        r1 = np.linalg.norm(b) / np.linalg.norm(a)
        r2 = np.linalg.norm(c) / np.linalg.norm(b)
        assert abs(r1 - rho) <= 2e-4 * rho and abs(r2 - rho) <= 2e-4 * rho, ((R, C), omega, r1, r2, rho)


def pin_harmonic_fixed_points(lib):
    R, C = 9, 12
    i, j = np.meshgrid(np.arange(R, dtype=float), np.arange(C, dtype=float), indexing="ij")
    for name, f in {"const": np.full((R, C), 0.375), "linear": 0.5 + 0.25 * i - 0.125 * j, "i2-j2": i * i - j * j,
                    "ij": i * j, "cubic": i ** 3 - 3 * i * j * j}.items():
        for omega in (1.0, 1.6, 0.5):
            got = run(lib, f, 15, omega)
            assert np.abs(got - f).max() <= 64 * EPS * max(1.0, np.abs(f).max()), (name, omega)


def pin_exact_rationals(lib):
    rng = np.random.default_rng(21)
    g = rng.integers(0, 32, size=(6, 7)).astype(np.float64) / 32
    R, C = g.shape
    om = Fraction(5, 4)
    A = [[Fraction(x).limit_denominator(1 << 20) for x in row] for row in g]
    T = 5
    for _ in range(T):
        for colour in (0, 1):
            for i in range(1, R - 1):
                for j in range(1, C - 1):
                    if (i + j) % 2 == colour:
                        q = A[i - 1][j] + A[i + 1][j] + A[i][j - 1] + A[i][j + 1]
                        A[i][j] = (1 - om) * A[i][j] + om / 4 * q
    want = np.array([[float(x) for x in row] for row in A])
    got = run(lib, g, T, float(om))
    assert np.abs(got - want).max() <= 16 * T * EPS


def pin_transpose(lib):
    g = np.random.default_rng(23).random((11, 14))
    for omega in (1.0, 1.37):
        a = run(lib, g, 9, omega)
        b = run(lib, np.ascontiguousarray(g.T), 9, omega)
        assert np.array_equal(a.T, b), omega


ALL_PINS = [pin_hand_fixtures, pin_young_rates, pin_harmonic_fixed_points, pin_exact_rationals, pin_transpose]


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, lib):
    pin(lib)


@pytest.mark.parametrize("shape", [(2, 9), (9, 2), (0, 4), (3, 3)])
def test_degenerate_and_T0(lib, shape):
    g = np.random.default_rng(3).random(shape)
    if min(shape) < 3:
        assert np.array_equal(run(lib, g, 5, 1.2), g)
    assert np.array_equal(run(lib, g, 0, 1.2), g)


def test_semigroup(lib):
    g = np.random.default_rng(5).random((17, 19))
    assert np.array_equal(run(lib, run(lib, g, 4, 1.1), 6, 1.1), run(lib, g, 10, 1.1))


def test_invalid_arguments(lib):
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.oracle_sor2d(dp(), dp(), -1, 3, 1, 1.0) != 0
    assert lib.oracle_sor2d(dp(), dp(), 3, 3, -1, 1.0) != 0
    assert lib.oracle_sor2d(dp(), dp(), 3, 3, 1, 1.0) != 0
