"""Pins for the FP64 oracle: checks against what the definition and the
mathematics fix, none of which re-types the oracle's own loop.

* hand-computed 4x4 / 3x3 fixtures (tests/golden/hand_4x4.json);
* exact rational brute force on tiny grids (fractions.Fraction);
* closed-form eigenmodes of the zero-boundary problem (the paper's Sec. 6.1
  workload has a zero boundary): sin(p pi i/(R-1)) sin(q pi j/(C-1)) decays by
  exactly lambda = 0.2 + 0.4 (cos(p pi/(R-1)) + cos(q pi/(C-1))) per step;
* harmonic fixed points (degree <= 3 harmonic polynomials are exact zeros of
  the 5-point Laplacian);
* discrete maximum principle, transpose / reflection symmetry (bitwise),
  semigroup (bitwise), thread-count invariance (bitwise), linearity;
* closed-form stopping step of the tolerance mode on an eigenmode:
  A_t - A_{t-1} = lambda^(t-1) (lambda - 1) mode, so rel_t = |lambda|^(t-1);
* light-cone windows equal the full run.

Each pin is a function of the loaded library, so ``test_oracle_mutants``
can run the same pins against copies of the oracle with planted mistakes and
check that every mistake is caught.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1902_10345_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- pins ----------

def pin_hand_fixtures(lib):
    with open(os.path.join(HERE, "golden", "hand_4x4.json")) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        g = np.array(case["grid"], dtype=np.float64)
        for e in case["expect"]:
            out = oracle.jacobi2d(g, e["T"], lib=lib)
            want = np.array([[float(Fraction(v)) for v in row] for row in e["interior"]])
            got = out[1:-1, 1:-1]
            assert np.allclose(got, want, rtol=0, atol=16 * EPS * e["T"]), (case["name"], e["T"], got, want)
            ring = np.ones_like(g, dtype=bool)
            ring[1:-1, 1:-1] = False
            assert np.array_equal(out[ring], g[ring]), (case["name"], "boundary changed")


def _exact_jacobi(grid, T):
    R, C = grid.shape
    A = [[Fraction(float(v)) for v in row] for row in grid]
    fifth = Fraction(1, 5)
    for _ in range(T):
        B = [row[:] for row in A]
        for i in range(1, R - 1):
            for j in range(1, C - 1):
                B[i][j] = fifth * (A[i][j] + A[i - 1][j] + A[i + 1][j] + A[i][j - 1] + A[i][j + 1])
        A = B
    return np.array([[float(v) for v in row] for row in A])


def pin_exact_bruteforce(lib):
    r = np.random.default_rng(1234)
    for (R, C, T) in [(3, 3, 5), (3, 7, 9), (5, 4, 8), (6, 8, 12), (8, 8, 10), (4, 9, 3)]:
        g = r.random((R, C)) * 2.0 - 0.5
        got = oracle.jacobi2d(g, T, lib=lib)
        want = _exact_jacobi(g, T)
        bound = (T + 1) * 8 * EPS * np.abs(g).max()
        assert np.abs(got - want).max() <= bound, (R, C, T, np.abs(got - want).max(), bound)


def _lam(R, C, p, q):
    return 0.2 + 0.4 * (math.cos(p * math.pi / (R - 1)) + math.cos(q * math.pi / (C - 1)))


def pin_eigenmodes(lib):
    for (R, C, p, q, T) in [(9, 14, 2, 3, 37), (17, 6, 1, 4, 25), (33, 21, 5, 1, 60), (3, 11, 1, 2, 15)]:
        g = inputs.eigenmode(R, C, p, q)
        lam = _lam(R, C, p, q)
        got = oracle.jacobi2d(g, T, lib=lib)
        want = (lam ** T) * g
        assert np.abs(got - want).max() <= (T + 2) * 8 * EPS, (R, C, p, q, T, np.abs(got - want).max())


def pin_harmonic_fixed_points(lib):
    for kind in ["const", "x2-y2", "xy", "x3-3xy2"]:
        g = inputs.harmonic_field(23, 31, kind)
        T = 40
        got = oracle.jacobi2d(g, T, lib=lib)
        scale = max(1.0, np.abs(g).max())
        assert np.abs(got - g).max() <= T * 8 * EPS * scale, (kind, np.abs(got - g).max())


def pin_max_principle_and_boundary(lib):
    r = np.random.default_rng(7)
    g = r.random((19, 26)) * 3.0 - 1.0
    out = oracle.jacobi2d(g, 53, lib=lib)
    tol = 8 * EPS * np.abs(g).max()
    assert out.min() >= g.min() - tol and out.max() <= g.max() + tol
    assert np.array_equal(out[0], g[0]) and np.array_equal(out[-1], g[-1])
    assert np.array_equal(out[:, 0], g[:, 0]) and np.array_equal(out[:, -1], g[:, -1])


def pin_symmetries(lib):
    r = np.random.default_rng(11)
    g = r.random((13, 21))
    T = 17
    base = oracle.jacobi2d(g, T, lib=lib)
    assert np.array_equal(oracle.jacobi2d(g.T.copy(), T, lib=lib), base.T)
    assert np.array_equal(oracle.jacobi2d(g[::-1].copy(), T, lib=lib), base[::-1])
    assert np.array_equal(oracle.jacobi2d(g[:, ::-1].copy(), T, lib=lib), base[:, ::-1])


def pin_semigroup(lib):
    r = np.random.default_rng(5)
    g = r.random((15, 18))
    a = oracle.jacobi2d(oracle.jacobi2d(g, 7, lib=lib), 5, lib=lib)
    b = oracle.jacobi2d(g, 12, lib=lib)
    assert np.array_equal(a, b)


def pin_linearity(lib):
    r = np.random.default_rng(9)
    x = r.random((12, 16))
    y = r.random((12, 16))
    T = 9
    lhs = oracle.jacobi2d(2.5 * x + y, T, lib=lib)
    rhs = 2.5 * oracle.jacobi2d(x, T, lib=lib) + oracle.jacobi2d(y, T, lib=lib)
    assert np.abs(lhs - rhs).max() <= 1e-13


def pin_special_cases(lib):
    r = np.random.default_rng(3)
    for shape in [(1, 1), (1, 9), (2, 5), (7, 2), (2, 2)]:
        g = r.random(shape)
        assert np.array_equal(oracle.jacobi2d(g, 10, lib=lib), g)
    g = r.random((6, 6))
    assert np.array_equal(oracle.jacobi2d(g, 0, lib=lib), g)


def pin_tolerance_closed_form(lib):
    R, C, p, q = 12, 17, 1, 1
    g = inputs.eigenmode(R, C, p, q)
    lam = _lam(R, C, p, q)
    tol, stride, cap = 1e-3, 16, 5000
    # first multiple of stride with lam^(t-1) <= tol
    t_pred = next(t for t in range(stride, cap + 1, stride) if lam ** (t - 1) <= tol)
    margin = abs(math.log(lam ** (t_pred - 1) / tol))
    assert margin > 1e-6 and abs(math.log(lam ** (t_pred - 1 - stride) / tol)) > 1e-6
    out, steps, rel, r1 = oracle.jacobi2d_tol(g, cap, tol, stride, lib=lib)
    assert steps == t_pred, (steps, t_pred)
    assert abs(rel - lam ** (t_pred - 1)) <= 1e-9 * lam ** (t_pred - 1), (rel, lam ** (t_pred - 1))
    r1_pred = abs(lam - 1.0) * np.sqrt((g[1:-1, 1:-1] ** 2).sum())
    assert abs(r1 - r1_pred) <= 1e-12 * r1_pred, (r1, r1_pred)
    assert np.abs(out - lam ** t_pred * g).max() <= (t_pred + 2) * 8 * EPS
    # cap reached before tolerance: stops at the cap, residual reported there
    out2, steps2, rel2, _ = oracle.jacobi2d_tol(g, 100, tol, stride, lib=lib)
    assert steps2 == 100 and abs(rel2 - lam ** 99) <= 1e-9 * lam ** 99
    # zero first-step update (harmonic field): converged at the first check
    h = inputs.harmonic_field(10, 10, "const")
    _, steps3, rel3, r13 = oracle.jacobi2d_tol(h, 1000, 1e-6, 32, lib=lib)
    assert steps3 == 32 and rel3 == 0.0 and r13 == 0.0


def pin_window_light_cone(lib):
    r = np.random.default_rng(21)
    g = r.random((40, 47))
    T = 6
    full = oracle.jacobi2d(g, T, lib=lib)
    for (r0, r1, c0, c1) in [(0, 5, 0, 5), (17, 23, 20, 28), (35, 40, 40, 47), (10, 11, 0, 47)]:
        w = oracle.jacobi2d_window(g, T, r0, r1, c0, c1, lib=lib)
        assert np.array_equal(w, full[r0:r1, c0:c1]), (r0, r1, c0, c1)


ALL_PINS = [pin_hand_fixtures, pin_exact_bruteforce, pin_eigenmodes, pin_harmonic_fixed_points,
            pin_max_principle_and_boundary, pin_symmetries, pin_semigroup, pin_linearity,
            pin_special_cases, pin_tolerance_closed_form, pin_window_light_cone]


# --------------------------------------------------------------- tests ----------

@pytest.fixture(scope="module")
def lib():
    return oracle._get()


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_pin(pin, lib):
    pin(lib)


def test_thread_count_invariance(lib):
    r = np.random.default_rng(17)
    g = r.random((67, 45))
    a = oracle.jacobi2d(g, 23, threads=1, lib=lib)
    b = oracle.jacobi2d(g, 23, threads=4, lib=lib)
    assert np.array_equal(a, b)
    ta = oracle.jacobi2d_tol(g, 300, 1e-3, 16, threads=1, lib=lib)
    tb = oracle.jacobi2d_tol(g, 300, 1e-3, 16, threads=3, lib=lib)
    assert np.array_equal(ta[0], tb[0]) and ta[1:] == tb[1:]


def test_tol_mode_matches_plain_mode(lib):
    r = np.random.default_rng(19)
    g = r.random((20, 30))
    out, steps, _, _ = oracle.jacobi2d_tol(g, 200, 0.0, 16, lib=lib)
    assert steps == 200
    assert np.array_equal(out, oracle.jacobi2d(g, 200, lib=lib))


def test_invalid_arguments(lib):
    with pytest.raises(ValueError):
        oracle.jacobi2d(np.zeros((4, 4)), -1, lib=lib)
    with pytest.raises(ValueError):
        oracle.jacobi2d_tol(np.zeros((4, 4)), 10, 1e-3, 0, lib=lib)
