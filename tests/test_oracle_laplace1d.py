"""Pins for the oracle of the paper's Fig. 1 program (1-D Laplace on a
float64[2, N] array, ping-ponged for T steps, end cells never written).

* hand-computed steps on N = 5;
* exact rational brute force (the weights 1, -2, 1 and small dyadic inputs
  keep every intermediate exact in FP64, so equality is bitwise);
* closed form: with zero ends, sin(q pi i / (N-1)) is an eigenvector with
  eigenvalue -4 sin^2(q pi / (2(N-1))) (checked on the dominant mode);
* the two rows' own end values alternate between steps.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    return oracle._get()


def test_hand_steps(lib):
    A = np.array([[1.0, 2.0, 4.0, 8.0, 16.0], [100.0, 0.0, 0.0, 0.0, 200.0]])
    # step 1 reads row 0, writes row 1: 1-4+4=1, 2-8+8=2, 4-16+16=4
    s1 = oracle.laplace1d(A, 1, lib=lib)
    assert s1[1].tolist() == [100.0, 1.0, 2.0, 4.0, 200.0]
    assert s1[0].tolist() == A[0].tolist()
    # step 2 reads row 1 (ends 100, 200), writes row 0: 100-2+2=100, 1-4+4=1, 2-8+200=194
    s2 = oracle.laplace1d(A, 2, lib=lib)
    assert s2[0].tolist() == [1.0, 100.0, 1.0, 194.0, 16.0]


def _exact(A, T):
    rows = [[Fraction(float(v)) for v in r] for r in A]
    N = len(rows[0])
    for t in range(T):
        src, dst = rows[t % 2], rows[(t + 1) % 2]
        for i in range(1, N - 1):
            dst[i] = src[i - 1] - 2 * src[i] + src[i + 1]
    return np.array([[float(v) for v in r] for r in rows])


def test_exact_bruteforce(lib):
    r = np.random.default_rng(3)
    for N, T in [(3, 4), (7, 9), (12, 15), (33, 20)]:
        A = r.integers(-8, 9, size=(2, N)).astype(np.float64) / 4.0   # small dyadics: all exact
        assert np.array_equal(oracle.laplace1d(A, T, lib=lib), _exact(A, T))


def test_eigenvector_closed_form(lib):
    # the operator amplifies rounding noise in its highest modes by up to 4^T,
    # so pin with the dominant mode (|lambda| close to 4), where the relative
    # error stays at rounding level
    N, q, T = 41, 39, 12
    i = np.arange(N)
    v = np.sin(q * math.pi * i / (N - 1))
    v[0] = v[-1] = 0.0
    A = np.vstack([v, np.zeros(N)])
    lam = -4.0 * math.sin(q * math.pi / (2 * (N - 1))) ** 2
    out = oracle.laplace1d(A, T, lib=lib)
    assert np.abs(out[T % 2] - lam ** T * v).max() <= 1e-12 * abs(lam) ** T


def test_paper_configuration_runs(lib):
    # the figure's call: a = rand(2, 2033); Laplace(A=a, T=500)
    a = np.random.default_rng(0).random((2, 2033))
    out = oracle.laplace1d(a, 500, lib=lib)
    assert np.isfinite(out).all()
    assert out[0, 0] == a[0, 0] and out[1, -1] == a[1, -1]
