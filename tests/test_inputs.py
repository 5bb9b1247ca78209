"""Seeded input generators: determinism and the stated shapes/distributions."""
import math

import numpy as np

from paper_1902_10345_gb300 import inputs


def test_uniform_grid_deterministic():
    a = inputs.uniform_grid(33, 47, seed=3)
    b = inputs.uniform_grid(33, 47, seed=3)
    assert a.shape == (33, 47) and np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, inputs.uniform_grid(33, 47, seed=4))


def test_batch_specs_ranges():
    specs = inputs.batch_specs(512, seed=0)
    assert len(specs) == 512
    assert all(64 <= s.rows <= 2048 and 64 <= s.cols <= 2048 and 50 <= s.T <= 500 for s in specs)
    assert specs == inputs.batch_specs(512, seed=0)
    # log-uniform: median side near sqrt(64*2048) = 362
    med = np.median([s.rows for s in specs])
    assert 250 < med < 520
    assert len({s.seed for s in specs}) == 512


def test_sinusoid_field_stats():
    f = inputs.sinusoid_field(256, seed=1)
    assert f.shape == (256, 256)
    assert -0.06 <= f.min() and f.max() <= 1.06
    assert abs(f.mean() - 0.5) < 0.05


def test_served_requests_and_grid():
    reqs = inputs.served_requests(200, seed=0, rate_hz=1000.0)
    assert all(32 <= r.rows <= 4096 and 32 <= r.cols <= 4096 for r in reqs)
    t = [r.arrival_s for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    g = inputs.laplace_request_grid(inputs.Request(40, 57, seed=5))
    assert np.all(g[1:-1, 1:-1] == 0.0)
    x = np.arange(57) / 56.0
    assert np.abs(g[0] - x * x).max() <= 1e-3
    y = np.arange(40) / 39.0
    assert np.abs(g[:, 0] + y * y).max() <= 1e-3


def test_eigenmode_zero_ring():
    g = inputs.eigenmode(9, 14, 2, 3)
    assert np.all(g[0] == 0) and np.all(g[-1] == 0) and np.all(g[:, 0] == 0) and np.all(g[:, -1] == 0)
    assert abs(g[2, 3] - math.sin(2 * math.pi * 2 / 8) * math.sin(3 * math.pi * 3 / 13)) < 1e-15
