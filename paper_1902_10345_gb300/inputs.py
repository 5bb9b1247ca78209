"""Seeded synthetic inputs for the Jacobi-2D workloads.

This module holds only random draws and closed-form test fields: none of the
stencil's arithmetic.  Both the CUDA path and the FP64 oracle consume what it
produces, so it is the one module the two sides share.

All draws use numpy's ``default_rng(seed)`` (PCG64) in FP64; callers cast to
the storage type, and the oracle is fed ``float64(cast(x))`` so both sides see
identical values.

Workloads (shapes and distributions of the paper's Jacobi benchmark, Sec. 6.1:
a square 2-D domain, constant boundary, T in the hundreds to thousands):

* ``uniform_grid``      -- i.i.d. uniform[0,1) grid, boundary included (one
                           row-major draw);
* ``batch_specs``       -- 512 grids, rows and cols log-uniform in [64, 2048],
                           T uniform in [50, 500];
* ``sinusoid_field``    -- sum of 8 random 2-D sinusoids + 0.5 + noise;
* ``served_requests``   -- Laplace solves with boundary x^2 - y^2 (+ noise)
                           and a zero interior, Poisson arrivals;
* ``eigenmode`` / ``harmonic_field`` -- closed-form test fields.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_grid(rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """rows x cols draw of uniform[0,1) in one row-major call (boundary included)."""
    return rng_for(seed).random((rows, cols))


def uniform_box(depth: int, rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """depth x rows x cols draw of uniform[0,1) in one row-major call (shell
    included): the 3-D counterpart of uniform_grid."""
    return rng_for(seed).random((depth, rows, cols))


# --- the five workload recipes -------------------------------------------------

SINGLE_SMALL = dict(rows=256, cols=256, T=100, seed=0)        # FP64 parity case
SINGLE_LARGE = dict(rows=8192, cols=8192, T=1000, seed=0)     # FP32 throughput case


@dataclasses.dataclass
class GridSpec:
    rows: int
    cols: int
    T: int
    seed: int


def batch_specs(n: int = 512, seed: int = 0, lo: int = 64, hi: int = 2048, t_lo: int = 50, t_hi: int = 500):
    """Shapes and step counts of the uneven batch, drawn in order grid 0..n-1.

    For each grid: rows, cols = round(exp(U(ln lo, ln hi))) independently, then
    T = integers(t_lo, t_hi + 1).  Grid g's values come from ``batch_grid``
    with its own seed, so any subset can be regenerated without the others.
    """
    r = rng_for(seed)
    out = []
    for g in range(n):
        rows = int(round(math.exp(r.uniform(math.log(lo), math.log(hi)))))
        cols = int(round(math.exp(r.uniform(math.log(lo), math.log(hi)))))
        T = int(r.integers(t_lo, t_hi + 1))
        out.append(GridSpec(rows, cols, T, seed * 100003 + g + 1))
    return out


def batch_grid(spec: GridSpec) -> np.ndarray:
    return uniform_grid(spec.rows, spec.cols, spec.seed)


def sinusoid_field(n: int, seed: int = 0, modes: int = 8, k_max: int = 64, noise: float = 0.05) -> np.ndarray:
    """n x n field: 0.5 + sum of `modes` sinusoids + uniform noise.

    f = 0.5 + sum_m a_m sin(2 pi (kx_m x + ky_m y) + phi_m) + eta, with
    kx, ky integers uniform in [1, k_max], phi uniform in [0, 2 pi),
    a_m = 0.5 w_m / sum(w), w uniform in (0, 1), eta uniform in
    [-noise, noise], x = j / n, y = i / n.  Not clamped.
    """
    r = rng_for(seed)
    kx = r.integers(1, k_max + 1, size=modes)
    ky = r.integers(1, k_max + 1, size=modes)
    phi = r.uniform(0.0, 2.0 * math.pi, size=modes)
    w = r.uniform(0.0, 1.0, size=modes)
    a = 0.5 * w / w.sum()
    x = np.arange(n, dtype=np.float64) / n
    f = np.full((n, n), 0.5)
    for m in range(modes):
        # sin(A + B) expanded so the field is built from rank-1 outer products
        ax = 2.0 * math.pi * kx[m] * x
        ay = 2.0 * math.pi * ky[m] * x + phi[m]
        f += a[m] * (np.outer(np.cos(ay), np.sin(ax)) + np.outer(np.sin(ay), np.cos(ax)))
    f += r.uniform(-noise, noise, size=(n, n))
    return f


def sinusoid_field_device(n: int, seed: int = 0, modes: int = 8, k_max: int = 64, noise: float = 0.05,
                          device="cuda"):
    """The sinusoid field of ``sinusoid_field`` built on a torch device (for
    large n).  The random parameters come from the same numpy stream in the
    same order; the noise is drawn by numpy per row block so host memory stays
    bounded.  Values agree with ``sinusoid_field`` up to last-bit differences
    of the two libraries' sin/cos."""
    import torch
    r = rng_for(seed)
    kx = r.integers(1, k_max + 1, size=modes)
    ky = r.integers(1, k_max + 1, size=modes)
    phi = r.uniform(0.0, 2.0 * math.pi, size=modes)
    w = r.uniform(0.0, 1.0, size=modes)
    a = 0.5 * w / w.sum()
    x = torch.arange(n, dtype=torch.float64, device=device) / n
    f = torch.full((n, n), 0.5, dtype=torch.float64, device=device)
    for m in range(modes):
        ax = 2.0 * math.pi * float(kx[m]) * x
        ay = 2.0 * math.pi * float(ky[m]) * x + float(phi[m])
        f += float(a[m]) * (torch.outer(torch.cos(ay), torch.sin(ax)) + torch.outer(torch.sin(ay), torch.cos(ax)))
    block = max(1, (1 << 24) // n)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        f[i0:i1] += torch.from_numpy(r.uniform(-noise, noise, size=(i1 - i0, n))).to(device)
    return f


@dataclasses.dataclass
class Request:
    rows: int
    cols: int
    seed: int
    arrival_s: float = 0.0


def served_requests(n: int = 10000, seed: int = 0, lo: int = 32, hi: int = 4096, rate_hz: float | None = None):
    """Request stream for the served Laplace solves.

    Side lengths log-uniform in [lo, hi]; arrival times form a Poisson process
    of ``rate_hz`` (exponential gaps); rate None means all arrive at t=0.
    """
    r = rng_for(seed)
    reqs = []
    t = 0.0
    for i in range(n):
        rows = int(round(math.exp(r.uniform(math.log(lo), math.log(hi)))))
        cols = int(round(math.exp(r.uniform(math.log(lo), math.log(hi)))))
        if rate_hz:
            t += float(r.exponential(1.0 / rate_hz))
        reqs.append(Request(rows, cols, seed * 1000003 + i + 1, t))
    return reqs


def _ring_noise(req: Request, noise: float):
    """Boundary noise drawn in a fixed order: top row, bottom row, then the
    left and right columns without their corners."""
    R, C = req.rows, req.cols
    r = rng_for(req.seed)
    top = r.uniform(-noise, noise, size=C)
    bottom = r.uniform(-noise, noise, size=C)
    left = r.uniform(-noise, noise, size=max(R - 2, 0))
    right = r.uniform(-noise, noise, size=max(R - 2, 0))
    return top, bottom, left, right


def laplace_request_grid(req: Request, noise: float = 1e-3) -> np.ndarray:
    """Boundary x^2 - y^2 on the unit square (x = j/(C-1), y = i/(R-1)) plus
    uniform noise of amplitude ``noise`` on the boundary ring; interior zero."""
    R, C = req.rows, req.cols
    y = (np.arange(R, dtype=np.float64) / max(R - 1, 1))[:, None]
    x = (np.arange(C, dtype=np.float64) / max(C - 1, 1))[None, :]
    g = x * x - y * y
    top, bottom, left, right = _ring_noise(req, noise)
    g[0, :] += top
    g[-1, :] += bottom
    g[1:-1, 0] += left
    g[1:-1, -1] += right
    g[1:-1, 1:-1] = 0.0
    return g


def laplace_request_grid_device(req: Request, noise: float = 1e-3, device="cuda", dtype=None):
    """``laplace_request_grid`` built on a torch device (same values)."""
    import torch
    R, C = req.rows, req.cols
    y = (torch.arange(R, dtype=torch.float64, device=device) / max(R - 1, 1))[:, None]
    x = (torch.arange(C, dtype=torch.float64, device=device) / max(C - 1, 1))[None, :]
    g = x * x - y * y
    top, bottom, left, right = (torch.from_numpy(v).to(device) for v in _ring_noise(req, noise))
    g[0, :] += top
    g[-1, :] += bottom
    g[1:-1, 0] += left
    g[1:-1, -1] += right
    g[1:-1, 1:-1] = 0.0
    return g if dtype is None else g.to(dtype)


def poisson_arrivals(n: int, rate_hz: float, seed: int = 0) -> np.ndarray:
    r = rng_for(seed + 7919)
    return np.cumsum(r.exponential(1.0 / rate_hz, size=n))


# --- closed-form test fields ------------------------------------------------------

def eigenmode(rows: int, cols: int, p: int, q: int) -> np.ndarray:
    """sin(p pi i/(R-1)) sin(q pi j/(C-1)); zero on the boundary ring."""
    i = np.arange(rows, dtype=np.float64)[:, None]
    j = np.arange(cols, dtype=np.float64)[None, :]
    g = np.sin(p * math.pi * i / (rows - 1)) * np.sin(q * math.pi * j / (cols - 1))
    g[0, :] = 0.0
    g[-1, :] = 0.0
    g[:, 0] = 0.0
    g[:, -1] = 0.0
    return g


def harmonic_field(rows: int, cols: int, kind: str, h: float = 1.0 / 64) -> np.ndarray:
    """Harmonic polynomial in index coordinates x = j h, y = i h (same h)."""
    y = (np.arange(rows, dtype=np.float64) * h)[:, None]
    x = (np.arange(cols, dtype=np.float64) * h)[None, :]
    if kind == "const":
        return np.full((rows, cols), 0.375)
    if kind == "x2-y2":
        return x * x - y * y
    if kind == "xy":
        return x * y
    if kind == "x3-3xy2":
        return x * x * x - 3.0 * x * y * y
    raise ValueError(kind)
