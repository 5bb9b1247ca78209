"""Seeded random configurations against the FP64 oracle: shapes from 1 to
~400 per side (ragged widths included), T from 0 to 90, every dtype, kernel,
fused depth and segment height; and a scheduler stress batch of many tiny and
medium grids with mixed step counts and tolerances in one persistent launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

F32, BF16, F64 = binding.SDFG_F32, binding.SDFG_BF16, binding.SDFG_F64
TDT = {F32: torch.float32, BF16: torch.bfloat16, F64: torch.float64}
TOL = {F32: 1e-4, BF16: 2e-2, F64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = binding.lib()
    binding.sdfg_device_error(True)
    return L


def h64(t):
    return t.double().cpu().numpy()


CASES = []
_r = np.random.default_rng(2024)
for _i in range(36):
    R = int(_r.choice([1, 2, 3, 4, 7, 13, 31, 64, 97, 130, 255, 400]))
    C = int(_r.choice([1, 2, 3, 5, 8, 17, 33, 63, 128, 129, 250, 397]))
    T = int(_r.integers(0, 91))
    dt = int(_r.choice([F32, F32, BF16, F64]))
    kernel = int(_r.choice([binding.SDFG_KERNEL_NAIVE, binding.SDFG_KERNEL_TEMPORAL, binding.SDFG_KERNEL_PERSISTENT,
                            binding.SDFG_KERNEL_AUTO]))
    k = int(_r.choice([0, 1, 2, 4, 8]))
    seg = int(_r.choice([0, 12, 24, 48, 96]))
    CASES.append((R, C, T, dt, kernel, k, seg))


@pytest.mark.parametrize("R,C,T,dt,kernel,k,seg", CASES)
def test_random_configuration(R, C, T, dt, kernel, k, seg):
    g = inputs.uniform_grid(R, C, seed=R * 7919 + C * 31 + T)
    x = torch.from_numpy(g).to(TDT[dt]).cuda()
    y = torch.empty_like(x)
    binding.jacobi2d(x, y, T, binding.config(kernel=kernel, k=k, seg_rows=seg))
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    want = oracle.jacobi2d(h64(x), T)
    got = h64(y)
    if R < 3 or C < 3 or T == 0:
        assert np.array_equal(got, want)
    else:
        assert np.abs(got - want).max() <= TOL[dt]
        # the boundary ring is never written
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[-1], want[-1])
        assert np.array_equal(got[:, 0], want[:, 0]) and np.array_equal(got[:, -1], want[:, -1])


def test_scheduler_stress_many_grids():
    r = np.random.default_rng(77)
    xs, ys, descs, specs = [], [], [], []
    for i in range(300):
        R = int(r.choice([1, 3, 4, 9, 20, 57, 130, 300]))
        C = int(r.choice([2, 3, 8, 21, 64, 129, 260]))
        T = int(r.integers(0, 70))
        tol = float(r.choice([0.0, 0.0, 1e-2, 1e-3]))
        g = inputs.laplace_request_grid(inputs.Request(R, C, seed=i)) if tol and R > 2 and C > 2 else \
            inputs.uniform_grid(R, C, seed=i)
        x = torch.from_numpy(g).float().cuda()
        y = torch.zeros_like(x)
        xs.append(x)
        ys.append(y)
        descs.append(binding.desc_for(x, y, T, tol))
        specs.append((R, C, T, tol))
    binding.check(binding.sdfg_jacobi2d_batch(descs, 16))
    assert binding.sdfg_device_error(True) == 0
    for (R, C, T, tol), x, y, d in zip(specs, xs, ys, descs):
        assert d.status == 0
        if tol and R > 2 and C > 2 and T > 0:
            assert 0 < d.steps_done <= T and (d.steps_done == T or d.steps_done % 16 == 0)
        else:
            assert d.steps_done == (T if (R < 3 or C < 3 or not tol) else T)
        want = oracle.jacobi2d(h64(x), d.steps_done)
        assert np.abs(h64(y) - want).max() <= 1e-4, (R, C, T, tol)
