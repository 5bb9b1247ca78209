"""The allocation-free entry point, sdfg_jacobi2d_noalloc, for callers that
may not allocate device memory (a plug-in whose host application owns the
whole device memory budget, or a loop that cannot take an allocation's
implicit synchronisation): its scratch grid is a fixed array inside the
library.

Checked through the C ABI on two calls in a row -- the second call finds the
array holding the first call's data and must not depend on it -- against the
FP64 oracle (max-abs 1e-4, the FP32 tolerance) and against the ordinary
entry point (sdfg_jacobi2d) within the same tolerance; at the largest grid
the array holds; on grids with no interior (a copy); and for the host-side
rejection of grids larger than the array.  The entry point's own device
error word is read through sdfg_device_error.

This file is collected last, so a run that stops at its first failure has
already run every other test."""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
TOL32 = 1e-4
MAX_ELEMS = 8 << 20


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = binding.lib()
    binding.sdfg_device_error(True)
    return L


def reference(x, T):
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    binding.check(binding.sdfg_jacobi2d(x.data_ptr(), y.data_ptr(), x.shape[0], x.shape[1], T, s))
    torch.cuda.synchronize()
    return y


def noalloc(x, y, T):
    s = torch.cuda.current_stream().cuda_stream
    binding.check(binding.sdfg_jacobi2d_noalloc(x.data_ptr(), y.data_ptr(), x.shape[0], x.shape[1], T, s))
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0


def h64(t):
    return t.double().cpu().numpy()


def test_empty_call_is_the_set_up():
    # rows = 0 does only the per-device set-up (the documented warm-up call)
    binding.check(binding.sdfg_jacobi2d_noalloc(0, 0, 0, 16, 5, 0))
    binding.check(binding.sdfg_jacobi2d_noalloc(0, 0, 16, 0, 5, 0))


@pytest.mark.parametrize("shape,Ts", [((300, 516), (37, 16)), ((2048, 2048), (24, 9)), ((129, 132), (5, 8))])
def test_noalloc_matches_oracle_and_existing_entry_point_twice(shape, Ts):
    R, C = shape
    for call, T in enumerate(Ts):           # two calls in a row, different inputs and T
        x = torch.from_numpy(inputs.uniform_grid(R, C, seed=call + R)).float().cuda()
        y = torch.empty_like(x)
        noalloc(x, y, T)
        want = oracle.jacobi2d(h64(x), T, threads=0)
        err = np.abs(h64(y) - want).max()
        assert err <= TOL32, (shape, call, T, "oracle", err)
        err2 = (y.double() - reference(x, T).double()).abs().max().item()
        assert err2 <= TOL32, (shape, call, T, "sdfg_jacobi2d", err2)


def test_noalloc_in_place():
    x = torch.from_numpy(inputs.uniform_grid(200, 200, seed=9)).float().cuda()
    want = oracle.jacobi2d(h64(x), 13, threads=0)
    noalloc(x, x, 13)
    assert np.abs(h64(x) - want).max() <= TOL32


def test_noalloc_largest_grid_the_array_holds():
    R, C = 2048, MAX_ELEMS // 2048          # exactly 8,388,608 elements
    x = torch.from_numpy(inputs.uniform_grid(R, C, seed=5)).float().cuda()
    y = torch.empty_like(x)
    noalloc(x, y, 11)
    want = oracle.jacobi2d(h64(x), 11, threads=0)
    assert np.abs(h64(y) - want).max() <= TOL32


@pytest.mark.parametrize("shape", [(2, 8), (2, 4), (1, 12)])
def test_noalloc_no_interior_is_a_copy(shape):
    x = torch.from_numpy(inputs.uniform_grid(*shape, seed=3)).float().cuda()
    y = torch.full_like(x, -1.0)
    noalloc(x, y, 7)
    assert torch.equal(x, y)


def test_noalloc_rejects_oversize_and_unaligned():
    R = 4096
    C = MAX_ELEMS // R + 4                 # one row past the static array
    rc = binding.sdfg_jacobi2d_noalloc(1 << 20, 1 << 40, R, C, 3, 0)
    assert rc == binding.SDFG_ERR_INVAL and "static scratch" in binding.last_error()
    x = torch.zeros((10, 10), device="cuda")
    rc = binding.sdfg_jacobi2d_noalloc(x.data_ptr(), x.data_ptr(), 10, 10, 3, 0)
    assert rc == binding.SDFG_ERR_INVAL
