"""The allocation-free entry point, sdfg_jacobi2d_noalloc, for callers that
may not allocate device memory: its scratch grid is a fixed array inside the
library.  Checked through the C ABI against the ordinary entry point
(sdfg_jacobi2d) on two calls in a row -- the second call finds the array
holding the first call's data and must not depend on it -- and for the
host-side rejection of grids larger than the array.

This file is collected last, so a run that stops at its first failure has
already run every other test."""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("shape,Ts", [((300, 516), (37, 16)), ((2048, 2048), (24, 9)), ((129, 132), (5, 8))])
def test_noalloc_matches_existing_entry_point_twice(shape, Ts):
    R, C = shape
    for call, T in enumerate(Ts):           # two calls in a row, different inputs and T
        x = torch.from_numpy(inputs.uniform_grid(R, C, seed=call + R)).float().cuda()
        y = torch.empty_like(x)
        noalloc(x, y, T)
        want = reference(x, T)
        err = (y.double() - want.double()).abs().max().item()
        assert err <= TOL32, (shape, call, T, err)
    assert binding.sdfg_device_error(True) == 0


def test_noalloc_in_place():
    x = torch.from_numpy(inputs.uniform_grid(200, 200, seed=9)).float().cuda()
    want = reference(x, 13)
    noalloc(x, x, 13)
    assert (x.double() - want.double()).abs().max().item() <= TOL32


def test_noalloc_rejects_oversize_and_unaligned():
    R = 4096
    C = MAX_ELEMS // R + 4                 # one row past the static array
    rc = binding.sdfg_jacobi2d_noalloc(1 << 20, 1 << 40, R, C, 3, 0)
    assert rc == binding.SDFG_ERR_INVAL and "static scratch" in binding.last_error()
    x = torch.zeros((10, 10), device="cuda")
    rc = binding.sdfg_jacobi2d_noalloc(x.data_ptr(), x.data_ptr(), 10, 10, 3, 0)
    assert rc == binding.SDFG_ERR_INVAL
