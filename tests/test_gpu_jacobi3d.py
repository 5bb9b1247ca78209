"""Parity of the 3-D 7-point path (sdfg_jacobi3d) with the FP64 oracle.

Tolerances (max-abs against the FP64 oracle run on exactly the values the GPU
received): FP64 bitwise (same order of operations), FP32 1e-4, BF16 2e-2 on a
smooth field.  Shapes span several tiles along every axis with ragged tails
(tile: 16 rows x 120 columns for FP32, 60 for FP64, 112 for BF16; at least 32
planes per CTA), boxes of a single interior point, in-place runs, pitched and
unaligned layouts (staged through an aligned copy) and degenerate extents.
The full-size case (512^3, T=100) is checked on light-cone windows: the
oracle runs on a crop reaching T+1 cells past each window, which fixes the
window exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

F32, BF16, F64 = binding.SDFG_F32, binding.SDFG_BF16, binding.SDFG_F64
TDT = {F32: torch.float32, BF16: torch.bfloat16, F64: torch.float64}
TOL = {F32: 1e-4, BF16: 2e-2, F64: 0.0}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = binding.lib()
    binding.sdfg_device_error(True)
    return L


def h64(t):
    return t.double().cpu().numpy()


def run(x, T, out=None):
    y = torch.empty_like(x) if out is None else out
    binding.jacobi3d(x, y, T)
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    return y


def check(y, x, T, dt):
    want = oracle.jacobi3d(h64(x), T, threads=0)
    got = h64(y)
    if TOL[dt] == 0.0:
        assert np.array_equal(got, want), "FP64 path should equal the oracle bit for bit"
    else:
        assert np.abs(got - want).max() <= TOL[dt]
    # the shell is never written
    sh = np.ones(got.shape, bool)
    sh[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(got[sh], h64(x)[sh])


SHAPES = [(3, 3, 3), (5, 7, 9), (4, 17, 121), (33, 40, 130), (70, 17, 250), (40, 33, 64), (97, 20, 37)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T", [1, 2, 7])
def test_f64_bitwise(shape, T):
    g = np.random.default_rng(sum(shape) + T).random(shape)
    x = torch.from_numpy(g).cuda()
    check(run(x, T), x, T, F64)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T", [1, 6, 19])
def test_f32(shape, T):
    g = np.random.default_rng(7 * sum(shape) + T).random(shape)
    x = torch.from_numpy(g).float().cuda()
    check(run(x, T), x, T, F32)


@pytest.mark.parametrize("shape", [(20, 50, 300), (45, 64, 129)])
def test_bf16_smooth_field(shape):
    D, R, C = shape
    z = np.arange(D)[:, None, None] / D
    i = np.arange(R)[None, :, None] / R
    j = np.arange(C)[None, None, :] / C
    g = 0.5 + 0.25 * np.sin(2 * np.pi * (i + 2 * j)) * np.cos(2 * np.pi * z) + 0.1 * np.sin(6 * np.pi * z * j)
    x = torch.from_numpy(g).to(torch.bfloat16).cuda()
    check(run(x, 12), x, 12, BF16)


def test_in_place_and_odd_even_T():
    g = np.random.default_rng(1).random((34, 35, 140))
    for T in (1, 4, 5):
        x = torch.from_numpy(g).float().cuda()
        x0 = x.clone()
        binding.jacobi3d(x, x, T)
        torch.cuda.synchronize()
        assert binding.sdfg_device_error(True) == 0
        check(x, x0, T, F32)


def test_pitched_and_unaligned_layouts():
    D, R, C, T = 20, 30, 101, 5
    g = np.random.default_rng(2).random((D, R, C))
    # pitched: ld = 128 (16-byte rows), planes R * ld apart
    buf = torch.zeros((D, R, 128), device="cuda")
    buf[:, :, :C] = torch.from_numpy(g).float().cuda()
    x = buf[:, :, :C]
    out = torch.zeros_like(buf)[:, :, :C]
    y = run(x, T, out=out)
    check(y, x, T, F32)
    # unaligned: a view starting one element in (staged through an aligned copy)
    flat = torch.zeros(D * R * C + 1, device="cuda")
    xu = flat[1:].view(D, R, C)
    xu.copy_(torch.from_numpy(g).float())
    yu = run(xu, T)
    assert torch.equal(yu, y.contiguous())


@pytest.mark.parametrize("shape", [(2, 5, 5), (5, 2, 5), (5, 5, 2), (1, 1, 1)])
def test_degenerate_extents_copy(shape):
    x = torch.rand(shape, device="cuda")
    y = run(x, 9)
    assert torch.equal(x, y)


def test_T0_and_empty_and_errors():
    x = torch.rand((6, 7, 8), device="cuda")
    assert torch.equal(run(x, 0), x)
    e = torch.empty((0, 5, 5), device="cuda")
    run(e, 3)
    L = binding.lib()
    assert L.sdfg_jacobi3d(x.data_ptr(), x.data_ptr(), 6, 7, 8, 8, -1, F32, 0) == binding.SDFG_ERR_INVAL
    assert L.sdfg_jacobi3d(x.data_ptr(), x.data_ptr(), 6, 7, 8, 7, 1, F32, 0) == binding.SDFG_ERR_INVAL  # ld < cols
    assert L.sdfg_jacobi3d(None, None, 6, 7, 8, 8, 1, F32, 0) == binding.SDFG_ERR_INVAL


def test_full_size_512_T100_windows():
    """The 3-D benchmark configuration: 512^3 FP32, T = 100, uniform [0,1) noise."""
    n, T = 512, 100
    g = inputs.uniform_box(n, n, n, seed=0)
    x = torch.from_numpy(g).float().cuda()
    y = run(x, T)
    xs = h64(x)
    ys = y.double()
    windows = [((0, 0, 0), (6, 6, 6)), ((253, 250, 200), (259, 256, 206)), ((506, 100, 506), (512, 106, 512)),
               ((300, 506, 0), (306, 512, 6))]
    for lo, hi in windows:
        want = oracle.jacobi3d_window(xs, T, lo, hi, threads=0)
        got = ys[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].cpu().numpy()
        assert np.abs(got - want).max() <= TOL[F32], (lo, hi)
    # maximum principle over the whole box
    assert float(y.min()) >= float(x.min()) - 1e-6 and float(y.max()) <= float(x.max()) + 1e-6
