"""Parity of the register-resident pass kernel (SDFG_KERNEL_RESIDENT) with the
FP64 oracle, through the C ABI.

The kernel computes every point in the exact order of the definition,
0.2 * (c + ((n + s) + (w + e))), each FP32 operation rounded on its own, so
its FP32 result must equal that sequence written out in numpy bit for bit
(which also proves that no multiply was fused into an add), and lie within
1e-4 of the FP64 oracle.  BF16 storage (rounded when a pass stores) within
2e-2 on a smooth field; FP64 grids run the temporal kernel instead and stay
bitwise.  Shapes span several 256-row x 112-column tiles with ragged edges;
T covers partial last passes for k = 8, 4, 2 and 1.  At the paper's 2048^2
size (exactly 8 x 19 tiles) the closed-form eigenmode after 1024 steps.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

F32, BF16, F64 = binding.SDFG_F32, binding.SDFG_BF16, binding.SDFG_F64
RESIDENT = binding.SDFG_KERNEL_RESIDENT
TDT = {F32: torch.float32, BF16: torch.bfloat16, F64: torch.float64}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = binding.lib()
    binding.sdfg_device_error(True)
    return L


def run(x, T, k, out=None):
    y = torch.empty_like(x) if out is None else out
    binding.jacobi2d(x, y, T, binding.config(kernel=RESIDENT, k=k))
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    return y


def h64(t):
    return t.double().cpu().numpy()


def fp32_sequence(g32, T):
    """T Jacobi steps in float32, every operation rounded on its own:
    0.2f * (c + ((n + s) + (w + e))); the ring is never written."""
    A = np.array(g32, dtype=np.float32)
    f = np.float32(0.2)
    for _ in range(T):
        B = A.copy()
        n, s, w, e, c = A[:-2, 1:-1], A[2:, 1:-1], A[1:-1, :-2], A[1:-1, 2:], A[1:-1, 1:-1]
        B[1:-1, 1:-1] = f * (c + ((n + s) + (w + e)))
        A = B
    return A


SHAPES = [(3, 3), (5, 7), (9, 130), (130, 9), (257, 113), (300, 250), (520, 230), (129, 131), (140, 236)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T,k", [(1, 8), (8, 8), (13, 8), (9, 4), (5, 2), (3, 1)])
def test_f32_bitwise_sequence_and_oracle(shape, T, k):
    g = np.random.default_rng(sum(shape) + T).random(shape)
    x = torch.from_numpy(g).float().cuda()
    got = run(x, T, k).cpu().numpy()
    want32 = fp32_sequence(x.cpu().numpy(), T)
    diff = got != want32
    assert not diff.any(), (int(diff.sum()), float(np.abs(got - want32).max()), np.argwhere(diff)[:4].tolist())
    assert np.abs(got.astype(np.float64) - oracle.jacobi2d(h64(x), T, threads=0)).max() <= 1e-4


def test_more_tiles_than_sms_bitwise():
    """2100^2 is 9 x 19 = 171 tiles: more than one wave of CTAs (one per SM),
    with ring rows and columns at other band rows and lane elements than
    2048^2 has."""
    R, C, T = 2100, 2100, 13
    g = np.random.default_rng(11).random((R, C))
    x = torch.from_numpy(g).float().cuda()
    got = run(x, T, 8).cpu().numpy()
    assert np.array_equal(got, fp32_sequence(x.cpu().numpy(), T))


def test_bf16_smooth_field():
    R, C, T = 300, 250, 21
    g = inputs.sinusoid_field(max(R, C), seed=3, k_max=1)[:R, :C]
    x = torch.from_numpy(np.ascontiguousarray(g)).to(torch.bfloat16).cuda()
    got = h64(run(x, T, 8))
    assert np.abs(got - oracle.jacobi2d(h64(x), T, threads=0)).max() <= 2e-2
    ring = np.ones(got.shape, bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(got[ring], h64(x)[ring])


def test_f64_runs_the_temporal_kernel_bitwise():
    g = np.random.default_rng(7).random((70, 90))
    x = torch.from_numpy(g).cuda()
    assert np.array_equal(h64(run(x, 11, 8)), oracle.jacobi2d(g, 11, threads=0))


def test_in_place_pitched_and_unaligned():
    R, C, T = 150, 201, 10
    g = np.random.default_rng(8).random((R, C))
    want = fp32_sequence(g.astype(np.float32), T)
    x = torch.from_numpy(g).float().cuda()
    run(x, T, 8, out=x)
    assert np.array_equal(x.cpu().numpy(), want)
    buf = torch.zeros((R, 224), device="cuda")
    buf[:, :C] = torch.from_numpy(g).float().cuda()
    y = torch.zeros((R, 224), device="cuda")[:, :C]
    run(buf[:, :C], T, 8, out=y)
    assert np.array_equal(y.cpu().numpy(), want)
    flat = torch.zeros(R * C + 1, device="cuda")
    xu = flat[1:].view(R, C)
    xu.copy_(torch.from_numpy(g).float())
    assert np.array_equal(run(xu, T, 8).cpu().numpy(), want)


def test_paper_workload_eigenmode_2048_T1024():
    """The paper's workload: 2048^2, zero ring, T = 1024; the (3, 5)
    eigenmode decays by exactly lambda^T."""
    R = C = 2048
    T = 1024
    i = np.arange(R)[:, None]
    j = np.arange(C)[None, :]
    p, q = 3, 5
    mode = np.sin(p * np.pi * i / (R - 1)) * np.sin(q * np.pi * j / (C - 1))
    mode[0, :] = mode[-1, :] = 0.0
    mode[:, 0] = mode[:, -1] = 0.0
    x = torch.from_numpy(mode).float().cuda()
    lam = 0.2 + 0.4 * (np.cos(p * np.pi / (R - 1)) + np.cos(q * np.pi / (C - 1)))
    want = lam ** T * h64(x)
    got = h64(run(x, T, 8))
    assert np.abs(got - want).max() <= 1e-4


def test_unknown_kernel_family_and_depth_rejected():
    x = torch.rand((40, 50), device="cuda")
    y = torch.empty_like(x)
    for bad in (binding.config(kernel=binding.SDFG_KERNEL_SKEWED + 1), binding.config(kernel=-1), binding.config(kernel=RESIDENT, k=3),
                binding.config(kernel=RESIDENT, k=16)):
        rc = binding.sdfg_jacobi2d_cfg(x.data_ptr(), y.data_ptr(), 40, 50, 50, 5, F32, bad, 0)
        assert rc == binding.SDFG_ERR_INVAL, (bad.kernel, bad.k, rc)
    # a valid configuration still runs afterwards
    run(x, 5, 4, out=y)


def test_autotune_may_choose_the_resident_kernel_and_stays_correct():
    R = C = 1024
    T = 64
    cfg = binding.sdfg_autotune(R, C, T, F32, torch.cuda.current_stream().cuda_stream)
    g = np.random.default_rng(9).random((R, C))
    x = torch.from_numpy(g).float().cuda()
    y = torch.empty_like(x)
    binding.jacobi2d(x, y, T, cfg)
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    for (r0, c0) in [(0, 0), (500, 300), (1016, 1016)]:
        want = oracle.jacobi2d_window(h64(x), T, r0, r0 + 8, c0, c0 + 8, threads=0)
        assert np.abs(h64(y)[r0:r0 + 8, c0:c0 + 8] - want).max() <= 1e-4, (cfg.kernel, cfg.k)
