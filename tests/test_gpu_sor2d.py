"""Parity of the red-black SOR path (sdfg_sor2d) with the FP64 oracle.

FP64 is bit-identical (same order of operations); FP32 within 1e-4 and BF16
within 2e-2 on a smooth field.  Shapes span several tiles (64 rows x 112
columns for FP32 and BF16, 60 x 56 for FP64; 4 iterations per launch, 2 for
FP64, with partial last launches) with ragged tails, a single
interior point, both colours at the tile edges, several relaxation factors,
in-place runs, pitched and unaligned layouts and degenerate shapes.  At the
full 8192^2 size the oracle checks light-cone windows (one iteration moves
information at most two cells: the red half-sweep one, the black one more),
and a discrete-harmonic field must stay fixed for the benchmark's 1000
iterations.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

F32, BF16, F64 = binding.SDFG_F32, binding.SDFG_BF16, binding.SDFG_F64
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


def run(x, T, omega, out=None):
    y = torch.empty_like(x) if out is None else out
    binding.sor2d(x, y, T, omega)
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    return y


def check(y, x, T, omega, dt):
    want = oracle.sor2d(h64(x), T, omega)
    got = h64(y)
    if TOL[dt] == 0.0:
        assert np.array_equal(got, want), "FP64 path should equal the oracle bit for bit"
    else:
        assert np.abs(got - want).max() <= TOL[dt]
    ring = np.ones(got.shape, bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(got[ring], h64(x)[ring])


SHAPES = [(3, 3), (4, 4), (5, 7), (37, 130), (130, 37), (200, 515), (64, 241), (57, 61)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T,omega", [(1, 1.0), (2, 1.5), (9, 0.7), (6, 1.9)])
def test_f64_bitwise(shape, T, omega):
    g = np.random.default_rng(sum(shape) + T).random(shape)
    x = torch.from_numpy(g).cuda()
    check(run(x, T, omega), x, T, omega, F64)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T,omega", [(1, 1.0), (7, 1.5), (15, 1.9)])
def test_f32(shape, T, omega):
    g = np.random.default_rng(3 * sum(shape) + T).random(shape)
    x = torch.from_numpy(g).float().cuda()
    check(run(x, T, omega), x, T, omega, F32)


def test_bf16_smooth_field():
    n = 300
    g = inputs.sinusoid_field(n, seed=2, k_max=1)[:250, :300]
    x = torch.from_numpy(np.ascontiguousarray(g)).to(torch.bfloat16).cuda()
    check(run(x, 10, 1.0), x, 10, 1.0, BF16)


@pytest.mark.parametrize("shape", [(90, 250), (203, 97), (66, 113)])
@pytest.mark.parametrize("T,omega", [(3, 1.5), (4, 1.9)])
def test_bf16_tiles_and_relaxation(shape, T, omega):
    """BF16 storage across several tiles (64 rows x 112 columns) with ragged
    edges and partial last launches: every update is rounded to BF16, so the
    result follows the FP64 oracle within 2e-2 on a smooth field."""
    R, C = shape
    g = inputs.sinusoid_field(max(R, C), seed=R + C, k_max=1)[:R, :C]
    x = torch.from_numpy(np.ascontiguousarray(g)).to(torch.bfloat16).cuda()
    check(run(x, T, omega), x, T, omega, BF16)


def _bf16_rne(x):
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)


def _sor_fp32_order(g32, T, omega, bf16=False):
    """Red-black SOR in float32 with every operation rounded on its own, in
    the order the FP32 path states: q = (n + s) + (w + e), then
    (1 - omega) * c + (omega / 4) * q, with the two coefficients rounded from
    double once; BF16 storage rounds each new value to BF16."""
    A = np.array(g32, dtype=np.float32)
    R, C = A.shape
    a, b = np.float32(1.0 - omega), np.float32(0.25 * omega)
    for _ in range(T):
        for colour in (0, 1):
            for i in range(1, R - 1):
                js = np.arange(1 + ((i + 1 + colour) & 1), C - 1, 2)
                q = (A[i - 1, js] + A[i + 1, js]) + (A[i, js - 1] + A[i, js + 1])
                v = a * A[i, js] + b * q
                A[i, js] = _bf16_rne(v) if bf16 else v
    return A


@pytest.mark.parametrize("dt", [F32, BF16])
@pytest.mark.parametrize("shape", [(37, 130), (150, 60)])
def test_fp32_operation_order_bitwise(shape, dt):
    """The FP32 arithmetic (FP32 and BF16 storage) is exactly the stated
    sequence of separately rounded operations: no multiply is fused with an
    add.  Checked bit for bit against that sequence in numpy, across tile
    edges and a partial last launch (T = 6)."""
    T, om = 6, 1.7
    g = np.random.default_rng(sum(shape)).random(shape)
    x = torch.from_numpy(g).float().cuda()
    if dt == BF16:
        x = x.to(torch.bfloat16)
    want = _sor_fp32_order(x.float().cpu().numpy(), T, om, bf16=(dt == BF16))
    got = run(x, T, om).float().cpu().numpy()
    diff = got != want
    assert not diff.any(), (int(diff.sum()), float(np.abs(got - want).max()), np.argwhere(diff)[:4].tolist())


def test_in_place_odd_and_even_T():
    g = np.random.default_rng(4).random((90, 250))
    for T in (1, 4, 5):
        x = torch.from_numpy(g).float().cuda()
        x0 = x.clone()
        binding.sor2d(x, x, T, 1.3)
        torch.cuda.synchronize()
        assert binding.sdfg_device_error(True) == 0
        check(x, x0, T, 1.3, F32)


def test_pitched_and_unaligned_layouts():
    R, C, T, om = 70, 101, 5, 1.2
    g = np.random.default_rng(5).random((R, C))
    buf = torch.zeros((R, 128), device="cuda")
    buf[:, :C] = torch.from_numpy(g).float().cuda()
    x = buf[:, :C]
    y = run(x, T, om, out=torch.zeros_like(buf)[:, :C])
    check(y, x, T, om, F32)
    flat = torch.zeros(R * C + 1, device="cuda")
    xu = flat[1:].view(R, C)
    xu.copy_(torch.from_numpy(g).float())
    assert torch.equal(run(xu, T, om), y.contiguous())


@pytest.mark.parametrize("shape", [(2, 9), (9, 2), (1, 1)])
def test_degenerate_shapes_copy(shape):
    x = torch.rand(shape, device="cuda")
    assert torch.equal(run(x, 5, 1.5), x)


def test_T0_empty_and_errors():
    x = torch.rand((20, 30), device="cuda")
    assert torch.equal(run(x, 0, 1.5), x)
    run(torch.empty((0, 7), device="cuda"), 3, 1.0)
    L = binding.lib()
    assert L.sdfg_sor2d(x.data_ptr(), x.data_ptr(), 20, 30, 30, -1, 1.0, F32, 0) == binding.SDFG_ERR_INVAL
    assert L.sdfg_sor2d(x.data_ptr(), x.data_ptr(), 20, 30, 29, 1, 1.0, F32, 0) == binding.SDFG_ERR_INVAL
    assert L.sdfg_sor2d(x.data_ptr(), x.data_ptr(), 20, 30, 30, 1, float("nan"), F32, 0) == binding.SDFG_ERR_INVAL
    assert L.sdfg_sor2d(None, None, 20, 30, 30, 1, 1.0, F32, 0) == binding.SDFG_ERR_INVAL


def test_full_size_8192_windows_and_harmonic_field():
    """The SOR benchmark grid (8192^2 FP32, omega 1.9): light-cone windows of
    a 20-iteration run against the oracle, and a discrete-harmonic field kept
    for the benchmark's 1000 iterations."""
    n, om = 8192, 1.9
    g = inputs.uniform_grid(n, n, seed=0)
    x = torch.from_numpy(g).float().cuda()
    T = 20
    y = run(x, T, om)
    xs = h64(x)
    m = 2 * T + 2
    for (r0, r1, c0, c1) in [(0, 8, 0, 8), (4000, 4010, 5000, 5010), (8184, 8192, 100, 110), (37, 45, 8184, 8192)]:
        cr0, cr1, cc0, cc1 = max(0, r0 - m), min(n, r1 + m), max(0, c0 - m), min(n, c1 + m)
        # the crop must keep every point's colour: its corner at an even i + j
        if (cr0 + cc0) % 2:
            if cr0 > 0:
                cr0 -= 1
            else:
                cc0 -= 1
        # a crop's artificial edge is at least m > 2T cells away from the window
        want = oracle.sor2d(xs[cr0:cr1, cc0:cc1], T, om)[r0 - cr0:r1 - cr0, c0 - cc0:c1 - cc0]
        got = y[r0:r1, c0:c1].double().cpu().numpy()
        assert np.abs(got - want).max() <= TOL[F32], (r0, c0)
    i = np.arange(n, dtype=np.float64)[:, None] / n
    j = np.arange(n, dtype=np.float64)[None, :] / n
    h = torch.from_numpy(i * i - j * j).float().cuda()
    hy = run(h, 1000, om)
    assert float((hy - h).abs().max()) <= TOL[F32]
