"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances (max-abs against the FP64 oracle run on exactly the values the GPU
received): FP32 storage 1e-4, BF16 storage 2e-2, FP64 1e-12 (and bitwise, the
order of operations being the same).  FP32 units away from the boundary ring
reassociate the sum, so FP32 results are bit-identical for equal geometry
(fused depth k and segment height): the per-pass and persistent kernels must
agree bit for bit in that case.

Full-size cases (8192^2, T=1000) are checked on light-cone windows: the
oracle runs on a crop that extends T+1 cells past each window, which fixes the
window's values exactly; plus transpose symmetry and the maximum principle,
which hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

F32, BF16, F64 = binding.SDFG_F32, binding.SDFG_BF16, binding.SDFG_F64
TDT = {F32: torch.float32, BF16: torch.bfloat16, F64: torch.float64}
TOL = {F32: 1e-4, BF16: 2e-2, F64: 1e-12}
NAIVE = binding.SDFG_KERNEL_NAIVE
TEMPORAL = binding.SDFG_KERNEL_TEMPORAL


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = binding.lib()
    binding.sdfg_device_error(True)
    return L


def dev(grid64, dt, ld=None):
    t = torch.from_numpy(np.ascontiguousarray(grid64)).to(TDT[dt])
    R, C = t.shape
    if ld is None or ld == C:
        return t.cuda()
    buf = torch.zeros((R, ld), dtype=TDT[dt], device="cuda")
    buf[:, :C] = t.cuda()
    return buf[:, :C]


def host64(t):
    return t.double().cpu().numpy()


def run(inp, T, cfg=None, out=None, inplace=False):
    if inplace:
        out = inp
    elif out is None:
        out = torch.empty_like(inp) if inp.is_contiguous() else dev(np.zeros(inp.shape), binding.dtype_code(inp),
                                                                     inp.stride(0))
    binding.jacobi2d(inp, out, T, cfg)
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    return out


def cfg(kernel, k=0, seg_rows=0, warps=0):
    return binding.config(kernel=kernel, k=k, seg_rows=seg_rows, warps=warps)


PERSISTENT = binding.SDFG_KERNEL_PERSISTENT
SKEWED = binding.SDFG_KERNEL_SKEWED
# the chain kernel at several depths and chain lengths (short chains put many
# chain seams, and tiny first/last chains, into small grids)
SKEWED_CFGS = [cfg(SKEWED, 8), cfg(SKEWED, 8, seg_rows=32), cfg(SKEWED, 4, seg_rows=24), cfg(SKEWED, 2, seg_rows=8),
               cfg(SKEWED, 1, seg_rows=4)]
ALL_CFGS = [cfg(NAIVE)] + [cfg(TEMPORAL, k) for k in (1, 2, 4, 8)] + [cfg(TEMPORAL, 8, seg_rows=16, warps=4),
                                                                     cfg(TEMPORAL, 4, seg_rows=24, warps=2)] + SKEWED_CFGS
# (per-pass, persistent) pairs with the same geometry: bit-identical results
SAME_GEOMETRY = [(cfg(TEMPORAL, 8, seg_rows=24, warps=4), cfg(PERSISTENT, 8, seg_rows=24, warps=4)),
                 (cfg(TEMPORAL, 4, seg_rows=48, warps=2), cfg(PERSISTENT, 4, seg_rows=48, warps=4))]


@pytest.mark.parametrize("shape", [(3, 3), (4, 4), (5, 7), (9, 130), (17, 33), (64, 64), (129, 131), (200, 515),
                                   (40, 1100)])
@pytest.mark.parametrize("T", [1, 5, 16, 37])
def test_f32_matches_oracle_all_kernels(shape, T):
    R, C = shape
    g = inputs.uniform_grid(R, C, seed=R * 1000 + C)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), T, threads=0)
    for c in ALL_CFGS:
        y = host64(run(x, T, c))
        err = np.abs(y - want).max()
        assert err <= TOL[F32], (shape, T, c.kernel, c.k, err)
    for c1, c2 in SAME_GEOMETRY:
        assert np.array_equal(host64(run(x, T, c1)), host64(run(x, T, c2))), "same geometry, different bits"
    # input untouched
    assert np.array_equal(host64(x), g.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("dt", [BF16, F64])
@pytest.mark.parametrize("shape,T", [((33, 70), 9), ((130, 257), 21), ((300, 1000), 40)])
def test_other_dtypes_match_oracle(dt, shape, T):
    R, C = shape
    # same smoothness as the 16384^2 precision workload (wavelengths >= 256 cells)
    n = max(R, C)
    g = inputs.sinusoid_field(n, seed=3, k_max=max(1, n // 256))[:R, :C]
    x = dev(g, dt)
    want = oracle.jacobi2d(host64(x), T, threads=0)
    outs = []
    for c in [cfg(NAIVE), cfg(TEMPORAL, 1), cfg(TEMPORAL, 2), cfg(TEMPORAL, 4), cfg(TEMPORAL, 8)] + SKEWED_CFGS:
        y = host64(run(x, T, c))
        err = np.abs(y - want).max()
        assert err <= TOL[dt], (dt, shape, T, c.k, err)
        outs.append(y)
    if dt == F64:
        for y in outs[1:]:
            assert np.array_equal(y, outs[0])
        assert np.array_equal(outs[0], want), "FP64 path should equal the oracle bit for bit"
    else:
        # BF16 rounds when a pass stores; the persistent kernel with the same
        # geometry as the per-pass kernel agrees bit for bit
        for c1, c2 in SAME_GEOMETRY:
            assert np.array_equal(host64(run(x, T, c1)), host64(run(x, T, c2)))


def test_f64_256_grid_T100_bitwise():
    g = inputs.uniform_grid(256, 256, seed=0)
    x = dev(g, F64)
    want = oracle.jacobi2d(g, 100)
    y = host64(run(x, 100))
    assert np.abs(y - want).max() <= TOL[F64]
    assert np.array_equal(y, want)


def test_f32_256_grid_T100():
    g = inputs.uniform_grid(256, 256, seed=0)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), 100)
    assert np.abs(host64(run(x, 100)) - want).max() <= TOL[F32]


@pytest.mark.parametrize("T", [6, 8, 9, 16, 17])
def test_in_place(T):
    g = inputs.uniform_grid(70, 90, seed=T)
    want = oracle.jacobi2d(g.astype(np.float32).astype(np.float64), T)
    for c in [cfg(TEMPORAL, 8), cfg(TEMPORAL, 4), cfg(NAIVE), cfg(SKEWED, 8, seg_rows=32), cfg(SKEWED, 4, seg_rows=16)]:
        x = dev(g, F32)
        run(x, T, c, inplace=True)
        assert np.abs(host64(x) - want).max() <= TOL[F32]


@pytest.mark.parametrize("ld_extra", [4, 12, 3, 1])
def test_pitched_and_unaligned_layouts(ld_extra):
    # ld*4 % 16 == 0 for extra 4/12 (TMA reads the caller's buffers directly);
    # 3 and 1 need the staged path
    R, C, T = 50, 68, 13
    g = inputs.uniform_grid(R, C, seed=ld_extra)
    x = dev(g, F32, ld=C + ld_extra)
    want = oracle.jacobi2d(host64(x), T)
    for c in [cfg(TEMPORAL, 4), cfg(SKEWED, 4, seg_rows=16)]:
        y = dev(np.zeros((R, C)), F32, ld=C + ld_extra)
        run(x, T, c, out=y)
        assert np.abs(host64(y) - want).max() <= TOL[F32], c.kernel


@pytest.mark.parametrize("cols", [61, 127, 129, 8190 // 64])
def test_ragged_widths(cols):
    R, T = 45, 11
    g = inputs.uniform_grid(R, cols, seed=cols)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), T)
    for c in [cfg(TEMPORAL, 8), cfg(TEMPORAL, 2), cfg(SKEWED, 8, seg_rows=32)]:
        assert np.abs(host64(run(x, T, c)) - want).max() <= TOL[F32]


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (2, 9), (9, 2), (2, 2), (3, 40)])
def test_degenerate_shapes(shape):
    g = inputs.uniform_grid(*shape, seed=1)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), 7)
    got = host64(run(x, 7))
    if min(shape) < 3:
        assert np.array_equal(got, want)       # no interior: an exact copy
    else:
        assert np.abs(got - want).max() <= TOL[F32]


def test_T0_and_empty():
    g = inputs.uniform_grid(20, 30, seed=2)
    x = dev(g, F32)
    assert np.array_equal(host64(run(x, 0)), host64(x))
    e = torch.empty((0, 5), device="cuda")
    binding.check(binding.sdfg_jacobi2d(e.data_ptr(), e.data_ptr(), 0, 5, 3, 0))


def test_raw_entry_point_and_host_call():
    R, C, T = 96, 160, 24
    g = inputs.uniform_grid(R, C, seed=11)
    x = dev(g, F32)
    y = torch.empty_like(x)
    binding.check(binding.sdfg_jacobi2d(x.data_ptr(), y.data_ptr(), R, C, T, torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    want = oracle.jacobi2d(host64(x), T)
    assert np.abs(host64(y) - want).max() <= TOL[F32]
    hi = x.cpu().pin_memory()
    ho = torch.empty_like(hi).pin_memory()
    binding.check(binding.sdfg_jacobi2d_host(hi.data_ptr(), ho.data_ptr(), R, C, T, F32, 0))
    assert np.array_equal(ho.double().numpy(), host64(y))


@pytest.mark.parametrize("shape,T", [((96, 160), 24), ((1100, 1300), 37)])
def test_host_many_pipelined_equals_host_calls(shape, T):
    """Pipelined host solves (two device slots, two streams): each result
    equals the one-call result bit for bit, and the oracle within 1e-4; the
    1100 x 1300 grid runs the chain kernel."""
    R, C = shape
    his = [torch.from_numpy(inputs.uniform_grid(R, C, seed=20 + i)).float().pin_memory() for i in range(3)]
    hos = [torch.empty_like(h).pin_memory() for h in his]
    stream = torch.cuda.current_stream().cuda_stream
    binding.check(binding.sdfg_jacobi2d_host_many([h.data_ptr() for h in his], [h.data_ptr() for h in hos],
                                                  R, C, T, F32, stream))
    for i, (hi, ho) in enumerate(zip(his, hos)):
        one = torch.empty_like(hi).pin_memory()
        binding.check(binding.sdfg_jacobi2d_host(hi.data_ptr(), one.data_ptr(), R, C, T, F32, stream))
        assert torch.equal(ho, one), i
    want = oracle.jacobi2d(his[2].double().numpy(), T, threads=0)
    assert np.abs(hos[2].double().numpy() - want).max() <= TOL[F32]
    assert binding.sdfg_jacobi2d_host_many([], [], R, C, T, F32, stream) == binding.SDFG_OK
    assert binding.sdfg_jacobi2d_host_many([his[0].data_ptr()], [0], R, C, T, F32, stream) == binding.SDFG_ERR_INVAL


def test_full_size_8192_T1000_windows_and_properties():
    """The bench workload: 8192^2 FP32, T=1000, in the bench's launch config."""
    R = C = 8192
    T = 1000
    g = inputs.uniform_grid(R, C, seed=0)
    x = dev(g, F32)
    bench_cfg = binding.config(kernel=binding.SDFG_KERNEL_PERSISTENT, k=8, seg_rows=128, warps=4)
    y = run(x, T, bench_cfg)
    yh = y.cpu().numpy()
    xh = x.cpu().numpy().astype(np.float64)
    for (r0, c0) in [(0, 0), (0, C - 24), (R - 24, 0), (R - 24, C - 24), (4000, 4100), (0, 3000), (5000, C - 24)]:
        w = oracle.jacobi2d_window(xh, T, r0, r0 + 24, c0, c0 + 24, threads=0)
        err = np.abs(yh[r0:r0 + 24, c0:c0 + 24].astype(np.float64) - w).max()
        assert err <= TOL[F32], (r0, c0, err)
    # discrete maximum principle
    assert yh.min() >= xh.min() - 1e-6 and yh.max() <= xh.max() + 1e-6
    # transpose symmetry (bit for bit in exact arithmetic; the reassociated
    # FP32 sum makes it hold to the FP32 tolerance)
    yt = run(x.t().contiguous(), T, bench_cfg)
    assert (yt.t().double() - y.double()).abs().max().item() <= TOL[F32]
    # boundary ring untouched
    assert torch.equal(y[0], x[0]) and torch.equal(y[-1], x[-1])
    assert torch.equal(y[:, 0], x[:, 0]) and torch.equal(y[:, -1], x[:, -1])


def test_full_size_8192_T1000_whole_grid():
    """The bench workload in the bench's launch configuration (persistent
    kernel, k = 8, 128-row segments, 4 warps per CTA), compared with the FP64
    oracle on EVERY element: every unit seam of the reassociated interior
    units, the edge units and the boundary ring.  The oracle runs the whole
    grid on all host threads."""
    R = C = 8192
    T = 1000
    g = inputs.uniform_grid(R, C, seed=0)
    x = dev(g, F32)
    bench_cfg = binding.config(kernel=binding.SDFG_KERNEL_PERSISTENT, k=8, seg_rows=128, warps=4)
    y = host64(run(x, T, bench_cfg))
    want = oracle.jacobi2d(host64(x), T, threads=0)
    err = np.abs(y - want)
    assert err.max() <= TOL[F32], (float(err.max()), np.unravel_index(int(err.argmax()), err.shape))


@pytest.mark.parametrize("shape", [(520, 520), (530, 700), (400, 1130)])
@pytest.mark.parametrize("T", [8, 37, 64])
def test_bench_geometry_multi_seam_whole(shape, T):
    """The bench's geometry (k = 8, 128-row segments) on grids of at least
    three segments and three strips, so that reassociated interior units and
    all their seams (128-row and 112-column) are compared whole with the
    oracle, for the streamed and the persistent kernel; T = 37 adds the
    remainder passes (4 + 1 steps).  The two kernels run the same units and
    must agree bit for bit."""
    R, C = shape
    g = inputs.uniform_grid(R, C, seed=R + 7 * C + T)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), T, threads=0)
    outs = []
    for kern in (TEMPORAL, PERSISTENT):
        y = host64(run(x, T, cfg(kern, 8, seg_rows=128, warps=4)))
        err = np.abs(y - want).max()
        assert err <= TOL[F32], (shape, T, kern, err)
        outs.append(y)
    assert np.array_equal(outs[0], outs[1]), "same geometry, different bits"
    info = binding.sdfg_plan_geometry(R, C, F32, 8, 128)
    assert info["n_strips"] >= 3 and info["n_segs"] >= 3, info


@pytest.mark.parametrize("shape,L", [((2100, 700), 1024), ((1300, 1130), 256), ((777, 333), 100)])
@pytest.mark.parametrize("T", [8, 37, 96])
def test_skewed_chains_whole(shape, L, T):
    """The chain kernel (chains of L rows skewed down by k rows per pass,
    chunk-level dependencies): several chains and strips, compared whole
    with the oracle; T = 37 adds remainder passes (8 x 4 + 4 + 1), whose
    depths change from pass to pass; the boundary ring comes out exact; and
    a repeat call (cached plan, counters reset) gives the same bits."""
    R, C = shape
    g = inputs.uniform_grid(R, C, seed=R + C + T)
    x = dev(g, F32)
    want = oracle.jacobi2d(host64(x), T, threads=0)
    c = cfg(SKEWED, 8, seg_rows=L)
    y1 = run(x, T, c)
    err = np.abs(host64(y1) - want).max()
    assert err <= TOL[F32], (shape, L, T, err)
    assert torch.equal(y1[0], x[0]) and torch.equal(y1[-1], x[-1])
    assert torch.equal(y1[:, 0], x[:, 0]) and torch.equal(y1[:, -1], x[:, -1])
    y2 = run(x, T, c)
    assert torch.equal(y1, y2)


def test_skewed_full_size_8192_T1000_whole_grid():
    """The chain kernel on the bench workload in the bench's launch
    configuration (k = 8, 640-row chains, the library default), against the
    FP64 oracle on every element."""
    R = C = 8192
    T = 1000
    x = dev(inputs.uniform_grid(R, C, seed=0), F32)
    y = host64(run(x, T, cfg(SKEWED, 8, seg_rows=640)))
    want = oracle.jacobi2d(host64(x), T, threads=0)
    err = np.abs(y - want)
    assert err.max() <= TOL[F32], (float(err.max()), np.unravel_index(int(err.argmax()), err.shape))


def test_paper_workload_eigenmode_2048_T1024():
    """Zero boundary, 2048^2, T=1024 (the paper's Jacobi workload), on a
    closed-form eigenmode: the amplitude after T steps is lambda^T."""
    import math
    R = C = 2048
    T = 1024
    g = inputs.eigenmode(R, C, 3, 5)
    lam = 0.2 + 0.4 * (math.cos(3 * math.pi / (R - 1)) + math.cos(5 * math.pi / (C - 1)))
    x = dev(g, F32)
    y = host64(run(x, T))
    want = (lam ** T) * host64(x)
    assert np.abs(y - want).max() <= TOL[F32]
    # the configuration the benchmark times: the autotuner's choice for this shape
    cfg = binding.sdfg_autotune(R, C, T, F32, torch.cuda.current_stream().cuda_stream)
    y = host64(run(x, T, cfg))
    assert np.abs(y - want).max() <= TOL[F32], (cfg.kernel, cfg.k, cfg.seg_rows)
    # and the benchmark's input (uniform interior, zero ring), on light-cone windows
    u = inputs.uniform_grid(R, C, seed=0)
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    xu = dev(u, F32)
    yu = run(xu, T, cfg)
    xs = host64(xu)
    for r0, c0 in [(0, 0), (1000, 700), (2040, 2040), (5, 2040)]:
        want_w = oracle.jacobi2d_window(xs, T, r0, r0 + 8, c0, c0 + 8, threads=0)
        got_w = host64(yu[r0:r0 + 8, c0:c0 + 8])
        assert np.abs(got_w - want_w).max() <= TOL[F32], (r0, c0)


@pytest.mark.parametrize("dt,T1,T2", [(F64, 7, 13), (F64, 40, 1), (F32, 16, 21), (F32, 64, 64)])
def test_resume_equals_uninterrupted(dt, T1, T2):
    """Checkpoint/resume: the state of a solve is exactly (grid, t), so
    running T1 steps, then T2 more from the result, equals T1 + T2 steps.
    Bitwise for FP64 at any split; for FP32 when T1 is a multiple of k (the
    passes, and so the rounding, are then the same)."""
    g = inputs.uniform_grid(300, 260, seed=T1)
    c = binding.config(kernel=binding.SDFG_KERNEL_PERSISTENT, k=8 if dt == F32 else 4, seg_rows=64)
    x = dev(g, dt)
    mid = run(x, T1, c)
    a = run(mid, T2, c)
    b = run(x, T1 + T2, c)
    assert torch.equal(a, b)
    assert np.abs(host64(b) - oracle.jacobi2d(host64(x), T1 + T2)).max() <= TOL[dt]
