"""Batch paths through the C ABI: batches of uneven grids on the persistent
and on the chain kernel, CUDA graph replay, tolerance solves (data-dependent
stop), the bounded-wait failure path, and the single-grid persistent kernel.

Every result is compared with the FP64 oracle; fixed-step results must also
equal the single-grid temporal kernel bit for bit (the same order of
operations), and tolerance solves must stop within one check stride of the
oracle's stopping step and match the oracle run for exactly the GPU's step
count."""
import math

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


def dev(g, dt, ld=None):
    t = torch.from_numpy(np.ascontiguousarray(g)).to(TDT[dt])
    R, C = t.shape
    if ld is None or ld == C:
        return t.cuda()
    buf = torch.zeros((R, ld), dtype=TDT[dt], device="cuda")
    buf[:, :C] = t.cuda()
    return buf[:, :C]


def h64(t):
    return t.double().cpu().numpy()


def alloc_like(x):
    if x.is_contiguous():
        return torch.zeros_like(x)
    buf = torch.zeros((x.shape[0], x.stride(0)), dtype=x.dtype, device="cuda")
    return buf[:, :x.shape[1]]


def temporal_ref(x, T, seg_rows=96):
    """Per-pass kernel with the batch's default geometry (k=8, 96-row segments)."""
    y = alloc_like(x)
    binding.jacobi2d(x, y, T, binding.config(kernel=binding.SDFG_KERNEL_TEMPORAL, k=8, seg_rows=seg_rows))
    torch.cuda.synchronize()
    return y


def make_batch(seed=0):
    r = np.random.default_rng(seed)
    shapes = [(64, 64), (70, 131), (257, 96), (3, 50), (2, 40), (130, 130), (33, 517), (400, 77), (19, 19),
              (200, 301)]
    grids = []
    for i, (R, C) in enumerate(shapes):
        g = inputs.uniform_grid(R, C, seed=100 + i)
        ld = C + (3 if i == 7 else (4 if i == 2 else 0))   # one staged (unaligned), one pitched
        T = int(r.integers(0 if i == 8 else 5, 90))
        grids.append((g, ld, T))
    return grids


def test_batch_fixed_steps_matches_oracle_and_single_kernel():
    xs, ys, descs, specs = [], [], [], make_batch()
    for i, (g, ld, T) in enumerate(specs):
        x = dev(g, F32, ld)
        y = x if i == 5 else alloc_like(x)          # one in-place grid
        x0 = x.clone() if i == 5 else x
        xs.append(x0)
        ys.append(y)
        descs.append(binding.desc_for(x, y, T))
    ref = [temporal_ref(x, T) for x, (g, ld, T) in zip(xs, specs)]
    binding.check(binding.sdfg_jacobi2d_batch(descs, 64, torch.cuda.current_stream().cuda_stream))
    for i, ((g, ld, T), x, y, d) in enumerate(zip(specs, xs, ys, descs)):
        assert d.status == 0
        want = oracle.jacobi2d(h64(x), T)
        got = h64(y)
        assert np.abs(got - want).max() <= TOL[F32], (i, np.abs(got - want).max())
        assert torch.equal(y, ref[i]), f"grid {i}: batch and single-grid kernels disagree"


def _plan_run(descs, cfg, runs=1):
    """Build a plan over `descs` with `cfg`, run it `runs` times, fill the outputs."""
    import ctypes
    L = binding.lib()
    arr = (binding.sdfg_desc * len(descs))(*descs)
    plan = ctypes.c_void_p()
    binding.check(L.sdfg_batch_plan_create(ctypes.byref(plan), arr, len(descs), 64, ctypes.byref(cfg), 0))
    try:
        for _ in range(runs):
            binding.check(L.sdfg_batch_plan_run(plan, torch.cuda.current_stream().cuda_stream))
        binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    finally:
        binding.check(L.sdfg_batch_plan_destroy(plan))
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    return list(arr)


@pytest.mark.parametrize("k,L", [(8, 512), (8, 32), (4, 24), (2, 16)])
@pytest.mark.parametrize("dt", [F32, BF16, F64])
def test_chain_batch_matches_oracle(k, L, dt):
    """Fixed-step batches on the chain kernel: uneven grids (tiny, non-square,
    one pitched, one unaligned and so staged, one in place, one with T = 0),
    step counts with remainder passes, short chains so that grids hold several
    chains; every grid whole against the FP64 oracle (FP64 bit for bit), and
    a second run of the same plan gives the same bits."""
    if dt == F64 and k > 4:
        k = 4
    xs, ys, descs, specs = [], [], [], make_batch(3)
    for i, (g, ld, T) in enumerate(specs):
        x = dev(g, dt, ld)
        y = x if i == 5 else alloc_like(x)
        x0 = x.clone() if i == 5 else x
        xs.append(x0)
        ys.append(y)
        descs.append(binding.desc_for(x, y, T))
    cfg = binding.config(kernel=binding.SDFG_KERNEL_SKEWED, k=k, seg_rows=96)
    binding.check(binding.sdfg_test_hook(3, 0))      # every fixed-step grid on chains ...
    binding.check(binding.sdfg_test_hook(4, L))      # ... of L rows
    try:
        out = _plan_run(descs, cfg)
        firsts = [y.clone() for y in ys]
        ys[5].copy_(xs[5])                           # grid 5 is in place: restore its input
        _plan_run(descs, cfg)                        # and replay
    finally:
        binding.sdfg_test_hook(3, -1)
        binding.sdfg_test_hook(4, 0)
    for a, b in zip(firsts, ys):
        assert torch.equal(a, b)
    for i, ((g, ld, T), x, y, d) in enumerate(zip(specs, xs, ys, out)):
        assert d.status == 0 and d.steps_done == T
        want = oracle.jacobi2d(h64(x), T)
        err = np.abs(h64(y) - want).max()
        if dt == F64:
            assert np.array_equal(h64(y), want), (i, err)
        else:
            assert err <= TOL[dt], (i, (g.shape, ld, T), err)
        # the boundary ring comes out exact
        assert torch.equal(y[0], x[0]) and torch.equal(y[-1], x[-1])
        assert torch.equal(y[:, 0], x[:, 0]) and torch.equal(y[:, -1], x[:, -1])


def test_hybrid_batch_with_tolerance_grids():
    """SDFG_KERNEL_SKEWED on a mixed batch: fixed-step grids above the size
    threshold on chains, the rest (and every tolerance solve) on the
    persistent kernel, in one plan; each result against the oracle, and each
    tolerance solve equal to the same solve alone on the persistent kernel."""
    specs = make_batch(5)
    xs, ys, descs = [], [], []
    for i, (g, ld, T) in enumerate(specs):
        x = dev(g, F32, ld)
        xs.append(x)
        ys.append(alloc_like(x))
        descs.append(binding.desc_for(x, ys[-1], T + 200, 1e-3) if i % 3 == 0 else binding.desc_for(x, ys[-1], T))
    cfg = binding.config(kernel=binding.SDFG_KERNEL_SKEWED, k=8, seg_rows=96)
    binding.check(binding.sdfg_test_hook(3, 10000))  # grids of >= 10000 points on chains
    binding.check(binding.sdfg_test_hook(4, 64))
    try:
        out = _plan_run(descs, cfg)
    finally:
        binding.sdfg_test_hook(3, -1)
        binding.sdfg_test_hook(4, 0)
    for i, ((g, ld, T), x, y, d) in enumerate(zip(specs, xs, ys, out)):
        assert d.status == 0
        want = oracle.jacobi2d(h64(x), d.steps_done)
        assert np.abs(h64(y) - want).max() <= TOL[F32], i
        if i % 3 == 0 and min(g.shape) >= 3:
            alone = alloc_like(x)
            da = binding.desc_for(x, alone, T + 200, 1e-3)
            binding.check(binding.sdfg_jacobi2d_solve(da, 64, binding.config(kernel=3, k=8, seg_rows=96)))
            assert da.steps_done == d.steps_done and torch.equal(alone, y), i
        elif min(g.shape) >= 3:
            assert d.steps_done == T


def test_batch_plan_graph_replay():
    specs = make_batch(1)
    xs = [dev(g, F32, ld) for g, ld, T in specs]
    ys = [alloc_like(x) for x in xs]
    descs = [binding.desc_for(x, y, T) for x, y, (g, ld, T) in zip(xs, ys, specs)]
    L = binding.lib()
    arr = (binding.sdfg_desc * len(descs))(*descs)
    plan = binding.ctypes.c_void_p()
    binding.check(L.sdfg_batch_plan_create(binding.ctypes.byref(plan), arr, len(descs), 64, None, 0))
    s = torch.cuda.current_stream().cuda_stream
    binding.check(L.sdfg_batch_plan_run(plan, s))
    binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    first = [y.clone() for y in ys]
    for y in ys:
        y.zero_()
    binding.check(L.sdfg_batch_plan_run(plan, s))
    binding.check(L.sdfg_batch_plan_run(plan, s))
    binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    binding.check(L.sdfg_batch_plan_destroy(plan))
    for a, b, x, (g, ld, T) in zip(first, ys, xs, specs):
        assert torch.equal(a, b)
        assert np.abs(h64(b) - oracle.jacobi2d(h64(x), T)).max() <= TOL[F32]


def _lam(R, C, p, q):
    return 0.2 + 0.4 * (math.cos(p * math.pi / (R - 1)) + math.cos(q * math.pi / (C - 1)))


@pytest.mark.parametrize("k", [8, 4])
def test_solve_stops_at_closed_form_step(k):
    R, C = 40, 57
    g = inputs.eigenmode(R, C, 1, 1)
    lam = _lam(R, C, 1, 1)
    tol, stride, cap = 1e-4, 16, 20000
    t_pred = next(t for t in range(stride, cap + 1, stride) if lam ** (t - 1) <= tol)
    x = dev(g, F64)
    y = torch.zeros_like(x)
    d = binding.desc_for(x, y, cap, tol)
    binding.check(binding.sdfg_jacobi2d_solve(d, stride, binding.config(kernel=3, k=k)))
    assert d.status == 0
    assert d.steps_done == t_pred, (d.steps_done, t_pred)
    assert abs(d.rel_residual - lam ** (t_pred - 1)) <= 1e-9 * lam ** (t_pred - 1)
    want, steps_o, rel_o, _ = oracle.jacobi2d_tol(g, cap, tol, stride)
    assert steps_o == t_pred
    assert np.array_equal(h64(y), want)


def test_solve_random_matches_oracle():
    R, C = 90, 133
    g = inputs.laplace_request_grid(inputs.Request(R, C, seed=7))
    x = dev(g, F32)
    y = torch.zeros_like(x)
    tol, stride, cap = 1e-3, 32, 4000
    d = binding.desc_for(x, y, cap, tol)
    binding.check(binding.sdfg_jacobi2d_solve(d, stride))
    _, steps_o, rel_o, _ = oracle.jacobi2d_tol(h64(x), cap, tol, stride)
    assert abs(d.steps_done - steps_o) <= stride, (d.steps_done, steps_o)
    want = oracle.jacobi2d(h64(x), d.steps_done)
    assert np.abs(h64(y) - want).max() <= TOL[F32]
    assert abs(d.rel_residual - rel_o) <= 1e-3 * rel_o + 1e-9 or d.steps_done != steps_o


@pytest.mark.parametrize("shape,tol,cap", [((90, 133), 1e-3, 40000), ((300, 260), 3e-2, 100000),
                                           ((64, 70), 1e-6, 3000)])
def test_solve_f64_residual_matches_oracle(shape, tol, cap):
    """FP64 storage: the states equal the oracle's bit for bit, the residual
    is squared and summed in FP64 from the first difference, so the stopping
    step is the oracle's and the reported relative residual agrees with the
    oracle's to FP64 rounding of the summation order (1e-12 relative)."""
    R, C = shape
    g = inputs.laplace_request_grid(inputs.Request(R, C, seed=11))
    x = dev(g, F64)
    y = torch.zeros_like(x)
    stride = 32
    d = binding.desc_for(x, y, cap, tol)
    binding.check(binding.sdfg_jacobi2d_solve(d, stride))
    want, steps_o, rel_o, _ = oracle.jacobi2d_tol(h64(x), cap, tol, stride, threads=0)
    assert d.steps_done == steps_o, (d.steps_done, steps_o)
    assert abs(d.rel_residual - rel_o) <= 1e-12 * rel_o, (d.rel_residual, rel_o)
    assert np.array_equal(h64(y), want)


def test_solve_bf16_invariants():
    """BF16 storage rounds the grid each time a pass stores it (every k
    steps), so on a Laplace solve with boundary values near +-1 (ulp 2^-7)
    increments below half an ulp per pass stall and the state drifts from the
    FP64 trajectory; the FP64-oracle tolerance does not apply.
    What must hold: the stop rule (rel <= tol at a check step, or the cap),
    the discrete maximum principle up to one BF16 ulp, an untouched boundary,
    and the same result alone as in a batch."""
    R, C = 90, 133
    x = dev(inputs.laplace_request_grid(inputs.Request(R, C, seed=7)), BF16)
    y = torch.zeros_like(x)
    tol, stride, cap = 1e-3, 32, 4000
    d = binding.desc_for(x, y, cap, tol)
    # the batch's default geometry (k=8, 96-row segments), for the comparison below
    binding.check(binding.sdfg_jacobi2d_solve(d, stride, binding.config(kernel=3, k=8, seg_rows=96)))
    assert 0 < d.steps_done <= cap
    assert d.steps_done == cap or (d.steps_done % stride == 0 and d.rel_residual <= tol)
    xh, yh = h64(x), h64(y)
    assert yh.min() >= xh.min() - 2 ** -7 and yh.max() <= xh.max() + 2 ** -7
    assert np.array_equal(yh[0], xh[0]) and np.array_equal(yh[-1], xh[-1])
    assert np.array_equal(yh[:, 0], xh[:, 0]) and np.array_equal(yh[:, -1], xh[:, -1])
    y2 = torch.zeros_like(x)
    d2 = binding.desc_for(x, y2, cap, tol)
    binding.check(binding.sdfg_jacobi2d_batch([d2, binding.desc_for(x.clone(), torch.zeros_like(x), 64, 0.0)], stride))
    assert d2.steps_done == d.steps_done and torch.equal(y2, y)


def test_batch_mixed_tolerance_and_fixed():
    specs = [(48, 70, 3000, 1e-3), (100, 64, 120, 0.0), (65, 65, 3000, 1e-4), (30, 200, 77, 0.0)]
    xs, ys, descs = [], [], []
    for i, (R, C, T, tol) in enumerate(specs):
        g = inputs.laplace_request_grid(inputs.Request(R, C, seed=20 + i)) if tol else inputs.uniform_grid(R, C, i)
        x = dev(g, F32)
        y = torch.zeros_like(x)
        xs.append(x)
        ys.append(y)
        descs.append(binding.desc_for(x, y, T, tol))
    binding.check(binding.sdfg_jacobi2d_batch(descs, 32))
    for (R, C, T, tol), x, y, d in zip(specs, xs, ys, descs):
        if tol:
            _, steps_o, _, _ = oracle.jacobi2d_tol(h64(x), T, tol, 32)
            assert abs(d.steps_done - steps_o) <= 32
            # alone: the same grid solved by itself stops at the same step, bit for bit
            y1 = torch.zeros_like(x)
            d1 = binding.desc_for(x, y1, T, tol)
            binding.check(binding.sdfg_jacobi2d_batch([d1], 32))
            assert d1.steps_done == d.steps_done and torch.equal(y1, y)
        else:
            assert d.steps_done == T
        want = oracle.jacobi2d(h64(x), d.steps_done)
        assert np.abs(h64(y) - want).max() <= TOL[F32]


def test_bounded_wait_timeout_reports_and_recovers():
    g = inputs.uniform_grid(300, 300, seed=3)
    x = dev(g, F32)
    y = torch.zeros_like(x)
    binding.check(binding.sdfg_test_hook(2, 2_000_000))      # 2 ms waits
    binding.check(binding.sdfg_test_hook(1, 1))              # first item waits on a flag nothing sets
    try:
        rc = binding.sdfg_jacobi2d_batch([binding.desc_for(x, y, 40)], 64)
    finally:
        binding.sdfg_test_hook(1, 0)
        binding.sdfg_test_hook(2, 0)
    assert rc == binding.SDFG_ERR_TIMEOUT, rc
    # the context is still usable and the next run is correct
    d = binding.desc_for(x, y, 40)
    binding.check(binding.sdfg_jacobi2d_batch([d], 64))
    assert np.abs(h64(y) - oracle.jacobi2d(h64(x), 40)).max() <= TOL[F32]


@pytest.mark.parametrize("shape,T", [((129, 131), 37), ((64, 600), 16), ((300, 90), 9)])
def test_persistent_single_grid_equals_temporal(shape, T):
    g = inputs.uniform_grid(*shape, seed=5)
    for inplace in (False, True):
        x = dev(g, F32)
        ref = temporal_ref(x, T, seg_rows=128)
        y = x if inplace else torch.zeros_like(x)
        for _ in range(2):                                      # second call reuses the cached plan
            if inplace:
                y.copy_(dev(g, F32))
            binding.jacobi2d(y if inplace else x, y, T,
                             binding.config(kernel=binding.SDFG_KERNEL_PERSISTENT, k=8, seg_rows=128))
            torch.cuda.synchronize()
            assert binding.sdfg_device_error(True) == 0
            assert torch.equal(y, ref)


@pytest.mark.parametrize("kernel,k,seg,min_pts", [("persistent", 4, 256, -1), ("skewed", 8, 256, -1),
                                                  ("skewed", 4, 128, -1), ("skewed", 8, 256, 0)])
def test_full_512_grid_batch_in_the_bench_configuration(kernel, k, seg, min_pts):
    """The benchmark's batch (512 uneven grids, rows and columns log-uniform
    in [64, 2048], T in [50, 500], each grid pitched to 16-byte rows) in the
    configurations its autotuner chooses between, replayed from a plan: the
    persistent kernel at k = 4 with 256-row segments; the hybrid (grids of
    >= 2^20 points on 512-row chains, the rest on the persistent kernel) at
    k = 8 and k = 4; and every grid on chains:
    every grid runs exactly T steps, and every one of the 512 results matches
    the FP64 oracle on every element."""
    import ctypes
    specs = inputs.batch_specs(512, seed=0)
    xs, ys, descs = [], [], []
    for sp in specs:
        ld = (sp.cols + 3) // 4 * 4
        x = torch.zeros((sp.rows, ld), device="cuda")[:, :sp.cols]
        x.copy_(torch.from_numpy(inputs.batch_grid(sp)).float())
        y = torch.zeros((sp.rows, ld), device="cuda")[:, :sp.cols]
        xs.append(x)
        ys.append(y)
        descs.append(binding.desc_for(x, y, sp.T))
    L = binding.lib()
    arr = (binding.sdfg_desc * len(descs))(*descs)
    kern = binding.SDFG_KERNEL_PERSISTENT if kernel == "persistent" else binding.SDFG_KERNEL_SKEWED
    cfg = binding.config(kernel=kern, k=k, seg_rows=seg, warps=4)
    plan = ctypes.c_void_p()
    binding.check(binding.sdfg_test_hook(3, min_pts))
    try:
        binding.check(L.sdfg_batch_plan_create(ctypes.byref(plan), arr, len(descs), 64, ctypes.byref(cfg), 0))
        binding.check(L.sdfg_batch_plan_run(plan, torch.cuda.current_stream().cuda_stream))
        binding.check(L.sdfg_batch_plan_results(plan, arr, len(descs)))
    finally:
        binding.sdfg_test_hook(3, -1)
        binding.check(L.sdfg_batch_plan_destroy(plan))
    torch.cuda.synchronize()
    assert binding.sdfg_device_error(True) == 0
    for d, sp in zip(arr, specs):
        assert d.status == 0 and d.steps_done == sp.T
    # every grid whole against the oracle (all host threads)
    for g, (sp, x, y) in enumerate(zip(specs, xs, ys)):
        want = oracle.jacobi2d(h64(x), sp.T, threads=0)
        err = np.abs(h64(y) - want).max()
        assert err <= TOL[F32], (g, sp, err)
