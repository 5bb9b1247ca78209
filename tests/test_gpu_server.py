"""The continuous-batching server through the C ABI: requests admitted under
an HBM budget and a slot limit, results identical alone and in the mix, and
equal to the FP64 oracle run for the reported step count."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return binding.lib()


def h64(t):
    return t.double().cpu().numpy()


class Server:
    def __init__(self, budget, slots, quantum, stride):
        self.L = binding.lib()
        self.h = ctypes.c_void_p()
        binding.check(self.L.sdfg_server_create(ctypes.byref(self.h), budget, slots, quantum, stride, 0))

    def submit(self, d):
        rid = ctypes.c_uint64()
        binding.check(self.L.sdfg_server_submit(self.h, ctypes.byref(d), ctypes.byref(rid)))
        return rid.value

    def poll(self, rid):
        out = binding.sdfg_desc()
        rc = self.L.sdfg_server_poll(self.h, rid, ctypes.byref(out))
        return rc, out

    def snapshot(self, rid):
        return self.L.sdfg_server_snapshot(self.h, rid)

    def drain(self, ms):
        return self.L.sdfg_server_drain(self.h, ms)

    def close(self):
        binding.check(self.L.sdfg_server_destroy(self.h))


def requests(n, seed, lo=32, hi=200):
    reqs = inputs.served_requests(n, seed=seed, lo=lo, hi=hi)
    out = []
    for r in reqs:
        g = inputs.laplace_request_grid(r)
        x = torch.from_numpy(g).float().cuda()
        out.append((r, x))
    return out


# the server's default geometry for FP32 grids: k = 4, 96-row segments
SERVER_CFG = dict(kernel=binding.SDFG_KERNEL_PERSISTENT, k=4, seg_rows=96, warps=4)


def solve_alone(x, T, tol, stride, t_start=0, r_first2=0.0, y=None):
    """The same request solved by itself (single-grid solve, the server's geometry)."""
    y = torch.zeros_like(x) if y is None else y
    d = binding.desc_for(x, y, T, tol, t_start=t_start, r_first2=r_first2)
    binding.check(binding.sdfg_jacobi2d_solve(d, stride, binding.config(**SERVER_CFG)))
    return y, d


@pytest.mark.parametrize("budget_mb,slots", [(4096, 64), (2, 3)])
def test_server_results_same_alone_and_in_mix(budget_mb, slots):
    stride, quantum, cap, tol = 32, 128, 3000, 1e-4
    reqs = requests(14, seed=3)
    sv = Server(budget_mb << 20, slots, quantum, stride)
    ys, ids = [], []
    try:
        for i, (r, x) in enumerate(reqs):
            y = torch.zeros_like(x)
            T = cap if i % 4 else 500              # some requests hit the cap
            t = tol if i % 5 else 0.0              # some run a fixed T
            d = binding.desc_for(x, y, T, t)
            ids.append(sv.submit(d))
            ys.append((y, T, t))
            if i == 6:
                time.sleep(0.01)                   # later requests arrive while others run
        assert sv.drain(120_000) == 0
        for rid, (r, x), (y, T, t) in zip(ids, reqs, ys):
            rc, res = sv.poll(rid)
            assert rc == 0 and res.status == 0
            ya, da = solve_alone(x, T, t, stride)
            assert res.steps_done == da.steps_done
            assert torch.equal(y, ya), "result differs alone vs in the mix"
            want = oracle.jacobi2d(h64(x), res.steps_done)
            assert np.abs(h64(y) - want).max() <= TOL32
            if t:
                _, steps_o, _, _ = oracle.jacobi2d_tol(h64(x), T, t, stride)
                assert abs(res.steps_done - steps_o) <= stride
            else:
                assert res.steps_done == T
    finally:
        sv.close()


def test_server_poll_pending_unknown_and_budget():
    sv = Server(1 << 20, 4, 64, 32)
    try:
        big = torch.zeros((1024, 1024), device="cuda")
        d = binding.desc_for(big, big, 100, 0.0)
        rid = ctypes.c_uint64()
        rc = sv.L.sdfg_server_submit(sv.h, ctypes.byref(d), ctypes.byref(rid))
        assert rc == binding.SDFG_ERR_NOMEM           # larger than the whole budget
        x = torch.rand((40, 40), device="cuda")
        y = torch.zeros_like(x)
        r1 = sv.submit(binding.desc_for(x, y, 64 * 50, 0.0))
        rc, _ = sv.poll(r1)
        assert rc in (binding.SDFG_PENDING, 0)
        assert sv.drain(60_000) == 0
        rc, res = sv.poll(r1)
        assert rc == 0 and res.steps_done == 64 * 50
        rc, _ = sv.poll(r1)                           # already collected
        assert rc == binding.SDFG_ERR_INVAL
        assert np.abs(h64(y) - oracle.jacobi2d(h64(x), 64 * 50)).max() <= TOL32
    finally:
        sv.close()


def test_snapshot_then_resume_equals_uninterrupted():
    """Pause a running solve at a wave boundary, resume it from its snapshot
    (grid, steps done, ||A_1 - A_0||^2), and get the uninterrupted result bit
    for bit."""
    stride, quantum, cap, tol = 32, 64, 6000, 1e-7
    r = inputs.Request(160, 150, seed=99)
    x = torch.from_numpy(inputs.laplace_request_grid(r)).float().cuda()
    y_full, d_full = solve_alone(x, cap, tol, stride)
    sv = Server(1 << 30, 4, quantum, stride)
    try:
        y = torch.zeros_like(x)
        rid = sv.submit(binding.desc_for(x, y, cap, tol))
        time.sleep(0.02)
        assert sv.snapshot(rid) == 0
        assert sv.drain(60_000) == 0
        rc, res = sv.poll(rid)
        if rc == 0:
            pytest.skip("the solve finished before the snapshot took effect")
        assert rc == binding.SDFG_PAUSED
        assert res.steps_done % quantum == 0 and 0 < res.steps_done < d_full.steps_done
        assert res.r_first2 > 0.0
        snap = y.clone()
        assert np.abs(h64(snap) - oracle.jacobi2d(h64(x), res.steps_done)).max() <= TOL32
        # resume through the server ...
        y2 = torch.zeros_like(x)
        rid2 = sv.submit(binding.desc_for(snap, y2, cap, tol, t_start=res.steps_done, r_first2=res.r_first2))
        assert sv.drain(60_000) == 0
        rc2, res2 = sv.poll(rid2)
        assert rc2 == 0 and res2.steps_done == d_full.steps_done
        assert torch.equal(y2, y_full)
        # ... and through the single-grid solve
        y3, d3 = solve_alone(snap, cap, tol, stride, t_start=res.steps_done, r_first2=res.r_first2)
        assert d3.steps_done == d_full.steps_done and torch.equal(y3, y_full)
    finally:
        sv.close()


def test_priority_admission_order():
    """With one slot, queued requests are admitted highest priority first."""
    sv = Server(1 << 30, 1, 64, 32)
    try:
        xs = [torch.rand((96, 96), device="cuda") for _ in range(4)]
        ys = [torch.zeros_like(x) for x in xs]
        ids = [sv.submit(binding.desc_for(xs[0], ys[0], 64 * 40, 0.0))]          # occupies the slot
        time.sleep(0.01)
        for i, prio in zip((1, 2, 3), (0, 5, 9)):
            ids.append(sv.submit(binding.desc_for(xs[i], ys[i], 64 * 2, 0.0, priority=prio)))
        order = []
        t0 = time.time()
        while len(order) < 4 and time.time() - t0 < 60:
            for i, rid in enumerate(ids):
                if i in order:
                    continue
                rc, _ = sv.poll(rid)
                if rc != binding.SDFG_PENDING:
                    assert rc == 0
                    order.append(i)
            time.sleep(0.0005)
        assert order == [0, 3, 2, 1], order
    finally:
        sv.close()
