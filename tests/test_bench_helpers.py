"""Host logic of bench.py, on the CPU: the timing contract's defaults, the
lookup of a kernel's DRAM traffic in the committed ncu summaries, the median
and its confidence interval, and the kernel-family names."""
import glob
import math
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_keep_the_timing_contract(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.workload == "single"
    assert a.warmup >= 3 and a.steps >= 1
    assert (a.rows, a.cols, a.T) == (8192, 8192, 1000)
    assert bench.workload_name(a) == "jacobi2d_8192x8192_f32_T1000"


def _profiles():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        d = re.search(r"^kernel_digest:\s*(\S+)", text, re.M)
        w = re.search(r"^workload:\s*(\S+)", text, re.M)
        t = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
        out.append((os.path.basename(path), d and d.group(1), w and w.group(1), t and float(t.group(1))))
    return out


def test_every_profile_names_its_kernel_and_workload():
    profs = _profiles()
    assert profs, "no ncu summaries under profiles/"
    for name, digest, workload, _ in profs:
        assert digest and re.fullmatch(r"[0-9a-f]{16}", digest), name
        assert workload, name


def test_committed_traffic_lookup():
    for name, digest, workload, traffic in _profiles():
        if traffic is None:
            continue
        assert bench.committed_traffic(digest, workload) == traffic, name
        # another kernel build, or another workload, has no committed figure
        assert bench.committed_traffic("0" * 16, workload) is None, name
        assert bench.committed_traffic(digest, workload + "_other") is None, name


def test_kernel_digest_ignores_comments_and_layout_only():
    from paper_1902_10345_gb300 import build

    code = 'int a = 1; // one\n/* two\n lines */ asm("add.rn.f32x2 d, a, b; // kept");\nchar c = \'/\';'
    bare = 'int a = 1;\n asm("add.rn.f32x2 d, a, b; // kept");   char c = \'/\';'
    assert build._code_only(code) == build._code_only(bare)
    assert "// kept" in build._code_only(code)  # inside a string literal
    assert build._code_only(code) != build._code_only(code.replace("a = 1", "a = 2"))
    assert re.fullmatch(r"[0-9a-f]{16}", build.kernel_digest(build.KERNEL_FILES_CHAIN))


def test_median_ci95():
    assert bench.median_ci95([]) == (None, [None, None])
    assert bench.median_ci95([4.0]) == (4.0, [4.0, 4.0])
    xs = [float(v) for v in range(1, 31)]  # 30 values: median 15.5
    med, (lo, hi) = bench.median_ci95(list(reversed(xs)))
    assert med == 15.5
    # order statistics around n/2 -+ 1.96 sqrt(n)/2 (= 9.63 for n = 30)
    half = 1.96 * math.sqrt(30) / 2
    assert lo == xs[max(0, math.floor(15 - half) - 1)] and hi == xs[min(29, math.ceil(15 + half) - 1)]
    assert lo < med < hi


def test_kernel_names():
    class B:
        SDFG_KERNEL_TEMPORAL, SDFG_KERNEL_PERSISTENT, SDFG_KERNEL_RESIDENT, SDFG_KERNEL_SKEWED = 2, 3, 4, 5

    assert [bench.kernel_code(B, n) for n in ("temporal", "persistent", "resident", "skewed")] == [2, 3, 4, 5]
    with pytest.raises(KeyError):
        bench.kernel_code(B, "naive")
