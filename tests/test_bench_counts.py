"""Host-side checks of the benchmark's roofline bookkeeping (no GPU): the ncu
counter constants of the warp-tile step cover every shape the autotuner can
pick for the benchmark, lie in the ranges the kernel's work allows, and the
issue roofline is the plain quotient it claims to be."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("cap", [64, 80])
def test_warp_shapes_carry_every_counter(bench, cap):
    c = bench.counts("warp", 256, cap)
    for key in ("flops", "instr", "xu", "dram"):
        assert c.get(key), (cap, key)
    # three float32 nodes per cell-update: a few hundred executed flops, at most the
    # planning estimate; 400-700 thread instructions; a few tens of XU operations;
    # DRAM between the 24 B one-way state and the 48 B algorithmic traffic
    assert 300.0 < c["flops"] < bench.FLOPS_PER_CELL_UPDATE_PLAN
    assert 400.0 < c["instr"] < 700.0
    assert 10.0 < c["xu"] < 60.0
    assert 24.0 <= c["dram"] <= 1.1 * bench.BYTES_PER_CELL_UPDATE


def test_block_kernel_uses_its_own_flop_count(bench):
    assert bench.counts("block", 256, 64) == {"flops": bench.FLOPS_BLOCK}


def test_issue_roofline_is_the_plain_quotient(bench):
    n, t = 10_000_000, 0.1658e-3
    r = bench.issue_roofline(540.0, n, t)
    peak = 152 * 4 * 32 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(540.0 * n / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert bench.issue_roofline(None, n, t) is None
