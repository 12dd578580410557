"""The pipe-throughput probes behind the ALU rooflines (adot_measure_pipe):
every kind returns a rate in the range a GB300 can reach, and the paired
forms are counted per element (FFMA2 at 4 flops, the bf16x2 tanh at 2 ops)."""
import pytest

pytestmark = pytest.mark.gpu

# (kind name, lower, upper) in units of 1e12 per second; nominal GB300 figures:
# FP32 ~80 TFLOP/s, multi-function unit ~5e12 op/s, FP64 ~1.2 TFLOP/s
BOUNDS = [("PIPE_FFMA", 20, 200), ("PIPE_FFMA2", 20, 400), ("PIPE_RSQ", 1, 40),
          ("PIPE_SIN", 1, 40), ("PIPE_TANH", 1, 40), ("PIPE_TANH_BF16X2", 1, 80),
          ("PIPE_DFMA", 0.3, 10)]


@pytest.mark.parametrize("name,lo,hi", BOUNDS, ids=[b[0] for b in BOUNDS])
def test_pipe_probe_rates(gpu, name, lo, hi):
    rate, sec = gpu.adot_measure_pipe(getattr(gpu, name), 0)
    assert 0.001 < sec < 5.0
    assert lo * 1e12 <= rate <= hi * 1e12, (name, rate)
