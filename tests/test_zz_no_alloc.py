"""adot_step_noalloc: time stepping for callers that cannot allocate device
memory (a custom operation inside a framework that owns the device allocator,
a real-time loop that reserves all memory up front). It advances a
caller-owned float64 state in place, using a library-internal device array
instead of allocations. Checked through the C ABI against the ordinary
context path (adot_create / set_state / step / get_state) on two calls in a
row, to the float64 tolerance of the other step tests (1e-12 of each
variable's scale).

This file is collected last so that a failure here does not stop a run with -x
before the other tests."""
import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _context_run(gpu, P, steps):
    with gpu.Solver(gpu.config_for(P, gpu.FP64, block_threads=256, reg_cap=64)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(steps)
        t, _, _ = s.query()
        return s.get_state(), t


@pytest.mark.parametrize("make", [lambda: W.smooth_periodic(3001),
                                  lambda: W.movable_bed_riemann(200)])
def test_noalloc_matches_context_path_on_two_calls(gpu, make):
    torch = pytest.importorskip("torch")
    P = make()
    cfg = gpu.config_for(P, gpu.FP64)
    h, q, z = (torch.tensor(a, device="cuda") for a in (P.h, P.q, P.z))
    stream = torch.cuda.current_stream()
    t = 0.0
    for k_total, k_call in ((7, 7), (15, 8)):
        t = gpu.adot_step_noalloc(cfg, h, q, z, k_call, t, stream)
        ref, t_ref = _context_run(gpu, P, k_total)
        assert t == pytest.approx(t_ref, rel=1e-13)
        for a, b in zip((h, q, z), ref):
            a = a.cpu().numpy()
            assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("kind", ["second_order", "soni"])
def test_noalloc_second_order_and_friction(gpu, kind):
    """The second-order variant (warp tiles) and the Soni case (friction,
    sediment feed, power law: the extended step kernels) through the same
    entry point."""
    torch = pytest.importorskip("torch")
    if kind == "second_order":
        P, kw = W.movable_bed_riemann(300), {"order": 2}
    else:
        P, kw = W.soni_aggradation(), {"law": gpu.LAW_POWER, "beta": 5.0, "ks": 49.4}
    h, q, z = (torch.tensor(a, device="cuda") for a in (P.h, P.q, P.z))
    t = gpu.adot_step_noalloc(gpu.config_for(P, gpu.FP64, **kw), h, q, z, 20, 0.0,
                              torch.cuda.current_stream())
    with gpu.Solver(gpu.config_for(P, gpu.FP64, block_threads=256, reg_cap=64, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(20)
        t_ref, _, _ = s.query()
        ref = s.get_state()
    assert t == pytest.approx(t_ref, rel=1e-13)
    for a, b in zip((h, q, z), ref):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-12 * np.abs(b).max()


def test_noalloc_rejects_what_it_cannot_do(gpu):
    torch = pytest.importorskip("torch")
    P = W.smooth_periodic(64)
    h, q, z = (torch.tensor(a, device="cuda") for a in (P.h, P.q, P.z))
    with pytest.raises(gpu.AdotError) as e:
        gpu.adot_step_noalloc(gpu.config_for(P, gpu.FP32), h, q, z, 1)
    assert e.value.status == gpu.E_UNSUPPORTED
    big = W.smooth_periodic(65537)
    hb, qb, zb = (torch.tensor(a, device="cuda") for a in (big.h, big.q, big.z))
    with pytest.raises(gpu.AdotError) as e:
        gpu.adot_step_noalloc(gpu.config_for(big, gpu.FP64), hb, qb, zb, 1)
    assert e.value.status == gpu.E_INVALID_ARG


@pytest.mark.parametrize("order", [1, 2])
def test_noalloc_call_after_setup_allocates_nothing(gpu, order):
    """The property the entry point exists for. The first call on a device with
    a configuration may allocate (the driver loads the scratch array and the
    kernels it runs on first use); every later call with that configuration
    must leave the device's free memory exactly where it was."""
    torch = pytest.importorskip("torch")
    P = W.movable_bed_riemann(257)
    cfg = gpu.config_for(P, gpu.FP64, order=order)
    h, q, z = (torch.tensor(a, device="cuda") for a in (P.h, P.q, P.z))
    stream = torch.cuda.current_stream()
    t = gpu.adot_step_noalloc(cfg, h, q, z, 1, 0.0, stream)  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in (5, 6):
        t = gpu.adot_step_noalloc(cfg, h, q, z, k, t, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.isfinite(h.cpu().numpy()).all() and t > 0.0
