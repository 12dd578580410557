"""Checkpoint and resume through the C ABI: a run that is saved, restored into
a fresh context and continued takes steps bit-identical to the run that was
never interrupted (state words, time, step count and dt), in both precisions,
with host and device blobs, through single launches and graph replays, and
with a time-dependent boundary. Blobs from another config are refused."""
import dataclasses

import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problems():
    bump = W.gaussian_bump(1537)
    # inflow of q and a bed that degrades linearly in time at the left end
    bump_qz = dataclasses.replace(bump, name="gaussian_bump_qz", bc_left=W.BC_INFLOW_QZ,
                                  bcl=(0.6, 0.0, 0.002))
    return [W.smooth_periodic(4099), bump_qz, W.movable_bed_riemann(701)]


def _blob_state(gpu, s):
    return bytes(gpu.adot_checkpoint_save(s.ctx))


@pytest.mark.parametrize("P", _problems(), ids=lambda P: P.name)
@pytest.mark.parametrize("prec", ["FP32", "FP64"])
@pytest.mark.parametrize("k1,k2", [(37, 61), (48, 96), (5, 1)])
def test_resume_is_bit_exact(gpu, P, prec, k1, k2):
    cfg = gpu.config_for(P, getattr(gpu, prec))
    with gpu.Solver(cfg) as a:
        a.set_state(P.h, P.q, P.z)
        a.step(k1)
        blob = a.checkpoint()
        assert blob.size == gpu.adot_checkpoint_size(a.ctx) == 128 + 24 * P.n
        a.step(k2)
        ref_q = a.query()
        ref_state = a.get_state()
        ref_blob = _blob_state(gpu, a)
    with gpu.Solver(cfg) as b:
        b.restore(blob)
        t, steps, _ = b.query()
        assert steps == k1
        b.step(k2)
        got_q = b.query()
        got_state = b.get_state()
        got_blob = _blob_state(gpu, b)
    assert got_q == ref_q  # time, step count and last dt, bit for bit
    for x, y in zip(got_state, ref_state):
        assert np.array_equal(x, y)
    assert got_blob == ref_blob  # the stored words themselves (float-float pairs included)


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_resume_is_bit_exact_with_friction_and_feed(gpu, prec):
    """The Soni case (the step kernels with the friction source, the sediment
    feed and the slope-continuing ghosts compiled in)."""
    P = W.soni_aggradation()
    cfg = gpu.config_for(P, getattr(gpu, prec), law=gpu.LAW_POWER, beta=5.0, ks=49.4)
    with gpu.Solver(cfg) as a:
        a.set_state(P.h, P.q, P.z)
        a.step(53)
        blob = a.checkpoint()
        a.step(101)
        ref = a.get_state(), a.query()
    with gpu.Solver(cfg) as b:
        b.restore(blob)
        b.step(101)
        got = b.get_state(), b.query()
    assert got[1] == ref[1]
    for x, y in zip(got[0], ref[0]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_device_blob_and_rewind_in_place(gpu, prec):
    torch = pytest.importorskip("torch")
    P = W.smooth_periodic(2049)
    with gpu.Solver(gpu.config_for(P, getattr(gpu, prec))) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(13)
        nbytes = gpu.adot_checkpoint_size(s.ctx)
        dblob = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        s.checkpoint(dblob)
        host_blob = s.checkpoint()
        assert np.array_equal(dblob.cpu().numpy(), host_blob)
        s.step(29)
        first = s.get_state(), s.query()
        s.restore(dblob)  # rewind the same context
        s.step(29)
        second = s.get_state(), s.query()
    for x, y in zip(first[0], second[0]):
        assert np.array_equal(x, y)
    assert first[1] == second[1]


def test_run_to_after_resume_matches(gpu):
    P = W.movable_bed_riemann(701)
    cfg = gpu.config_for(P, gpu.FP32)
    with gpu.Solver(cfg) as a:
        a.set_state(P.h, P.q, P.z)
        a.run_to(0.3 * P.t_end)
        blob = a.checkpoint()
        a.run_to(P.t_end)
        ref = a.get_state(), a.query()
    with gpu.Solver(cfg) as b:
        b.restore(blob)
        b.run_to(P.t_end)
        got = b.get_state(), b.query()
    for x, y in zip(got[0], ref[0]):
        assert np.array_equal(x, y)
    assert got[1] == ref[1]


def test_mismatched_or_damaged_blob_is_refused(gpu):
    P = W.smooth_periodic(1000)
    cfg = gpu.config_for(P, gpu.FP32)
    with gpu.Solver(cfg) as a:
        a.set_state(P.h, P.q, P.z)
        a.step(7)
        blob = a.checkpoint()
        before = a.get_state()
        other = gpu.config_for(P, gpu.FP32)
        other.cfl = 0.7
        with gpu.Solver(other) as b:
            b.set_state(P.h, P.q, P.z)
            with pytest.raises(gpu.AdotError):
                b.restore(blob)
        with gpu.Solver(gpu.config_for(P, gpu.FP64)) as b:
            with pytest.raises(gpu.AdotError):
                b.restore(blob)
        bad = blob.copy()
        bad[0] ^= 0xFF
        with pytest.raises(gpu.AdotError):
            a.restore(bad)
        with pytest.raises(gpu.AdotError):
            a.restore(blob[:-8].copy())
        after = a.get_state()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("field", ["ks", "u_cr"])
def test_blob_of_another_friction_or_threshold_is_refused(gpu, field):
    """The fingerprint covers the friction coefficient and the law's threshold
    and exponent: configs that differ only there do not share checkpoints."""
    P = W.movable_bed_riemann(400)
    kw = {"law": gpu.LAW_POWER, "beta": 3.0, "u_cr": 0.1, "ks": 30.0}
    with gpu.Solver(gpu.config_for(P, gpu.FP64, **kw)) as a:
        a.set_state(P.h, P.q, P.z)
        a.step(5)
        blob = a.checkpoint()
        kw2 = dict(kw)
        kw2[field] = kw[field] * 1.5
        with gpu.Solver(gpu.config_for(P, gpu.FP64, **kw2)) as b:
            b.set_state(P.h, P.q, P.z)
            with pytest.raises(gpu.AdotError):
                b.restore(blob)
        with gpu.Solver(gpu.config_for(P, gpu.FP64, **kw)) as c:
            c.set_state(P.h, P.q, P.z)
            c.restore(blob)
            assert c.query()[1] == 5


def test_save_before_state_is_refused(gpu):
    P = W.smooth_periodic(64)
    with gpu.Solver(gpu.config_for(P, gpu.FP32)) as a:
        with pytest.raises(gpu.AdotError):
            a.checkpoint()
