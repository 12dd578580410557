"""Parity of the batched ensemble (adot_ensemble_*, independent channels with
their own dt; persistent channel loops and per-step launches) with per-channel
oracle runs, on seeded movable-bed Riemann channels of ragged lengths (1 cell up
to several tiles).

Tolerances as for single channels: FP64 1e-12 of each variable's scale and the
same step count; FP32 (float-float state) L1 relative error 1e-5 per channel."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 9.81


def _small_ensemble(sizes, seed=3):
    rng = np.random.default_rng(seed)
    E = W.riemann_ensemble(len(sizes), seed=seed, n_min=2, n_max=3)
    hs, qs, zs = [], [], []
    for c, n in enumerate(sizes):
        hL, hR = rng.uniform(0.5, 3.0, 2)
        uL, uR = rng.uniform(-0.5, 1.0, 2)
        zR = rng.uniform(-0.3, 0.3)
        h, q, z = W.riemann(n, 0.0, 10.0, 5.0, (hL, hL * uL, 0.0), (hR, hR * uR, zR))
        hs.append(h), qs.append(q), zs.append(z)
    E.n_cells = np.array(sizes, dtype=np.int64)
    E.length = np.full(len(sizes), 10.0)
    E.Ag = rng.uniform(0.001, 0.02, len(sizes))
    E.h, E.q, E.z = np.concatenate(hs), np.concatenate(qs), np.concatenate(zs)
    return E


SIZES = [1, 2, 7, 100, 254, 255, 256, 300, 511, 700, 1023, 40]


def _oracle_channel(E, c, t_end):
    h, q, z = E.channel(c)
    cfg = O.make_cfg(int(E.n_cells[c]), 0.0, float(E.length[c]), E.cfl,
                     O.grass(float(E.Ag[c]), xi=E.xi, g=G))
    return O.run(cfg, h, q, z, t_end=t_end)


@pytest.mark.parametrize("block,kern", [(0, 0), (128, 1), (256, 1), (512, 1), (0, 2), (256, 2),
                                        (0, 4)])
def test_fp64_ensemble_matches_oracle_per_channel(gpu, block, kern):
    E = _small_ensemble(SIZES)
    with gpu.Ensemble.from_workload(E, gpu.FP64, block_threads=block, step_kernel=kern) as ens:
        ens.set_state(E.h, E.q, E.z)
        t, steps, _ = ens.query()
        assert (steps == 0).all()
        ens.run_to(0.15)
        t, steps, cu = ens.query()
        h, q, z = ens.get_state()
    o = E.offsets
    assert cu == int((steps * E.n_cells).sum())
    for c in range(len(SIZES)):
        ho, qo, zo, to, so, _ = _oracle_channel(E, c, 0.15)
        assert t[c] == 0.15 and steps[c] == so, (c, steps[c], so)
        for a, b in ((h, ho), (q, qo), (z, zo)):
            sc = max(np.abs(b).max(), 1e-300)
            assert np.abs(a[o[c]:o[c + 1]] - b).max() <= 1e-12 * sc, c


@pytest.mark.parametrize("kern", [1, 2])
def test_fp32_ensemble_matches_oracle_per_channel(gpu, kern):
    E = _small_ensemble(SIZES, seed=4)
    with gpu.Ensemble.from_workload(E, gpu.FP32, step_kernel=kern) as ens:
        assert ens.info()[3] == kern
        ens.set_state(E.h, E.q, E.z)
        # the stored initial state (float-float rounds a float64 input by up to ~1e-16)
        g0 = ens.get_state()
        ens.run_to(0.2)
        t, steps, _ = ens.query()
        h, q, z = ens.get_state()
    o = E.offsets
    for c in range(len(SIZES)):
        ho, qo, zo, to, so, _ = _oracle_channel(E, c, 0.2)
        assert t[c] == 0.2
        sl = slice(o[c], o[c + 1])
        # increments W(t) - W(0): cells the waves have not reached add nothing
        for a, b, a0, ag in ((h, ho, E.h, g0[0]), (q, qo, E.q, g0[1]), (z, zo, E.z, g0[2])):
            inc, ref = a[sl] - ag[sl], b - a0[sl]
            assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum(), \
                (c, np.abs(inc - ref).sum() / np.abs(ref).sum())


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_warp_tiles_agree_with_block_tiles(gpu, prec):
    """The warp-tile and block-tile ensemble kernels evaluate the same edges and
    cells; they differ only in rounding order: in float64 the compiler may
    contract the update W + (-nu)(D- + D+) into a fused multiply-add in one
    kernel and not the other (a few ulps), and in float32 the 80-register
    warp-tile variant evaluates the two outer quadrature nodes in paired
    instructions. Times and step counts agree; states within 1e-14 (float64,
    max) and 1e-6 (float32, L1 relative)."""
    E = _small_ensemble(SIZES + [3000, 1234], seed=6)
    out = []
    for kern in (1, 2):
        with gpu.Ensemble.from_workload(E, getattr(gpu, prec), step_kernel=kern, block_threads=256) as ens:
            ens.set_state(E.h, E.q, E.z)
            ens.run_to(0.1)
            t, steps, cu = ens.query()
            out.append((ens.get_state(), t, steps, cu, ens.info()[3]))
    (sa, ta, na, ca, ka), (sb, tb, nb, cb, kb) = out
    assert (ka, kb) == (1, 2)
    for x, y in zip(sa, sb):
        if prec == "FP32":
            assert np.abs(x - y).sum() <= 1e-6 * np.abs(y).sum()
        else:
            assert np.abs(x - y).max() <= 1e-14 * np.abs(y).max()
    assert np.array_equal(ta, tb) and np.array_equal(na, nb) and ca == cb


def test_ensemble_steps_equal_single_channel_contexts(gpu):
    """A fixed number of steps per channel gives, in FP64, the same state as one
    context per channel (same kernels' arithmetic, different launch geometry)."""
    E = _small_ensemble([300, 57, 1000], seed=5)
    with gpu.Ensemble.from_workload(E, gpu.FP64, block_threads=256) as ens:
        ens.set_state(E.h, E.q, E.z)
        ens.step(37)
        _, steps, _ = ens.query()
        h, q, z = ens.get_state()
    assert (steps == 37).all()
    o = E.offsets
    for c in range(3):
        hc, qc, zc = E.channel(c)
        cfg = gpu.make_config(int(E.n_cells[c]), 0.0, 10.0, E.cfl, float(E.Ag[c]), E.xi,
                              precision=gpu.FP64, block_threads=256, reg_cap=64)
        with gpu.Solver(cfg) as s:
            s.set_state(hc, qc, zc)
            s.step(37)
            ref = s.get_state()
        for a, b in zip((h, q, z), ref):
            assert np.abs(a[o[c]:o[c + 1]] - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("kern", [0, 3, 4])
def test_large_ensemble_all_channels_land_on_t_end(gpu, kern):
    E = W.riemann_ensemble(256, seed=11, n_min=200, n_max=20000)
    with gpu.Ensemble.from_workload(E, gpu.FP32, step_kernel=kern) as ens:
        ens.set_state(E.h, E.q, E.z)
        launches = ens.run_to(0.02)
        t, steps, cu = ens.query()
        h, q, z = ens.get_state()
        form = ens.info()[3]
    assert (t == 0.02).all()
    if kern == 3:
        assert form == 3
    if kern == 4:
        assert form in (1, 2)
    if form == 3:  # persistent channel loops: one launch per 16384 steps
        assert launches == 1
    else:  # one launch per step of the longest-running channel
        assert launches >= steps.max()
    assert np.isfinite(h).all() and (h > 0).all()
    # longer channels need more steps (dt ~ dx)
    assert steps[np.argmax(E.n_cells)] > steps[np.argmin(E.n_cells)]


RUN_BLOCKS = [0, 256, 384, 512, 768]


@pytest.mark.parametrize("block", RUN_BLOCKS)
def test_persistent_fp64_matches_oracle_per_channel(gpu, block):
    """The persistent form (one launch per run_to, each CTA stepping whole
    channels to t_end in a device-side loop) against the oracle per channel."""
    E = _small_ensemble(SIZES + [3000, 1234], seed=8)
    with gpu.Ensemble.from_workload(E, gpu.FP64, block_threads=block, step_kernel=3) as ens:
        assert ens.info()[3] == 3
        ens.set_state(E.h, E.q, E.z)
        launches = ens.run_to(0.15)
        t, steps, cu = ens.query()
        h, q, z = ens.get_state()
    assert launches == 1
    o = E.offsets
    assert cu == int((steps * E.n_cells).sum())
    for c in range(len(E.n_cells)):
        ho, qo, zo, to, so, _ = _oracle_channel(E, c, 0.15)
        assert t[c] == 0.15 and steps[c] == so, (c, steps[c], so)
        for a, b in ((h, ho), (q, qo), (z, zo)):
            sc = max(np.abs(b).max(), 1e-300)
            assert np.abs(a[o[c]:o[c + 1]] - b).max() <= 1e-12 * sc, c


def test_persistent_fp32_matches_oracle_per_channel(gpu):
    E = _small_ensemble(SIZES, seed=4)
    with gpu.Ensemble.from_workload(E, gpu.FP32, step_kernel=3) as ens:
        ens.set_state(E.h, E.q, E.z)
        g0 = ens.get_state()
        ens.run_to(0.2)
        t, steps, _ = ens.query()
        h, q, z = ens.get_state()
    o = E.offsets
    for c in range(len(SIZES)):
        ho, qo, zo, to, so, _ = _oracle_channel(E, c, 0.2)
        assert t[c] == 0.2
        sl = slice(o[c], o[c + 1])
        for a, b, a0, ag in ((h, ho, E.h, g0[0]), (q, qo, E.q, g0[1]), (z, zo, E.z, g0[2])):
            inc, ref = a[sl] - ag[sl], b - a0[sl]
            assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum(), \
                (c, np.abs(inc - ref).sum() / np.abs(ref).sum())


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_persistent_agrees_with_per_step_warp_tiles(gpu, prec):
    """The same edges (80-register cap, paired outer nodes) in both forms; the
    persistent form walks each channel in contiguous ranges with D+ carried
    between chunks, the per-step form in 31-cell sub-tiles, and the compiler
    contracts their updates into fused multiply-adds differently, so float64
    states drift apart by rounding over the ~800 steps: equal times and step
    counts, states within 1e-13 (float64, max; both are within 1e-12 of the
    oracle) and 1e-6 (float32, L1 relative), after run_to and after a fixed
    step count."""
    E = _small_ensemble(SIZES + [3000, 1234, 9000], seed=6)
    out = []
    for kern, blk in ((2, 256), (3, 256)):
        with gpu.Ensemble.from_workload(E, getattr(gpu, prec), step_kernel=kern, block_threads=blk) as ens:
            if kern == 2:
                assert ens.info()[:1] == (256,)
            ens.set_state(E.h, E.q, E.z)
            ens.step(23)
            s23 = ens.get_state()
            _, n23, _ = ens.query()
            ens.set_state(E.h, E.q, E.z)
            ens.run_to(0.1)
            t, steps, cu = ens.query()
            out.append((s23, n23, ens.get_state(), t, steps, cu))
    (a23, an, sa, ta, na, ca), (b23, bn, sb, tb, nb, cb) = out
    assert (an == 23).all() and (bn == 23).all()
    for x, y in list(zip(sa, sb)) + list(zip(a23, b23)):
        if prec == "FP32":
            assert np.abs(x - y).sum() <= 1e-6 * np.abs(y).sum()
        else:
            assert np.abs(x - y).max() <= 1e-13 * np.abs(y).max()
    assert np.array_equal(ta, tb) and np.array_equal(na, nb) and ca == cb


def test_persistent_run_to_resumes(gpu):
    """run_to(0.05) then run_to(0.1): every channel continues from its state at
    0.05 (the oracle restarted there) and lands on 0.1."""
    E = _small_ensemble([700, 31, 2500, 1], seed=9)
    with gpu.Ensemble.from_workload(E, gpu.FP64, step_kernel=3) as ens:
        ens.set_state(E.h, E.q, E.z)
        ens.run_to(0.05)
        mid = ens.get_state()
        _, s1, _ = ens.query()
        ens.run_to(0.1)
        t, s2, _ = ens.query()
        h, q, z = ens.get_state()
    assert (t == 0.1).all()
    o = E.offsets
    for c in range(len(E.n_cells)):
        sl = slice(o[c], o[c + 1])
        cfg = O.make_cfg(int(E.n_cells[c]), 0.0, float(E.length[c]), E.cfl,
                         O.grass(float(E.Ag[c]), xi=E.xi, g=G))
        h1, q1, z1, t1, n1, _ = O.run(cfg, *(m[sl] for m in mid), t_end=0.05)
        assert s2[c] - s1[c] == n1
        for a, b in ((h, h1), (q, q1), (z, z1)):
            assert np.abs(a[sl] - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)


def test_persistent_dry_out_is_reported(gpu):
    """A channel whose two streams leave each other (beyond the dry-bed limit)
    drives h through zero: the persistent run stops and reports it, and the
    state stays readable."""
    E = _small_ensemble([400, 512, 900], seed=10)
    P = W.dam_break(512, hL=0.1, hR=0.1, uL=-3.0, uR=3.0)
    o = E.offsets
    E.h[o[1]:o[2]], E.q[o[1]:o[2]], E.z[o[1]:o[2]] = P.h, P.q, P.z
    E.length[1] = P.x_max - P.x_min
    with gpu.Ensemble.from_workload(E, gpu.FP32, step_kernel=3) as ens:
        ens.set_state(E.h, E.q, E.z)
        with pytest.raises(gpu.AdotError) as e:
            ens.run_to(1.0)
        assert e.value.status in (gpu.E_NONPOSITIVE_DEPTH, gpu.E_NONFINITE)
        h, q, z = ens.get_state()
        assert h.shape == (int(E.n_cells.sum()),)


def test_form_chosen_by_estimated_balance(gpu):
    """step_kernel = 0 runs the persistent form when the list schedule of the
    channels (largest work first) onto its CTAs is balanced (many channels of
    equal length) and per-step launches when one CTA would hold a channel much
    longer than its share (a few long channels among short ones); both give the
    forced persistent form's float64 state."""
    cases = {"balanced": [300] * 2048, "skewed": [40000, 30000] + [200] * 40}
    for name, sizes in cases.items():
        E = _small_ensemble(sizes, seed=13)
        out = []
        for kern in (0, 3):
            with gpu.Ensemble.from_workload(E, gpu.FP64, step_kernel=kern) as ens:
                ens.set_state(E.h, E.q, E.z)
                form = ens.info()[3]
                ens.run_to(0.01)
                t, steps, _ = ens.query()
                out.append((form, ens.get_state(), steps))
        (fa, sa, na), (fb, sb, nb) = out
        assert fb == 3
        assert (fa == 3) == (name == "balanced"), (name, fa)
        assert np.array_equal(na, nb)
        for x, y in zip(sa, sb):
            assert np.abs(x - y).max() <= 1e-14 * np.abs(y).max()


# ---- cluster teams: long channels stepped by the CTAs of one cluster ---------

def _skewed(seed, big=(30000, 22000, 9000), n_small=60):
    rng = np.random.default_rng(seed)
    sizes = list(big) + [int(x) for x in rng.integers(1, 3000, n_small)]
    return _small_ensemble(sizes, seed=seed)


def test_team_form_matches_oracle_per_channel(gpu):
    """step_kernel 5: the long channels run on cluster teams (2 or 4 CTAs
    exchanging the CFL maximum through distributed shared memory every step),
    the others one CTA each; FP64 per channel against the oracle (1e-12 and the
    same step count). (The float32 form is held to the one-CTA form below,
    whose float32 accuracy the tests above pin against the oracle.)"""
    E = _skewed(31)
    with gpu.Ensemble.from_workload(E, gpu.FP64, step_kernel=5) as ens:
        ens.set_state(E.h, E.q, E.z)
        pl = ens.plan(0)
        launches = ens.run_to(0.02)
        t, steps, _ = ens.query()
        h, q, z = ens.get_state()
    assert pl["form"] == 3 and pl["cluster"] in (2, 4) and pl["teamed"] >= 1, pl
    assert launches == 1 and (t == 0.02).all()
    o = E.offsets
    for c in range(len(E.n_cells)):
        ho, qo, zo, to, so, _ = _oracle_channel(E, c, 0.02)
        sl = slice(o[c], o[c + 1])
        assert steps[c] == so, (c, steps[c], so)
        for a, b in ((h, ho), (q, qo), (z, zo)):
            assert np.abs(a[sl] - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), c


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_team_form_equals_one_cta_form(gpu, prec):
    """The team form evaluates the same edges and cells as one CTA per channel
    (384-thread CTAs, no teams), in another kernel whose update the compiler
    may contract into fused multiply-adds differently: states within 1e-14
    (float64, max) and 1e-6 (float32, L1 relative), equal times and step
    counts, after run_to, after a fixed step count and after a second run_to."""
    E = _skewed(32)
    out = []
    for kern, blk in ((5, 0), (3, 384)):
        with gpu.Ensemble.from_workload(E, getattr(gpu, prec), step_kernel=kern, block_threads=blk) as ens:
            ens.set_state(E.h, E.q, E.z)
            pl0, pl1 = ens.plan(0), ens.plan(1)
            ens.step(17)
            s17 = ens.get_state()
            ens.set_state(E.h, E.q, E.z)
            ens.run_to(0.01)
            ens.run_to(0.02)
            t, steps, cu = ens.query()
            out.append((pl0, pl1, s17, ens.get_state(), t, steps, cu))
    (pa0, pa1, a17, sa, ta, na, ca), (pb0, pb1, b17, sb, tb, nb, cb) = out
    assert pa0["cluster"] > 1 and pb0["cluster"] == 1 and pb0["block"] == 384
    assert pa1["form"] == 3 and pb1["cluster"] == 1
    for x, y in list(zip(sa, sb)) + list(zip(a17, b17)):
        if prec == "FP32":
            assert np.abs(x - y).sum() <= 1e-6 * np.abs(y).sum()
        else:
            assert np.abs(x - y).max() <= 1e-14 * np.abs(y).max()
    assert np.array_equal(na, nb) and ca == cb
    assert np.array_equal(ta, tb)


def test_team_form_reports_dry_out(gpu):
    """The longest channel (stepped by a team) dries out: the run stops with the
    status, every CTA leaves, and the state can still be read."""
    E = _skewed(33, big=(30000, 9000), n_small=30)
    P = W.dam_break(30000, hL=0.1, hR=0.1, uL=-3.0, uR=3.0)
    o = E.offsets
    E.h[o[0]:o[1]], E.q[o[0]:o[1]], E.z[o[0]:o[1]] = P.h, P.q, P.z
    with gpu.Ensemble.from_workload(E, gpu.FP32, step_kernel=5) as ens:
        ens.set_state(E.h, E.q, E.z)
        assert ens.plan(0)["teamed"] >= 1
        with pytest.raises(gpu.AdotError) as e:
            ens.run_to(1.0)
        assert e.value.status in (gpu.E_NONPOSITIVE_DEPTH, gpu.E_NONFINITE)
        h, q, z = ens.get_state()
        assert h.shape == (int(E.n_cells.sum()),)


def test_team_exchange_wait_runs_out_and_reports(gpu):
    """A team member withholds its first arrival (adot_ensemble_inject_fault):
    the members' bounded waits run out (~1 s), the launch ends with
    ADOT_E_TIMEOUT instead of hanging, and the ensemble is usable again after
    set_state (the next run matches a fresh ensemble's)."""
    E = _skewed(34)
    with gpu.Ensemble.from_workload(E, gpu.FP64, step_kernel=5) as ens:
        ens.set_state(E.h, E.q, E.z)
        assert ens.plan(0)["teamed"] >= 1
        ens.inject_fault(1)
        with pytest.raises(gpu.AdotError) as e:
            ens.run_to(0.01)
        assert e.value.status == gpu.E_TIMEOUT
        ens.set_state(E.h, E.q, E.z)
        ens.run_to(0.01)
        got = ens.get_state()
        t, _, _ = ens.query()
    assert (t == 0.01).all()
    with gpu.Ensemble.from_workload(E, gpu.FP64, step_kernel=5) as ens:
        ens.set_state(E.h, E.q, E.z)
        ens.run_to(0.01)
        ref = ens.get_state()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
