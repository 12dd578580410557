"""Parity of whole CUDA time-stepping runs (fused edge + update + CFL kernel,
Eq. scheme) with the FP64 oracle, on the benchmark workloads at sizes the
oracle finishes in seconds (several blocks plus a ragged tail), plus the
runtime's contracts: graph replays equal single launches bit for bit, run_to
lands on t_end, sums are reproducible, errors are reported.

Tolerances. FP64: every value within 1e-12 relative to the variable's scale
after the run (rounding-order differences only). FP32 (float-float state,
float32 fluctuations): the increment W^K - W^0 matches the oracle's to an L1
relative error of 1e-5, the target precision of the float32 path."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 9.81


def _ocfg(P):
    law = O.grass(P.Ag, xi=P.xi, g=P.g)
    return O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, law, P.bc_left, P.bc_right, P.bcl, P.bcr)


def _scale(a):
    return max(np.abs(a).max(), 1e-300)


def _run_gpu(gpu, P, prec, steps=None, t_end=None, **kw):
    with gpu.Solver(gpu.config_for(P, prec, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        if t_end is not None:
            s.run_to(t_end)
        else:
            s.step(steps)
        t, nsteps, dt = s.query()
        h, q, z = s.get_state()
    return h, q, z, t, nsteps, dt


VARIANTS = [(128, 64, 1), (128, -1, 1), (256, 64, 1), (256, -1, 1), (512, 64, 1), (512, -1, 1),
            (256, 64, 2), (128, 64, 2), (128, 72, 2), (256, 80, 2)]


@pytest.mark.parametrize("n", [1, 2, 31, 32, 255, 256, 511, 1000, 2049])
@pytest.mark.parametrize("block,cap,kern", VARIANTS)
def test_fp64_smooth_periodic_matches_oracle(gpu, n, block, cap, kern):
    P = W.smooth_periodic(n)
    K = 60
    ho, qo, zo, to, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, max_steps=K)
    h, q, z, t, steps, _ = _run_gpu(gpu, P, gpu.FP64, steps=K, block_threads=block, reg_cap=cap,
                                    step_kernel=kern)
    assert steps == K
    assert t == pytest.approx(to, rel=1e-13)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * _scale(b)


@pytest.mark.parametrize("n", [200, 701])
def test_fp64_movable_bed_riemann_to_t_end(gpu, n):
    """Movable-bed Riemann problem (transmissive ends) run to t_end = 1 s."""
    P = W.movable_bed_riemann(n)
    ho, qo, zo, to, so, _ = O.run(_ocfg(P), P.h, P.q, P.z, t_end=P.t_end)
    h, q, z, t, steps, _ = _run_gpu(gpu, P, gpu.FP64, t_end=P.t_end)
    assert t == P.t_end and steps == so
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * _scale(b)


def test_fp64_inflow_outflow_boundaries(gpu):
    """Test 2 boundary data (inflow q and time-dependent z, outflow h)."""
    from oracle import exact as X
    q0 = 2.0
    qb, zb, rate, hR = X.berthon_boundary(q0)
    n = 300
    h0, qq0, z0 = X.berthon_cell_average(n, q0, 0.0)
    P = W.Problem("berthon", n, 0.0, 7.0, 0.9, 10.0, 0.005, 1.0, h0, qq0, z0,
                  W.BC_INFLOW_QZ, W.BC_OUTFLOW_H, (qb, zb, rate), (hR, 0.0, 0.0))
    ho, qo, zo, to, so, _ = O.run(_ocfg(P), P.h, P.q, P.z, t_end=2.0)
    h, q, z, t, steps, _ = _run_gpu(gpu, P, gpu.FP64, t_end=2.0)
    assert t == 2.0 and steps == so
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * _scale(b)


def test_fp64_gaussian_bump_inflow_outflow(gpu):
    P = W.gaussian_bump(997)
    ho, qo, zo, _, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, max_steps=150)
    h, q, z, _, _, _ = _run_gpu(gpu, P, gpu.FP64, steps=150)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * _scale(b)


@pytest.mark.parametrize("n", [257, 4099])
def test_fp32_increment_matches_oracle(gpu, n):
    P = W.smooth_periodic(n)
    K = 200
    ho, qo, zo, _, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, max_steps=K)
    h, q, z, _, _, _ = _run_gpu(gpu, P, gpu.FP32, steps=K)
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        inc, ref = a - a0, b - a0
        assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum()


def test_fp32_movable_bed_riemann_l1(gpu):
    P = W.movable_bed_riemann(200)
    ho, qo, zo, to, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, t_end=P.t_end)
    h, q, z, t, _, _ = _run_gpu(gpu, P, gpu.FP32, t_end=P.t_end)
    assert t == P.t_end
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).sum() <= 1e-5 * np.abs(b).sum()


def test_fp32_variants_agree(gpu):
    """Every compiled variant evaluates each edge and cell with the same code:
    float32 increments agree to 1e-7 of their L1 norm."""
    P = W.smooth_periodic(5003)
    ref = None
    for block, cap, kern in VARIANTS:
        h, q, z, *_ = _run_gpu(gpu, P, gpu.FP32, steps=50, block_threads=block, reg_cap=cap,
                               step_kernel=kern)
        inc = np.concatenate([h - P.h, q - P.q, z - P.z])
        if ref is None:
            ref = inc
        assert np.abs(inc - ref).sum() <= 1e-7 * np.abs(ref).sum()


def test_autotune_keeps_state_and_picks_a_variant(gpu):
    P = W.smooth_periodic(20000)
    with gpu.Solver(gpu.config_for(P, gpu.FP32, block_threads=256, reg_cap=64)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(12)
        ref = s.get_state()
    with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:  # every field free: tuned in set_state
        s.set_state(P.h, P.q, P.z)
        b, r, k = gpu.adot_autotune(s.ctx, 4)
        assert (b, r, k) in VARIANTS
        t, steps, _ = s.query()
        assert t == 0.0 and steps == 0
        s.step(12)
        got = s.get_state()
    for a, b_ in zip(got, ref):
        assert np.abs((a - b_)).sum() <= 1e-7 * max(np.abs(b_).sum(), 1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_single_launches(gpu, prec):
    """steps_per_graph = 6 (graph replays) and a run that is never graph-aligned
    (one step first) give bit-identical states after the same number of steps."""
    P = W.smooth_periodic(3001)
    a = _run_gpu(gpu, P, prec, steps=61, steps_per_graph=6)
    with gpu.Solver(gpu.config_for(P, prec, steps_per_graph=60)) as s:
        s.set_state(P.h, P.q, P.z)
        for _ in range(61):
            s.step(1)
        b = s.get_state() + s.query()
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3] == b[3] and a[4] == b[4] == 61


@pytest.mark.parametrize("prec", [0, 1])
def test_run_to_lands_on_t_end_and_stops(gpu, prec):
    P = W.movable_bed_riemann(200)
    with gpu.Solver(gpu.config_for(P, prec)) as s:
        s.set_state(P.h, P.q, P.z)
        k1 = s.run_to(0.25)
        t, steps, _ = s.query()
        assert t == 0.25 and steps == k1 > 0
        assert s.run_to(0.25) == 0  # already there
        k2 = s.run_to(0.5)
        t, steps, _ = s.query()
        assert t == 0.5 and steps == k1 + k2
    if prec == 0:
        ho, qo, zo, to, so, _ = O.run(_ocfg(P), P.h, P.q, P.z, t_end=0.25)
        assert so == k1


@pytest.mark.parametrize("prec", [0, 1])
def test_conserved_sums(gpu, prec):
    """Fixed-order device sums equal numpy's sums of the state, are bit-reproducible,
    and the periodic run conserves sum h."""
    P = W.smooth_periodic(100003)
    with gpu.Solver(gpu.config_for(P, prec)) as s:
        s.set_state(P.h, P.q, P.z)
        s0 = s.conserved_sums()
        assert np.allclose(s0, [P.h.sum(), P.q.sum(), P.z.sum()], rtol=1e-13, atol=1e-9)
        s.step(30)
        s1 = s.conserved_sums()
        s2 = s.conserved_sums()
        assert np.array_equal(s1, s2)
        h, q, z = s.get_state()
        assert np.allclose(s1, [h.sum(), q.sum(), z.sum()], rtol=1e-12, atol=1e-9)
        tol = 1e-13 if prec == 0 else 1e-9
        assert abs(s1[0] - s0[0]) <= tol * s0[0]


def test_lake_at_rest_gpu(gpu):
    P = W.lake_at_rest(4096)
    for prec, qb in ((0, 1e-12), (1, 2e-5)):
        h, q, z, _, _, _ = _run_gpu(gpu, P, prec, steps=300)
        assert np.abs(q).max() <= qb
        assert np.abs(h + z - 1.0).max() <= 50 * qb


def test_bad_state_is_reported(gpu):
    P = W.smooth_periodic(512)
    with gpu.Solver(gpu.config_for(P, 0)) as s:
        h = P.h.copy()
        h[17] = -1.0
        with pytest.raises(gpu.AdotError) as e:
            s.set_state(h, P.q, P.z)
        assert e.value.status == gpu.E_NONPOSITIVE_DEPTH
        q = P.q.copy()
        q[3] = np.nan
        with pytest.raises(gpu.AdotError) as e:
            s.set_state(P.h, q, P.z)
        assert e.value.status == gpu.E_NONFINITE
        # the context stays usable
        s.set_state(P.h, P.q, P.z)
        s.step(5)


def test_dry_out_is_reported(gpu):
    """Two streams leaving each other (u = -+3 m/s on h = 0.1 m, beyond the
    2(c_L + c_R) dry-bed limit) drive h through zero, as in the oracle: the run
    reports ADOT_E_NONPOSITIVE_DEPTH or ADOT_E_NONFINITE and the state can
    still be read."""
    P = W.dam_break(512, hL=0.1, hR=0.1, uL=-3.0, uR=3.0)
    with pytest.raises(O.OracleError):
        O.run(_ocfg(P), P.h, P.q, P.z, max_steps=50)
    with gpu.Solver(gpu.config_for(P, 0)) as s:
        s.set_state(P.h, P.q, P.z)
        with pytest.raises(gpu.AdotError) as e:
            s.step(400)
        assert e.value.status in (gpu.E_NONPOSITIVE_DEPTH, gpu.E_NONFINITE)
        h, q, z = s.get_state()
        assert h.shape == (512,)


def test_device_state_roundtrip(gpu):
    torch = pytest.importorskip("torch")
    P = W.smooth_periodic(2000)
    ho, qo, zo, _, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, max_steps=10)
    stream = torch.cuda.current_stream()
    with gpu.Solver(gpu.config_for(P, 0), stream=stream) as s:
        th, tq, tz = (torch.tensor(a, device="cuda") for a in (P.h, P.q, P.z))
        s.set_state(th, tq, tz)
        s.step(10)
        oh, oq, oz = (torch.empty(2000, dtype=torch.float64, device="cuda") for _ in range(3))
        gpu.adot_get_state(s.ctx, oh, oq, oz)
        torch.cuda.synchronize()
        for a, b in ((oh, ho), (oq, qo), (oz, zo)):
            assert np.abs(a.cpu().numpy() - b).max() <= 1e-12 * _scale(b)


@pytest.mark.parametrize("law", ["grass", "mpm"])
def test_fp32_time_step_matches_oracle(gpu, law):
    """The float32 CFL maximum (Newton on the flow-side extreme root) gives the
    oracle's dt (trigonometric roots, R2) to float32 rounding, on states with
    both signs of u, sub- and supercritical."""
    n = 4001
    rng = np.random.default_rng(77)
    for trial in range(4):
        h = rng.uniform(0.1, 3.0, n)
        fr = rng.uniform(-2.5, 2.5, n)
        q = fr * np.sqrt(G * h) * h
        z = rng.uniform(0.0, 0.2, n)
        if law == "grass":
            Ag = rng.uniform(0.001, 0.05)
            olaw = O.grass(Ag, xi=W.XI_P04, g=G)
            cfg = gpu.make_config(n, 0.0, 10.0, 0.9, Ag, W.XI_P04, precision=gpu.FP32)
        else:
            olaw = O.mpm(2.65, 1e-3, 0.02, xi=W.XI_P04, g=G)
            cfg = gpu.make_config(n, 0.0, 10.0, 0.9, 0.0, W.XI_P04, precision=gpu.FP32,
                                  law=gpu.LAW_MPM, s_rel=2.65, d50=1e-3, manning_n=0.02)
        ocfg = O.make_cfg(n, 0.0, 10.0, 0.9, olaw)
        _, _, _, _, _, dt_ref = O.run(ocfg, h, q, z, max_steps=1)
        with gpu.Solver(cfg) as s:
            s.set_state(h, q, z)
            _, dt = s.step(1)
        assert dt == pytest.approx(dt_ref, rel=2e-6)


@pytest.mark.parametrize("block,cap", [(256, 64), (256, 80)])
@pytest.mark.parametrize("shape", ["one_chunk_each", "one_more", "one_less", "two_chunk_static",
                                   "long_static"])
def test_fp64_warp_ranges_at_partition_edges(gpu, block, cap, shape):
    """The warp kernel processes ranges of 32 k - 1 cells (chunks of 32 edges,
    D+ carried from lane 31 into the next chunk's lane 0): with W resident warps
    and K = n / 32 chunks, every warp first takes a static contiguous range of
    k_s = floor((4/8) K / W) chunks when k_s >= 2, then 63-cell groups from the
    work pool. 31 W cells (and one more or less) go to the pool alone, about
    half the warps getting a group; 6 x 31 W + 17 gives static ranges of 2
    chunks, then pool groups with a ragged last one; 12 x 31 W + 5 gives static
    ranges of 5 chunks. FP64 against the oracle, every value within 1e-12."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = sms * (65536 // (block * cap)) * block // 32
    n = {"one_chunk_each": 31 * w, "one_more": 31 * w + 1, "one_less": 31 * w - 1,
         "two_chunk_static": 6 * 31 * w + 17, "long_static": 12 * 31 * w + 5}[shape]
    P = W.smooth_periodic(n)
    K = 12
    ho, qo, zo, to, _, _ = O.run(_ocfg(P), P.h, P.q, P.z, max_steps=K)
    h, q, z, t, steps, _ = _run_gpu(gpu, P, gpu.FP64, steps=K, block_threads=block, reg_cap=cap,
                                    step_kernel=2)
    assert steps == K
    assert t == pytest.approx(to, rel=1e-13)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * _scale(b)


@pytest.mark.parametrize("bc,ks", [("periodic", 0.0), ("transmissive", 0.0), ("transmissive", 30.0)])
def test_fp32_deferred_redo_on_every_cell(gpu, bc, ks):
    """Near-critical flow on a fixed bed (A_g = 0, Fr = 1 + 0.002 sin): the
    roots u - c and 0 nearly coalesce at almost every node, so the float32
    warp-tile step lists almost every cell for k_fixup, which recomputes them
    with float64 edges (the periodic wrap, the transmissive end cells and, with
    K_s = 30, the friction source included). 20 steps against the oracle: the
    increments within 1e-5 in L1 relative."""
    n = 3001
    x = W.cell_centres(n, 0.0, 10.0)
    h = 1.0 + 0.01 * np.sin(2 * np.pi * x / 10.0)
    fr = 1.0 + 0.002 * np.sin(4 * np.pi * x / 10.0)
    q = fr * np.sqrt(G * h) * h
    z = np.zeros(n)
    bcs = (W.BC_PERIODIC, W.BC_PERIODIC) if bc == "periodic" else (W.BC_TRANSMISSIVE, W.BC_TRANSMISSIVE)
    K = 20
    cfg = O.make_cfg(n, 0.0, 10.0, 0.9, O.grass(0.0, xi=W.XI_P04, g=G), bcs[0], bcs[1], ks=ks)
    ho, qo, zo, *_ = O.run(cfg, h, q, z, max_steps=K)
    gcfg = gpu.make_config(n, 0.0, 10.0, 0.9, 0.0, W.XI_P04, precision=gpu.FP32, bc_left=bcs[0],
                           bc_right=bcs[1], ks=ks, block_threads=256, reg_cap=80, step_kernel=2)
    with gpu.Solver(gcfg) as s:
        s.set_state(h, q, z)
        nodes, redo = gpu.adot_precision_stats(s.ctx)
        g0 = s.get_state()
        s.step(K)
        got = s.get_state()
    assert redo > 0.5 * nodes, (redo, nodes)
    for v, a, b, a0, ag in zip("hqz", got, (ho, qo, zo), (h, q, z), g0):
        inc, ref = a - ag, b - a0
        if v == "z":  # the fixed bed: motion at rounding level only, on both sides
            assert np.abs(inc).max() <= 1e-15 and np.abs(ref).max() <= 1e-15
            continue
        assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum(), np.abs(inc - ref).sum() / np.abs(ref).sum()


@pytest.mark.parametrize("block,cap,order", [(256, 64, 1), (256, 80, 1), (256, 80, 2)])
@pytest.mark.parametrize("case", ["smooth", "riemann"])
def test_fp32_step_cfl_maximum_equals_fresh_maximum(gpu, block, cap, order, case):
    """The float32 warp-tile steps (first order, and the second-order
    variant) form the next step's CFL maximum while they write the cells,
    skipping a cell's Newton iteration once its first iterate (an upper bound of
    the radius) falls below the lane's running maximum. The maximum must be the
    one the separate reduction (k_rho, no skipping) gives on the same state:
    after one step, the next step's dt from the running form equals, bit for
    bit, the first dt of a solver set to the state read back."""
    P = W.smooth_periodic(200_003) if case == "smooth" else W.movable_bed_riemann(150_001)
    kw = dict(block_threads=block, reg_cap=cap, step_kernel=2, order=order)
    for k in range(3):
        with gpu.Solver(gpu.config_for(P, gpu.FP32, **kw)) as s:
            s.set_state(P.h, P.q, P.z)
            s.step(k + 1)
            state = s.get_state()
            s.step(1)
            dt_run = s.query()[2]
        with gpu.Solver(gpu.config_for(P, gpu.FP32, **kw)) as s:
            s.set_state(*state)
            s.step(1)
            dt_fresh = s.query()[2]
        assert dt_run == dt_fresh, (k, dt_run, dt_fresh)
