"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

Single channel: the smooth periodic workload at N = 1e7 (two 240 MB
float-float state buffers, larger than L2), autotuned kernel variant (as in
bench.py) and the persistent warp-tile variant pinned, three time steps,
against the oracle's own three-step run of the full grid (its CFL maximum over
all 1e7 cells, every edge's fluctuations) compared cell by cell.
Ensemble: the 4096-channel movable-bed Riemann ensemble (8.6e7 cells) in the
default persistent channel loops (as the benchmark times it) and in per-step
launches, with a set of sampled channels (longest, shortest, random) run by the
oracle one by one to the same end time. The single-channel
workload also runs with the Strickler friction source (K_s = 30) and with the
second-order MUSCL-Hancock variant.

Tolerances as for the small cases: FP64 every value within 1e-12 of the
variable's scale and the same time; FP32 (float-float state, float32
fluctuations) the increment W^K - W^0 within 1e-5 in L1 relative and 1e-4 of
its largest entry cell by cell, the time within 1e-5 (the CFL maximum is a
float32 spectral radius)."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N_FULL = 10_000_000
K = 3


@pytest.fixture(scope="module")
def full_problem():
    return W.smooth_periodic(N_FULL)


@pytest.fixture(scope="module")
def full_oracle(full_problem, oracle):
    P = full_problem
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                     P.bc_right, P.bcl, P.bcr)
    h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=K)
    assert steps == K
    return h, q, z, t


def _gpu_run(gpu, P, prec, **kw):
    with gpu.Solver(gpu.config_for(P, prec, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(K)
        t, steps, _ = s.query()
        h, q, z = s.get_state()
    assert steps == K
    return h, q, z, t


@pytest.mark.parametrize("variant", [{}, {"block_threads": 256, "reg_cap": 64, "step_kernel": 2}],
                         ids=["autotuned", "warp256x64"])
def test_fp64_full_size_matches_oracle(gpu, full_problem, full_oracle, variant):
    P = full_problem
    h, q, z, t = _gpu_run(gpu, P, gpu.FP64, **variant)
    ho, qo, zo, to = full_oracle
    assert t == pytest.approx(to, rel=1e-13)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("variant", [{}, {"block_threads": 256, "reg_cap": 64, "step_kernel": 2}],
                         ids=["autotuned", "warp256x64"])
def test_fp32_full_size_matches_oracle(gpu, full_problem, full_oracle, variant):
    P = full_problem
    h, q, z, t = _gpu_run(gpu, P, gpu.FP32, **variant)
    ho, qo, zo, to = full_oracle
    assert t == pytest.approx(to, rel=1e-5)
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        inc, ref = a - a0, b - a0
        err = np.abs(inc - ref)
        assert err.sum() <= 1e-5 * np.abs(ref).sum(), err.sum() / np.abs(ref).sum()
        assert err.max() <= 1e-4 * np.abs(ref).max(), err.max() / np.abs(ref).max()


KS_FULL = 30.0  # Strickler friction (Sec. 2) on the same workload: s_f ~ 1e-4


@pytest.fixture(scope="module")
def full_oracle_friction(full_problem, oracle):
    P = full_problem
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                     P.bc_right, P.bcl, P.bcr, ks=KS_FULL)
    h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=K)
    assert steps == K
    return h, q, z, t


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_full_size_with_friction_matches_oracle(gpu, full_problem, full_oracle_friction, prec):
    """The same workload with the Strickler friction source: the step kernels
    with the source compiled in, warp tiles 256 x 64 as the benchmark's friction
    line times them."""
    P = full_problem
    h, q, z, t = _gpu_run(gpu, P, getattr(gpu, prec), block_threads=256, reg_cap=64, step_kernel=2,
                          ks=KS_FULL)
    ho, qo, zo, to = full_oracle_friction
    if prec == "FP64":
        assert t == pytest.approx(to, rel=1e-13)
        for a, b in ((h, ho), (q, qo), (z, zo)):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        return
    assert t == pytest.approx(to, rel=1e-5)
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        inc, ref = a - a0, b - a0
        err = np.abs(inc - ref)
        assert err.sum() <= 1e-5 * np.abs(ref).sum(), err.sum() / np.abs(ref).sum()
        assert err.max() <= 1e-4 * np.abs(ref).max(), err.max() / np.abs(ref).max()


@pytest.fixture(scope="module")
def full_oracle_order2(full_problem, oracle):
    P = full_problem
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                     P.bc_right, P.bcl, P.bcr, order=2)
    h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=K)
    assert steps == K
    return h, q, z, t


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_full_size_second_order_matches_oracle(gpu, full_problem, full_oracle_order2, prec):
    """The second-order variant (MUSCL-Hancock) on the same workload, autotuned
    among its warp-tile variants as the benchmark's second-order line runs it."""
    P = full_problem
    h, q, z, t = _gpu_run(gpu, P, getattr(gpu, prec), order=2)
    ho, qo, zo, to = full_oracle_order2
    if prec == "FP64":
        assert t == pytest.approx(to, rel=1e-13)
        for a, b in ((h, ho), (q, qo), (z, zo)):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        return
    assert t == pytest.approx(to, rel=1e-5)
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        inc, ref = a - a0, b - a0
        err = np.abs(inc - ref)
        assert err.sum() <= 1e-5 * np.abs(ref).sum(), err.sum() / np.abs(ref).sum()
        assert err.max() <= 1e-4 * np.abs(ref).max(), err.max() / np.abs(ref).max()


def _sampled_channels(E, k_random=4, seed=5):
    order = np.argsort(E.n_cells)
    rng = np.random.default_rng(seed)
    mid = rng.choice(order[2:-2], k_random, replace=False)
    return sorted(set(order[:2].tolist() + order[-2:].tolist() + mid.tolist()))


@pytest.mark.parametrize("kern", [0, 4], ids=["persistent", "per_step"])
@pytest.mark.parametrize("prec,t_end", [("FP64", 0.002), ("FP32", 0.005)])
def test_full_ensemble_sampled_channels_match_oracle(gpu, oracle, prec, t_end, kern):
    E = W.riemann_ensemble(4096)
    assert int(E.n_cells.sum()) > 8e7
    with gpu.Ensemble.from_workload(E, getattr(gpu, prec), step_kernel=kern) as ens:
        ens.set_state(E.h, E.q, E.z)
        ens.run_to(t_end)
        t, steps, _ = ens.query()
        h, q, z = ens.get_state()
    assert (t == t_end).all()
    o = E.offsets
    for c in _sampled_channels(E):
        hc, qc, zc = E.channel(c)
        cfg = O.make_cfg(int(E.n_cells[c]), 0.0, float(E.length[c]), E.cfl,
                         O.grass(float(E.Ag[c]), xi=E.xi, g=9.81))
        ho, qo, zo, to, so, _ = O.run(cfg, hc, qc, zc, t_end=t_end)
        sl = slice(o[c], o[c + 1])
        for a, b, a0 in ((h[sl], ho, hc), (q[sl], qo, qc), (z[sl], zo, zc)):
            if prec == "FP64":
                assert steps[c] == so, (c, steps[c], so)
                assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), c
            else:
                # increments W(t_end) - W(0), not whole states
                inc, ref = a - a0, b - a0
                assert np.abs(ref).sum() > 0.0, c
                assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum(), \
                    (c, np.abs(inc - ref).sum() / np.abs(ref).sum())


# Trans-critical flow over the Gaussian bump at N = 1e6 (inflow q = 0.6, outflow
# h = 0.33): the fixed-bed flow spun up by the oracle on 2000 cells to t = 6 s
# (it crosses Fr = 1 over the crest), prolonged to 1e6 cells, then K_BUMP steps
# with the fixed bed (A_g = 0: the roots u - c, 0, u + c coalesce at Fr = 1, where
# the float32 kernels redo nodes in float64), with Grass (A_g = 0.001) and with
# Meyer-Peter & Mueller (s = 2.65, d50 = 1 mm, n = 0.02).
N_BUMP = 1_000_000
K_BUMP = 100
MPM = dict(s_rel=2.65, d50=1e-3, manning_n=0.02)


@pytest.fixture(scope="module")
def bump_spin_up(oracle):
    P0 = W.gaussian_bump(2000, Ag=0.0)
    cfg = O.make_cfg(P0.n, P0.x_min, P0.x_max, P0.cfl, O.grass(0.0, xi=P0.xi), P0.bc_left,
                     P0.bc_right, P0.bcl, P0.bcr)
    h, q, z, t, *_ = O.run(cfg, P0.h, P0.q, P0.z, t_end=6.0)
    return h, q


@pytest.mark.parametrize("kind", ["fixed", "grass", "mpm"])
def test_bump_full_size_matches_oracle(gpu, bump_spin_up, kind):
    P = W.gaussian_bump_prolonged(*bump_spin_up, N_BUMP, Ag=0.0 if kind == "fixed" else 0.001)
    fr = P.q / P.h / np.sqrt(P.g * P.h)
    assert fr.min() < 0.9 and fr.max() > 1.1  # trans-critical
    if kind == "mpm":
        olaw, kw = O.mpm(xi=P.xi, **MPM), dict(law=gpu.LAW_MPM, **MPM)
    else:
        olaw, kw = O.grass(P.Ag, xi=P.xi), {}
    ocfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, olaw, P.bc_left, P.bc_right, P.bcl, P.bcr)
    ho, qo, zo, to, so, _ = O.run(ocfg, P.h, P.q, P.z, max_steps=K_BUMP)
    assert so == K_BUMP
    h, q, z, t = _gpu_run_k(gpu, P, gpu.FP64, K_BUMP, **kw)
    assert t == pytest.approx(to, rel=1e-13)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= 1e-12, err
    with gpu.Solver(gpu.config_for(P, gpu.FP32, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        nodes, redo = gpu.adot_precision_stats(s.ctx)
        s.step(K_BUMP)
        h, q, z = s.get_state()
    assert nodes == 3 * (N_BUMP + 1)
    if kind == "fixed":
        assert redo > 0  # coalescence at the crest: the float64 redo fires
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        inc, ref = a - a0, b - a0
        if kind == "fixed" and a0 is P.z:
            # a fixed bed stays in place up to the rounding of its zero row of |A| dW
            assert np.abs(inc).max() <= 1e-8 * np.abs(a0).max()
            continue
        assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum(), \
            np.abs(inc - ref).sum() / np.abs(ref).sum()


def _gpu_run_k(gpu, P, prec, k, **kw):
    with gpu.Solver(gpu.config_for(P, prec, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(k)
        t, steps, _ = s.query()
        h, q, z = s.get_state()
    assert steps == k
    return h, q, z, t
