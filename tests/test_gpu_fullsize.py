"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

Single channel: the smooth periodic workload at N = 1e7 (two 240 MB
float-float state buffers, larger than L2), autotuned kernel variant (as in
bench.py) and the persistent warp-tile variant pinned, three time steps,
against the oracle's own three-step run of the full grid (its CFL maximum over
all 1e7 cells, every edge's fluctuations) compared cell by cell.
Ensemble: the 4096-channel movable-bed Riemann ensemble (8.6e7 cells, one
launch per step), with a set of sampled channels (longest, shortest, random)
run by the oracle one by one to the same end time. The single-channel
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


@pytest.mark.parametrize("prec,t_end", [("FP64", 0.002), ("FP32", 0.005)])
def test_full_ensemble_sampled_channels_match_oracle(gpu, oracle, prec, t_end):
    E = W.riemann_ensemble(4096)
    assert int(E.n_cells.sum()) > 8e7
    with gpu.Ensemble.from_workload(E, getattr(gpu, prec)) as ens:
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
        for a, b in ((h[sl], ho), (q[sl], qo), (z[sl], zo)):
            if prec == "FP64":
                assert steps[c] == so, (c, steps[c], so)
                assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), c
            else:
                assert np.abs(a - b).sum() <= 1e-5 * max(np.abs(b).sum(), 1e-12), c
