"""The friction source (Eq. scheme with S = (0, -g h s_f, 0), Strickler
s_f = q|q| / (K_s^2 h^(10/3)), Sec. 2), the sediment feed through an end and the
slope-continuing ghosts (Sec. 5.1, the Soni case), and the power law of the
velocity (Eq. Soni_qs) on the GPU, through the C ABI, against the FP64 oracle.

Tolerances: FP64 every value within 1e-12 of the variable's scale (and the
same step count). FP32 (float-float state, float32 fluctuations and source):
every value within 1e-6 of the variable's scale, and the bed increment
z^K - z^0 within 1e-4 in L1 relative. On these sloping, rubbing flows the
momentum change of a step is the small difference of two balanced terms (the
bed-slope term g h dz and the friction, each ~1e-3 of q per step); their
float32 rounding (~1e-7) is a large part of that difference, so the
increment-relative criterion of the other FP32 runs does not apply to h and q,
while the error stays far below 1e-6 of the state because friction damps it
within a few seconds. A wrong source or feed term is >= 1e-3 of the state
after one step.
Fluctuations of single edges: FP64 1e-12 and FP32 1e-4 of the edge's max-norm.
An equilibrium is kept to 1e-13 (FP64) and 1e-5 (FP32) of the state, while a
ghost that copies the bed instead of continuing the slope drives a 1-3 %
departure in the same run."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 9.81
KS, H0, Q0 = 49.4, 0.05, 0.02


def _soni_kw(gpu, P, **kw):
    out = {"law": gpu.LAW_POWER, "beta": P.extra["beta"], "ks": P.extra["ks"]}
    out.update(kw)
    return out


def _oracle_run(P, law, ks, **run):
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, law, P.bc_left, P.bc_right, P.bcl, P.bcr,
                     ks=ks)
    return O.run(cfg, P.h, P.q, P.z, **run)


def _gpu_run(gpu, P, prec, steps=None, t_end=None, **kw):
    with gpu.Solver(gpu.config_for(P, prec, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        if t_end is not None:
            s.run_to(t_end)
        else:
            s.step(steps)
        t, nsteps, _ = s.query()
        h, q, z = s.get_state()
    return h, q, z, t, nsteps


def _check(prec, got, ref, P, ctx=""):
    tol = 1e-12 if prec == 0 else 1e-6
    for name, a, b in zip("hqz", got[:3], ref[:3]):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= tol, (ctx, name, err)
    if prec == 1:
        num = np.abs(got[2] - ref[2]).sum()
        den = np.abs(ref[2] - P.z).sum()
        assert num <= 1e-4 * den, (ctx, "dz", num / den)


def _rel_err(dm, dp, rm, rp):
    sc = np.abs(rm).max(axis=0) + np.abs(rp).max(axis=0)
    sc = np.where(sc > 0, sc, 1.0)
    return np.maximum(np.abs(dm - rm).max(axis=0), np.abs(dp - rp).max(axis=0)) / sc


@pytest.mark.parametrize("beta,ucr", [(5.0, 0.0), (2.5, 0.3), (1.0, 0.0)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_power_law_edges_match_oracle(gpu, beta, ucr, prec, tol):
    n = 4099
    WL, WR = W.random_edges(n, 700 + int(10 * beta), fr_range=(-2.5, 2.5))
    A, xi = 0.004, W.XI_P04
    rm, rp = O.fluct(O.power(A, beta, u_cr=ucr, xi=xi, g=G), WL, WR)
    cfg = gpu.make_config(16, 0.0, 1.0, 0.9, A, xi, precision=prec, law=gpu.LAW_POWER, beta=beta,
                          u_cr=ucr)
    with gpu.Solver(cfg) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    err = _rel_err(dm, dp, rm, rp)
    assert err.max() <= tol, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("prec", [0, 1])
def test_soni_run_matches_oracle(gpu, prec):
    """The Soni case with its printed data (100 cells, 2400 s, about 1e4
    steps): power law beta = 5, Strickler friction, feed and slope-continuing
    ghosts all active."""
    P = W.soni_aggradation()
    law = O.power(P.Ag, P.extra["beta"], xi=P.xi, g=P.g)
    ref = _oracle_run(P, law, P.extra["ks"], t_end=P.t_end)
    got = _gpu_run(gpu, P, prec, t_end=P.t_end, **_soni_kw(gpu, P))
    assert got[3] == P.t_end
    if prec == 0:
        assert got[4] == ref[4]
    _check(prec, got, ref, P, "soni")
    assert got[2][0] - P.z[0] > 0.03  # the bed aggrades at the feed


@pytest.mark.parametrize("step_kernel", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_normal_flow_stays(gpu, step_kernel, prec):
    """Fixed bed (A = 0) at the textbook normal slope of the Soni flow: friction
    balances the bed-slope term and the ghosts continue the slope, in both step
    kernels."""
    s = (Q0 / (KS * H0 ** (5.0 / 3.0))) ** 2
    P = dataclasses.replace(W.soni_aggradation(n=300, s0=s), Ag=0.0, bcl=(Q0, 0.0, 0.0))
    h, q, z, t, steps = _gpu_run(gpu, P, prec, steps=500, step_kernel=step_kernel,
                                 **_soni_kw(gpu, P))
    tol = 1e-13 if prec == 0 else 1e-5
    assert steps == 500
    assert np.abs(q - Q0).max() <= tol * Q0
    assert np.abs(h - H0).max() <= tol * H0
    assert np.abs(z - P.z).max() <= tol * np.abs(P.z).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_friction_decay_matches_oracle(gpu, prec):
    """Uniform periodic flow on a flat bed decelerated by friction alone; the
    oracle's run is pinned to the closed-form decay q0 / (1 + k q0 t)."""
    n = 1000
    P = W.Problem("decay", n, 0.0, 1.0, 0.8, 5.0, 0.0, 1.0, np.full(n, 0.25), np.full(n, 0.5),
                  np.zeros(n), W.BC_PERIODIC, W.BC_PERIODIC)
    ref = _oracle_run(P, O.grass(0.0, xi=1.0, g=G), 20.0, t_end=P.t_end)
    got = _gpu_run(gpu, P, prec, t_end=P.t_end, ks=20.0)
    assert got[3] == P.t_end
    if prec == 0:
        assert got[4] == ref[4]
        assert np.abs(got[1] - ref[1]).max() <= 1e-13 * 0.5
    else:
        d, dref = got[1] - 0.5, ref[1] - 0.5
        assert np.abs(d - dref).max() <= 1e-5 * np.abs(dref).max()
    assert np.ptp(got[1]) <= (0.0 if prec == 0 else 1e-7)
    assert np.array_equal(got[0], P.h) and not got[2].any()


@pytest.mark.parametrize("prec,rtol", [(0, 1e-12), (1, 1e-5)])
def test_feed_first_step(gpu, prec, rtol):
    """Uniform flow on a flat bed (Grass law, h = 0.5 m, u = 0.5 m/s, values a
    float represents exactly) fed d more than its
    own discharge: one step changes only the first cell's bed, by dt/dx xi d."""
    n, qs = 64, 0.01 * 0.5 ** 3
    d = 0.37 * qs
    P = W.Problem("feed", n, 0.0, 10.0, 0.9, 1.0, 0.01, W.XI_P04, np.full(n, 0.5), np.full(n, 0.25),
                  np.zeros(n), W.BC_INFLOW_QS, W.BC_TRANSMISSIVE, (0.25, qs + d, 0.0))
    h, q, z, t, steps = _gpu_run(gpu, P, prec, steps=1)
    assert steps == 1
    assert np.array_equal(h, P.h) and np.array_equal(q, P.q) and not z[1:].any()
    assert z[0] == pytest.approx(t / P.dx * W.XI_P04 * d, rel=rtol)
    # fed exactly its own discharge, nothing moves
    P0 = dataclasses.replace(P, bcl=(0.25, qs, 0.0))
    h, q, z, t, steps = _gpu_run(gpu, P0, prec, steps=100)
    assert np.abs(z).max() <= (1e-17 if prec == 0 else 1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_feed_from_either_end(gpu, prec):
    """A sloping flume with friction fed from the left, and its mirror image fed
    from the right with the flow towards -x: each matches the oracle, and the
    FP64 runs mirror each other."""
    n, steps = 240, 400
    x = W.cell_centres(n, 0.0, 10.0)
    z0 = 0.5 - 0.002 * x + 0.01 * np.sin(x)
    qin = 2.5 * 0.01 * 0.5 ** 3
    left = W.Problem("feed_left", n, 0.0, 10.0, 0.9, 1.0, 0.01, W.XI_P04, np.full(n, 0.4),
                     np.full(n, 0.2), z0, W.BC_INFLOW_QS, W.BC_OUTFLOW_HS, (0.2, qin, 0.0),
                     (0.4, 0.0, 0.0))
    right = W.Problem("feed_right", n, 0.0, 10.0, 0.9, 1.0, 0.01, W.XI_P04, np.full(n, 0.4),
                      np.full(n, -0.2), z0[::-1].copy(), W.BC_OUTFLOW_HS, W.BC_INFLOW_QS,
                      (0.4, 0.0, 0.0), (-0.2, -qin, 0.0))
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    runs = []
    for P in (left, right):
        ref = _oracle_run(P, law, 25.0, max_steps=steps)
        got = _gpu_run(gpu, P, prec, steps=steps, ks=25.0)
        _check(prec, got, ref, P, P.name)
        runs.append(got)
    if prec == 0:
        a, b = runs
        for k, sign in ((0, 1), (1, -1), (2, 1)):
            assert np.abs(sign * b[k][::-1] - a[k]).max() <= 1e-12 * np.abs(a[k]).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_block_and_warp_kernels_agree(gpu, prec):
    """The block kernel and the warp-tile kernel, each with the friction source,
    the feed and the extrapolating ghosts compiled in, on the Soni case at 2000
    cells against each other and the oracle."""
    P = W.soni_aggradation(n=2000)
    law = O.power(P.Ag, P.extra["beta"], xi=P.xi, g=P.g)
    ref = _oracle_run(P, law, P.extra["ks"], max_steps=300)
    out = []
    for sk in (1, 2):
        got = _gpu_run(gpu, P, prec, steps=300, step_kernel=sk, **_soni_kw(gpu, P))
        _check(prec, got, ref, P, f"step_kernel {sk}")
        out.append(got)
    if prec == 0:
        for a, b in zip(out[0][:3], out[1][:3]):
            assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()
