"""The Grass law with a threshold velocity (Eq. GrassThr, read as
q_s = A_g sign(u) max(|u| - u_cr, 0)^3) on the GPU against the FP64 oracle:
edge fluctuations on seeded random edges whose quadrature nodes lie on both
sides of the threshold, a whole movable-bed Riemann run with the threshold
between the two initial velocities, and a run below the threshold everywhere,
where the bed must not move.

Tolerances as for the Grass law: fluctuations FP64 1e-12 and FP32 1e-4 of the
edge's max-norm; whole runs FP64 1e-12 of each variable's scale, FP32 the
increment W^K - W^0 within 1e-5 in L1 relative."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 9.81


def _rel_err(dm, dp, rm, rp):
    sc = np.abs(rm).max(axis=0) + np.abs(rp).max(axis=0)
    sc = np.where(sc > 0, sc, 1.0)
    return np.maximum(np.abs(dm - rm).max(axis=0), np.abs(dp - rp).max(axis=0)) / sc


@pytest.mark.parametrize("n", [7, 1000, 20011])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_random_edges_match_oracle(gpu, n, prec, tol):
    WL, WR = W.random_edges(n, 300 + n, fr_range=(-2.5, 2.5))
    Ag, xi, ucr = 0.01, W.XI_P04, 1.0
    uL, uR = np.abs(WL[1] / WL[0]), np.abs(WR[1] / WR[0])
    assert (np.minimum(uL, uR) < ucr).any() and (np.maximum(uL, uR) > ucr).any()
    rm, rp = O.fluct(O.grass_thr(Ag, ucr, xi=xi, g=G), WL, WR)
    cfg = gpu.make_config(16, 0.0, 1.0, 0.9, Ag, xi, precision=prec, law=gpu.LAW_GRASS_THR, u_cr=ucr)
    with gpu.Solver(cfg) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    err = _rel_err(dm, dp, rm, rp)
    assert err.max() <= tol, (err.max(), int(err.argmax()))


def _oracle_run(P, ucr, **kw):
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass_thr(P.Ag, ucr, xi=P.xi, g=P.g),
                     P.bc_left, P.bc_right, P.bcl, P.bcr)
    return O.run(cfg, P.h, P.q, P.z, **kw)


def _gpu_run(gpu, P, prec, ucr, steps=None, t_end=None):
    with gpu.Solver(gpu.config_for(P, prec, law=gpu.LAW_GRASS_THR, u_cr=ucr)) as s:
        s.set_state(P.h, P.q, P.z)
        if t_end is not None:
            s.run_to(t_end)
        else:
            s.step(steps)
        t, nsteps, _ = s.query()
        h, q, z = s.get_state()
    return h, q, z, t, nsteps


def test_riemann_run_with_threshold_between_the_states(gpu):
    """Left state u = 0.25 m/s above u_cr = 0.22, right state u = 0.2 below it."""
    P = W.movable_bed_riemann(701)
    ucr = 0.22
    ho, qo, zo, to, so, _ = _oracle_run(P, ucr, t_end=0.3)
    h, q, z, t, steps = _gpu_run(gpu, P, 0, ucr, t_end=0.3)
    assert steps == so and t == pytest.approx(to, rel=1e-13)
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(zo - P.z).max() > 1e-6  # the bed moves where the flow transports
    h, q, z, t, steps = _gpu_run(gpu, P, 1, ucr, t_end=0.3)
    assert t == 0.3
    for a, b, a0 in ((h, ho, P.h), (q, qo, P.q), (z, zo, P.z)):
        assert np.abs((a - a0) - (b - a0)).sum() <= 1e-5 * np.abs(b - a0).sum()


@pytest.mark.parametrize("prec", [0, 1])
def test_bed_fixed_below_threshold(gpu, prec):
    """u_cr above every velocity of the run: a = b = 0 at every node, the bed
    rows of A dW and |A| dW vanish, and the bed stays bit for bit where it was
    while h and q follow the oracle."""
    P = W.movable_bed_riemann(500)
    ucr = 10.0
    ho, qo, zo, to, so, _ = _oracle_run(P, ucr, max_steps=120)
    h, q, z, t, steps = _gpu_run(gpu, P, prec, ucr, steps=120)
    assert steps == 120
    assert np.array_equal(z, P.z)
    if prec == 0:
        for a, b in ((h, ho), (q, qo)):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    else:
        for a, b, a0 in ((h, ho, P.h), (q, qo, P.q)):
            assert np.abs((a - a0) - (b - a0)).sum() <= 1e-5 * np.abs(b - a0).sum()
