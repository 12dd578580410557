"""The second-order MUSCL-Hancock variant (order = 2: minmod slopes of h + z, q,
z, a Hancock half-step predictor, DOT edges of Eq. DOTjumpN between the
predicted states and the path integral of A inside each cell; Sec. 6 leaves the
order open) on the GPU, through the C ABI, against the FP64 oracle.

Tolerances as for the first-order runs: FP64 every value within 1e-12 of the
variable's scale and the same step count; FP32 (float-float state, float32
arithmetic) the increment W^K - W^0 within 1e-5 in L1 relative (smooth flow)
or 1e-4 (flows with jumps, where minmod switches on rounding-level
differences of the slopes)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WARP_VARIANTS = [(256, 64), (128, 64), (128, 72), (256, 80)]


def _oracle(P, **run):
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                     P.bc_right, P.bcl, P.bcr, order=2)
    return O.run(cfg, P.h, P.q, P.z, **run)


def _gpu(gpu, P, prec, steps=None, t_end=None, **kw):
    with gpu.Solver(gpu.config_for(P, prec, order=2, **kw)) as s:
        s.set_state(P.h, P.q, P.z)
        if t_end is not None:
            s.run_to(t_end)
        else:
            s.step(steps)
        t, nsteps, _ = s.query()
        h, q, z = s.get_state()
    return h, q, z, t, nsteps


def _check(prec, got, ref, P, tol32=1e-5):
    if prec == 0:
        assert got[4] == ref[4]
        assert got[3] == pytest.approx(ref[3], rel=1e-13)
        for name, a, b in zip("hqz", got[:3], ref[:3]):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), name
    else:
        for name, a, b, a0 in zip("hqz", got[:3], ref[:3], (P.h, P.q, P.z)):
            num = np.abs((a - a0) - (b - a0)).sum()
            den = np.abs(b - a0).sum()
            assert num <= tol32 * den, (name, num / den)


PROBLEMS = {
    "riemann": (lambda: W.movable_bed_riemann(701), {"t_end": 0.3}, 1e-4),
    "smooth": (lambda: W.smooth_periodic(1000), {"steps": 200}, 1e-5),
    "bump": (lambda: W.gaussian_bump(500), {"steps": 200}, 1e-4),
}


@pytest.mark.parametrize("which", list(PROBLEMS))
@pytest.mark.parametrize("prec", [0, 1])
def test_runs_match_oracle(gpu, which, prec):
    make, run, tol32 = PROBLEMS[which]
    P = make()
    if "t_end" in run:
        ref = _oracle(P, t_end=run["t_end"])
        got = _gpu(gpu, P, prec, t_end=run["t_end"])
    else:
        ref = _oracle(P, max_steps=run["steps"])
        got = _gpu(gpu, P, prec, steps=run["steps"])
    _check(prec, got, ref, P, tol32)


@pytest.mark.parametrize("n", [1, 2, 3, 29, 30, 31, 61, 149])
def test_small_and_ragged_periodic_grids(gpu, n):
    """Grids smaller than a tile, one cell more or less than a tile, and ragged
    tails: the wrap of cells around the periodic ends in every lane."""
    P = W.smooth_periodic(n)
    ref = _oracle(P, max_steps=40)
    got = _gpu(gpu, P, 0, steps=40)
    _check(0, got, ref, P)


@pytest.mark.parametrize("n", [2, 3, 30, 31, 89])
def test_small_and_ragged_grids_with_ghosts(gpu, n):
    P = W.movable_bed_riemann(n)
    ref = _oracle(P, max_steps=25)
    got = _gpu(gpu, P, 0, steps=25)
    _check(0, got, ref, P)


@pytest.mark.parametrize("prec", [0, 1])
def test_sloping_flume_with_continued_bed(gpu, prec):
    """The slope-continuing outflow ghost (OUTFLOW_HS) and the power law of
    Eq. Soni_qs with the second-order variant: the Soni flume without friction,
    inflow q at the left end."""
    S = W.soni_aggradation(n=200)
    P = dataclasses.replace(S, bc_left=W.BC_INFLOW_Q)
    law = O.power(P.Ag, 5.0, xi=P.xi, g=P.g)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, law, P.bc_left, P.bc_right, P.bcl, P.bcr, order=2)
    ref = O.run(cfg, P.h, P.q, P.z, max_steps=150)
    got = _gpu(gpu, P, prec, steps=150, law=gpu.LAW_POWER, beta=5.0)
    _check(prec, got, ref, P, 1e-4)


@pytest.mark.parametrize("block,cap", WARP_VARIANTS)
def test_every_warp_variant_matches_oracle(gpu, block, cap):
    P = W.movable_bed_riemann(1003)
    ref = _oracle(P, max_steps=120)
    got = _gpu(gpu, P, 0, steps=120, block_threads=block, reg_cap=cap, step_kernel=2)
    _check(0, got, ref, P)


@pytest.mark.parametrize("prec", [0, 1])
def test_lake_at_rest(gpu, prec):
    """FP64 to rounding; FP32 within the first-order kernel's FP32 bounds (q
    2e-5, h + z 1e-3 after 300 steps): in float32 the products c^2 dh and c^2 dz
    that cancel at rest are rounded separately (one of them fused), so neither
    order is exactly balanced there."""
    P = W.lake_at_rest(1000)
    h, q, z, t, steps = _gpu(gpu, P, prec, steps=300)
    assert steps == 300
    qb, eb = (1e-13, 1e-13) if prec == 0 else (2e-5, 1e-3)
    assert np.abs(q).max() <= qb and np.abs(h + z - 1.0).max() <= eb


def test_second_order_converges_on_the_gpu(gpu):
    """Small periodic waves on a uniform movable-bed flow against the exact
    solution of the linearised system (numpy eigendecomposition of the
    oracle's A): FP64 runs of both orders, rates about 2 and 1."""
    h0, q0, Ag, xi, eps, T = 1.0, 0.3, 0.005, W.XI_P04, 1e-7, 0.3
    lam, R = np.linalg.eig(O.flux_matrix(O.grass(Ag, xi=xi, g=9.81), h0, q0))
    lam, R = lam.real, R.real
    Rinv = np.linalg.inv(R)

    def dW0(x):
        return np.array([eps * np.sin(2 * np.pi * x), 0.5 * eps * np.cos(2 * np.pi * x),
                         0.3 * eps * np.sin(2 * np.pi * x + 0.4)])

    def cellavg(n, t):
        s, w = np.polynomial.legendre.leggauss(8)
        xc = (np.arange(n) + 0.5) / n
        return sum(0.5 * wk * sum(np.outer(R[:, i], Rinv[i] @ dW0(xc + 0.5 / n * sk - lam[i] * t))
                                  for i in range(3)) for sk, wk in zip(s, w))

    rates = {}
    for order in (1, 2):
        errs = []
        for n in (100, 200, 400):
            d0 = cellavg(n, 0.0)
            P = W.Problem("waves", n, 0.0, 1.0, 0.8, T, Ag, xi, h0 + d0[0], q0 + d0[1], d0[2],
                          W.BC_PERIODIC, W.BC_PERIODIC)
            with gpu.Solver(gpu.config_for(P, gpu.FP64, order=order)) as s:
                s.set_state(P.h, P.q, P.z)
                s.run_to(T)
                h, q, z = s.get_state()
            de = cellavg(n, T)
            errs.append(np.abs(np.array([h - h0, q - q0, z]) - de).sum(axis=1) / np.abs(de).sum(axis=1))
        errs = np.array(errs)
        rates[order] = np.log2(errs[:-1] / errs[1:])
    assert (rates[2] > 1.9).all(), rates
    assert (rates[1] < 1.1).all(), rates


def test_order_is_part_of_the_checkpoint_fingerprint(gpu):
    P = W.smooth_periodic(500)
    with gpu.Solver(gpu.config_for(P, gpu.FP64, order=2)) as a:
        a.set_state(P.h, P.q, P.z)
        a.step(5)
        blob = a.checkpoint()
        with gpu.Solver(gpu.config_for(P, gpu.FP64)) as b:
            b.set_state(P.h, P.q, P.z)
            with pytest.raises(gpu.AdotError):
                b.restore(blob)
        with gpu.Solver(gpu.config_for(P, gpu.FP64, order=2)) as c:
            c.set_state(P.h, P.q, P.z)
            c.restore(blob)
            a.step(7)
            c.step(7)
            for x, y in zip(a.get_state(), c.get_state()):
                assert np.array_equal(x, y)
