"""Pins of the oracle's second-order variant: MUSCL-Hancock in path-conservative
form (minmod slopes of (h + z, q, z), a Hancock half-step predictor with the
cell's own matrix, the DOT edge of Eq. DOTjumpN between predicted states and
the path integral of A inside each cell on the same Gauss-Legendre nodes; the
paper notes in Sec. 6 that nothing restricts the order). Checked against
things other than the oracle:

* with zero slopes the code path is the first-order scheme (Eq. scheme), bit
  for bit, so the assembly adds nothing when there is nothing to reconstruct;
* small periodic waves on a uniform movable-bed flow: the exact solution of the
  linearised system, sum_i r_i (l_i . dW0(x - lambda_i t)) from numpy's
  eigendecomposition, to O(eps^2); the variant converges to it at second order
  and the first-order scheme at first order;
* the exact movable-bed Riemann solution (oracle/exact.py, pinned to the
  textbook dam break and to the Rankine-Hugoniot conditions): lower error than
  the first-order scheme at the same grid;
* lake at rest, conservation of h and z on a periodic grid, mirror symmetry,
  and a domain of dependence of two cells per step.
"""
import numpy as np
import pytest

import oracle.exact as X
from paper_1912_04791_gb300 import workloads as W

G = 9.81


def _cfg(O, P, **kw):
    return O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                      P.bc_right, P.bcl, P.bcr, **kw)


@pytest.mark.parametrize("which", ["riemann", "smooth", "bump"])
def test_zero_slopes_is_the_first_order_scheme(oracle, which):
    O = oracle
    P = {"riemann": W.movable_bed_riemann(150), "smooth": W.smooth_periodic(160),
         "bump": W.gaussian_bump(120)}[which]
    a = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=60)
    b = O.run(_cfg(O, P, order=2, limiter=1), P.h, P.q, P.z, max_steps=60)
    assert a[4] == b[4] == 60 and a[3] == b[3]
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    c = O.run(_cfg(O, P, order=2), P.h, P.q, P.z, max_steps=60)
    assert max(np.abs(x - y).max() for x, y in zip(a[:3], c[:3])) > 1e-8  # the slopes do act


def _linear_waves(O, order, ns, eps=1e-7, T=0.3):
    """Errors of the run against the linearised exact solution (cell averages
    by 8-point Gauss-Legendre), L1 relative per variable."""
    h0, q0, Ag, xi = 1.0, 0.3, 0.005, W.XI_P04
    L = O.grass(Ag, xi=xi, g=G)
    lam, R = np.linalg.eig(O.flux_matrix(L, h0, q0))
    lam, R = lam.real, R.real
    Rinv = np.linalg.inv(R)

    def dW0(x):
        return np.array([eps * np.sin(2 * np.pi * x), 0.5 * eps * np.cos(2 * np.pi * x),
                         0.3 * eps * np.sin(2 * np.pi * x + 0.4)])

    def exact(x, t):
        return sum(np.outer(R[:, i], Rinv[i] @ dW0(x - lam[i] * t)) for i in range(3))

    def cellavg(n, t):
        s, w = np.polynomial.legendre.leggauss(8)
        xc = (np.arange(n) + 0.5) / n
        return sum(0.5 * wk * exact(xc + 0.5 / n * sk, t) for sk, wk in zip(s, w))

    errs = []
    for n in ns:
        d0 = cellavg(n, 0.0)
        cfg = O.make_cfg(n, 0.0, 1.0, 0.8, L, O.BC_PERIODIC, O.BC_PERIODIC, order=order)
        h, q, z, t, _, _ = O.run(cfg, h0 + d0[0], q0 + d0[1], d0[2], t_end=T)
        assert t == T
        de = cellavg(n, T)
        num = np.array([h - h0, q - q0, z])
        errs.append(np.abs(num - de).sum(axis=1) / np.abs(de).sum(axis=1))
    return np.array(errs)


def test_second_order_against_exact_linear_waves(oracle):
    """eps = 1e-7 keeps the nonlinear departure (O(eps) of the perturbation)
    far below the discretisation error on these grids."""
    ns = (50, 100, 200, 400)
    e2 = _linear_waves(oracle, 2, ns)
    e1 = _linear_waves(oracle, 1, ns)
    r2 = np.log2(e2[:-1] / e2[1:])
    r1 = np.log2(e1[:-1] / e1[1:])
    assert (r2 > 1.9).all() and (r2 < 2.2).all(), r2
    assert (r1 > 0.9).all() and (r1 < 1.1).all(), r1
    assert (e2[-1] < 0.01 * e1[-1]).all()


def test_riemann_error_below_first_order(oracle):
    """Movable-bed Riemann problem of the benchmark's small case against its
    exact solution at t = 1 s: the second-order variant converges, with the
    smaller error on every grid and variable."""
    O = oracle
    R = X.MovableBedRiemann((2.0, 0.5, 0.0), (1.0, 0.2, 0.5), Ag=0.01, xi=W.XI_P04)
    prev = None
    for n in (400, 800, 1600):  # at 200 cells the bed wave is not yet resolved
        P = W.movable_bed_riemann(n)
        xc = W.cell_centres(n, 0.0, 10.0)
        ex = R.sample(xc, 1.0, 5.0)
        errs = []
        for order in (1, 2):
            h, q, z, t, _, _ = O.run(_cfg(O, P, order=order), P.h, P.q, P.z, t_end=1.0)
            errs.append([np.abs(a - b).sum() / np.abs(b).sum() for a, b in zip((h, q, z), ex)])
        e1, e2 = np.array(errs)
        # the bed step is a near-stationary discontinuity where neither order
        # gains much; h and q gain more than a factor 1/0.6
        assert (e2 < e1).all() and (e2[:2] < 0.6 * e1[:2]).all(), (n, e1, e2)
        if prev is not None:
            assert (e2 < prev).all()
        prev = e2


def test_lake_at_rest(oracle):
    O = oracle
    P = W.lake_at_rest(300)
    h, q, z, t, steps, _ = O.run(_cfg(O, P, order=2), P.h, P.q, P.z, max_steps=200)
    assert steps == 200
    assert np.abs(q).max() <= 1e-12
    assert np.abs(h + z - 1.0).max() <= 1e-13


def test_h_and_z_conserved_on_a_periodic_grid(oracle):
    """The h rows of the edge and cell terms are q jumps that telescope around
    the periodic grid (a missing cell term would leave the edges' jumps of the
    reconstruction unbalanced); the z rows are the same Gauss sums of a dq_s
    and b dq as the first-order scheme's."""
    O = oracle
    P = W.smooth_periodic(400)
    h, q, z, t, steps, _ = O.run(_cfg(O, P, order=2), P.h, P.q, P.z, max_steps=300)
    assert abs(h.sum() - P.h.sum()) <= 1e-13 * P.h.sum()
    assert abs(z.sum() - P.z.sum()) <= 1e-13 * np.abs(P.z).sum()
    assert np.abs(h - P.h).max() > 1e-4


def test_mirror_symmetry(oracle):
    O = oracle
    P = W.movable_bed_riemann(120)
    a = O.run(_cfg(O, P, order=2), P.h, P.q, P.z, max_steps=60)
    b = O.run(_cfg(O, P, order=2), P.h[::-1].copy(), -P.q[::-1].copy(), P.z[::-1].copy(),
              max_steps=60)
    sc = np.abs(a[0]).max()
    assert np.abs(a[0] - b[0][::-1]).max() <= 1e-12 * sc
    assert np.abs(a[1] + b[1][::-1]).max() <= 1e-12 * sc
    assert np.abs(a[2] - b[2][::-1]).max() <= 1e-12 * sc


def test_two_cell_domain_of_dependence(oracle):
    """A cell's new value depends on cells i-2 .. i+2 (the neighbours' slopes
    feed the edge states). On a linear background in h, a one-cell dip at cell
    32 lowers the left neighbour's minmod slope, which reaches cell 30 in one
    step; after k steps the runs with and without the dip differ only within
    2k cells of it."""
    O = oracle
    n = 64
    x = W.cell_centres(n, 0.0, 1.0)
    h, q, z = 1.0 + 0.05 * x, np.full(n, 0.3), np.zeros(n)
    hp = h.copy()
    hp[32] -= 2e-4  # smaller than the background step 0.05 / 64
    cfg = O.make_cfg(n, 0.0, 1.0, 0.8, O.grass(0.005, xi=W.XI_P04, g=G), O.BC_TRANSMISSIVE,
                     O.BC_TRANSMISSIVE, order=2)
    for k in (1, 2, 3):
        a = O.run(cfg, h, q, z, max_steps=k)
        b = O.run(cfg, hp, q, z, max_steps=k)
        moved = np.nonzero(np.any([np.abs(u - v) > 0 for u, v in zip(a[:3], b[:3])], axis=0))[0]
        assert moved.min() >= 32 - 2 * k and moved.max() <= 32 + 2 * k, (k, moved)
        if k == 1:
            assert moved.min() == 30, moved


def test_friction_and_feed_are_first_order_only(oracle):
    O = oracle
    P = W.soni_aggradation(50)
    L = O.power(P.Ag, 5.0, xi=P.xi, g=P.g)
    for ks, bcl in ((49.4, P.bcl), (0.0, P.bcl)):
        cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, L, P.bc_left, P.bc_right, bcl, P.bcr, ks=ks,
                         order=2)
        with pytest.raises(O.OracleError):
            O.run(cfg, P.h, P.q, P.z, max_steps=1)
