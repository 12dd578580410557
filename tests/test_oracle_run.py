"""Pins of the oracle's time loop (Eq. scheme, S = 0) against exact solutions
(textbook shallow-water Riemann problem, the Test 2 closed form of Sec. 4.2),
conservation, lake at rest, upwind structure, mirror symmetry and the CFL
time-step reading."""
import numpy as np
import pytest

from oracle import exact as X
from paper_1912_04791_gb300 import workloads as W

G = 9.81


def _cfg(O, P, method=0):
    law = O.grass(P.Ag, xi=P.xi, g=P.g)
    return O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, law, P.bc_left, P.bc_right, P.bcl, P.bcr,
                      method)


def test_mass_and_bed_conserved_periodic(oracle):
    """Row 1 of D- + D+ is dq, so sum h telescopes exactly on a periodic grid.
    Row 3 is the GL3 quadrature of xi dq_s/ds, exact to rounding on smooth data
    where the rational integrand is resolved, so sum z is conserved too."""
    O = oracle
    P = W.smooth_periodic(256)
    h, q, z, t, steps, _ = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=300)
    assert steps == 300
    assert abs(h.sum() - P.h.sum()) <= 1e-13 * P.h.sum()
    assert abs(z.sum() - P.z.sum()) <= 1e-12 * np.abs(P.z).sum()
    assert np.abs(h - P.h).max() > 1e-3  # the state did evolve


def test_lake_at_rest_preserved(oracle):
    O = oracle
    P = W.lake_at_rest(200)
    h, q, z, t, steps, _ = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=200)
    assert steps == 200
    assert np.abs(q).max() <= 1e-12
    assert np.abs(h + z - 1.0).max() <= 1e-13


def test_upwind_dependency_supercritical(oracle):
    """Fixed bed with all speeds positive: a cell's new value depends only on
    itself and its left neighbour (cell i takes D+ of edge i-1/2 only)."""
    O = oracle
    n = 16
    rng = np.random.default_rng(5)
    h = rng.uniform(0.5, 0.6, n)
    q = 3.0 * np.sqrt(G * h) * h
    z = np.zeros(n)
    law = O.grass(0.0, xi=1.0, g=G)
    cfg = O.make_cfg(n, 0.0, 1.0, 0.5, law)
    # the CFL maximum is set by cell 3, so perturbing cell 9 leaves dt unchanged
    q[3] *= 1.5
    hp = h.copy()
    hp[9] *= 1.05
    a = O.run(cfg, h, q, z, max_steps=1)
    b = O.run(cfg, hp, q, z, max_steps=1)
    assert a[5] == b[5]  # same dt
    assert np.array_equal(a[0][:9], b[0][:9])
    assert np.array_equal(a[1][:9], b[1][:9])
    assert not np.array_equal(a[0][9:11], b[0][9:11])


def test_dam_break_converges_to_textbook_solution(oracle):
    """A_g = 0 and a flat bed reduce the dSVE system to the shallow-water
    equations; the first-order scheme converges to the exact Riemann solution."""
    O = oracle
    errs = []
    for n in (100, 200, 400, 800):
        P = W.dam_break(n)
        h, q, z, t, steps, _ = O.run(_cfg(O, P), P.h, P.q, P.z, t_end=P.t_end)
        assert t == P.t_end
        x = W.cell_centres(n, 0.0, 10.0)
        he, qe = X.swe_riemann(2.0, 0.0, 1.0, 0.0, x, t, x0=5.0)
        errs.append((np.abs(h - he).sum() / np.abs(he).sum(), np.abs(q - qe).sum() / np.abs(qe).sum()))
        assert np.abs(z).max() <= 1e-14  # the bed only sees rounding
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates > 0.6).all(), (errs, rates)
    assert errs[-1, 0] < 5e-3


def test_berthon_smooth_solution_first_order(oracle):
    """Test 2 (Sec. 4.2, Eq. berthon) with q0 = 2 m^2/s (the paper does not
    print q0) on [0, 7] m to t = 10 s: L1 errors against the exact cell
    averages halve when the grid is refined."""
    O = oracle
    q0 = 2.0
    qb, zb, rate, hR = X.berthon_boundary(q0)
    law = O.grass(0.005, xi=1.0, g=G)
    errs = []
    for n in (70, 140, 280, 560):
        h0, qq0, z0 = X.berthon_cell_average(n, q0, 0.0)
        cfg = O.make_cfg(n, 0.0, 7.0, 0.9, law, O.BC_INFLOW_QZ, O.BC_OUTFLOW_H,
                         (qb, zb, rate), (hR, 0.0, 0.0))
        h, q, z, t, steps, _ = O.run(cfg, h0, qq0, z0, t_end=10.0)
        assert t == 10.0
        he, qe, ze = X.berthon_cell_average(n, q0, 10.0)
        errs.append([np.abs(h - he).sum() / np.abs(he).sum(),
                     np.abs(q - qe).sum() / np.abs(qe).sum(),
                     np.abs(z - ze).sum() / np.abs(ze).sum()])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates > 0.6).all(), (errs, rates)
    assert (rates[-1] > 0.8).all(), (errs, rates)  # first order in the limit
    assert errs[-1].max() < 2e-2, errs


def test_mirror_symmetry_of_a_run(oracle):
    O = oracle
    P = W.movable_bed_riemann(120)
    a = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=60)
    b = O.run(_cfg(O, P), P.h[::-1].copy(), -P.q[::-1].copy(), P.z[::-1].copy(), max_steps=60)
    assert a[4] == b[4] == 60
    sc = np.abs(a[0]).max()
    assert np.abs(a[0] - b[0][::-1]).max() <= 1e-12 * sc
    assert np.abs(a[1] + b[1][::-1]).max() <= 1e-12 * sc
    assert np.abs(a[2] - b[2][::-1]).max() <= 1e-12 * sc


def test_time_step_reading(oracle):
    """dt = CFL dx / max_i max|lambda|(W_i) (spectral radius from LAPACK here);
    the run lands exactly on t_end."""
    O = oracle
    P = W.movable_bed_riemann(200)
    law = O.grass(P.Ag, xi=P.xi, g=G)
    rho = 0.0
    for hi, qi in zip(P.h, P.q):
        rho = max(rho, np.abs(np.linalg.eigvals(O.flux_matrix(law, hi, qi))).max())
    _, _, _, t, steps, dt = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=1)
    assert steps == 1
    assert dt == pytest.approx(P.cfl * P.dx / rho, rel=1e-13)
    _, _, _, t, steps, dt = O.run(_cfg(O, P), P.h, P.q, P.z, t_end=P.t_end)
    assert t == P.t_end and steps > 10 and 0 < dt <= P.cfl * P.dx / rho * 1.5


def test_mass_balance_with_boundary_fluxes(oracle):
    """Transmissive ends (zero jump at the boundary edges) pass the adjacent
    cells' fluxes: while the waves stay inside, sum h dx changes by exactly
    t (q_L - q_R). The bed balance sum z dx - t xi (q_sL - q_sR) is not zero to
    rounding at the initial bed step: row 3 of D- + D+ is a GL3 quadrature of a
    rational function of s. The defect is small and measurable."""
    O = oracle
    P = W.movable_bed_riemann(200)
    qsL, qsR = P.Ag * 0.25 ** 3, P.Ag * 0.2 ** 3
    for k in (1, 20, 100):
        h, q, z, t, steps, _ = O.run(_cfg(O, P), P.h, P.q, P.z, max_steps=k)
        dh = (h.sum() - P.h.sum()) * P.dx - t * (0.5 - 0.2)
        assert abs(dh) <= 1e-13 * P.h.sum() * P.dx
        dz = (z.sum() - P.z.sum()) * P.dx - t * P.xi * (qsL - qsR)
        assert 1e-12 < abs(dz) < 1e-6
