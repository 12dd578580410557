"""Pins of the oracle's Grass law with a threshold velocity (Eq. GrassThr,
q_s = A_g (u - u_cr)^3, read as q_s = A_g sign(u) max(|u| - u_cr, 0)^3: no
transport at or below the incipient velocity, transport along u above it)
against things other than itself: central finite differences, the plain Grass
law it reduces to at u_cr = 0, the fixed-bed textbook eigenvalues below the
threshold, LAPACK above it, and a bed that stays exactly in place when the
flow is everywhere below the threshold."""
import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

G = 9.81


def test_value_and_derivatives_vs_finite_differences(oracle):
    O = oracle
    L = O.grass_thr(0.01, 0.3, xi=1.0, g=G)
    qs, _, _ = O.sediment(L, 2.0, 1.2)  # u = 0.6: q_s = 0.01 (0.6 - 0.3)^3
    assert qs == pytest.approx(0.01 * 0.3 ** 3, rel=1e-14)
    qs, _, _ = O.sediment(L, 2.0, -1.2)
    assert qs == pytest.approx(-0.01 * 0.3 ** 3, rel=1e-14)
    rng = np.random.default_rng(5)
    h = rng.uniform(0.1, 3.0, 300)
    u = rng.choice([-1.0, 1.0], 300) * rng.uniform(0.35, 2.0, 300)  # above the threshold
    for hi, qi in zip(h, u * h):
        _, dh, dq = O.sediment(L, hi, qi)
        eh, eq = 1e-6 * hi, 1e-6 * abs(qi)
        fdh = (O.sediment(L, hi + eh, qi)[0] - O.sediment(L, hi - eh, qi)[0]) / (2 * eh)
        fdq = (O.sediment(L, hi, qi + eq)[0] - O.sediment(L, hi, qi - eq)[0]) / (2 * eq)
        sc = abs(fdh) + abs(fdq)
        assert abs(dh - fdh) <= 1e-7 * sc
        assert abs(dq - fdq) <= 1e-7 * sc


def test_zero_threshold_is_the_grass_law(oracle):
    O = oracle
    thr = O.grass_thr(0.02, 0.0, xi=W.XI_P04, g=G)
    ref = O.grass(0.02, xi=W.XI_P04, g=G)
    h, q = W.random_states(500, 9)
    for hi, qi in zip(h, q):
        assert np.array_equal(O.sediment(thr, hi, qi), O.sediment(ref, hi, qi))
    WL, WR = W.random_edges(400, 10)
    a, b = O.fluct(thr, WL, WR), O.fluct(ref, WL, WR)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_below_threshold_is_a_fixed_bed(oracle):
    O = oracle
    L = O.grass_thr(0.05, 0.8, xi=W.XI_P04, g=G)
    fixed = O.grass(0.0, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(6)
    h = rng.uniform(0.2, 3.0, 200)
    u = rng.uniform(-0.79, 0.79, 200)
    for hi, ui in zip(h, u):
        A = O.flux_matrix(L, hi, ui * hi)
        assert np.array_equal(A, O.flux_matrix(fixed, hi, ui * hi))
        assert not A[2].any()  # no bed row: the bed cannot move
        c = np.sqrt(G * hi)
        assert np.allclose(np.sort(np.linalg.eigvals(A).real), [ui - c, 0.0, ui + c], rtol=0, atol=1e-12 * c)


def test_above_threshold_eigenvalues_match_lapack(oracle):
    O = oracle
    L = O.grass_thr(0.02, 0.2, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(7)
    h = rng.uniform(0.1, 5.0, 1000)
    fr = rng.choice([-1.0, 1.0], 1000) * rng.uniform(0.2, 3.0, 1000)
    for hi, fi in zip(h, fr):
        u = fi * np.sqrt(G * hi)
        if abs(u) < 0.25:
            continue
        lam = O.eigvals_analytic(L, hi, u * hi)
        ref = np.sort(np.linalg.eigvals(O.flux_matrix(L, hi, u * hi)).real)
        assert np.abs(np.sort(lam) - ref).max() <= 1e-10 * (abs(u) + np.sqrt(G * hi))


def test_bed_stays_in_place_below_threshold(oracle):
    """A whole run with the flow everywhere below u_cr equals the run with a
    fixed bed (A_g = 0) bit for bit: a = b = 0 exactly, so the bed row of every
    node's flux matrix is zero. The bed then moves only by the rounding of
    |A|'s bed row formed as R |Lambda| R^-1 (entries (u - l)^2/c^2 - 1 of the
    two shallow-water eigenvectors, zero in exact arithmetic), while h and q
    evolve."""
    O = oracle
    P = W.gaussian_bump(300)  # q = 0.6 on h = 0.2 .. 0.4: |u| <= 3 m/s
    out = []
    for L in (O.grass_thr(0.01, 10.0, xi=P.xi, g=P.g), O.grass(0.0, xi=P.xi, g=P.g)):
        cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, L, P.bc_left, P.bc_right, P.bcl, P.bcr)
        h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=200)
        assert steps == 200
        out.append((h, q, z, t))
    (h, q, z, t), (hf, qf, zf, tf) = out
    assert np.array_equal(h, hf) and np.array_equal(q, qf) and np.array_equal(z, zf) and t == tf
    assert np.abs(z - P.z).max() <= 1e-14 * np.abs(P.z).max()
    assert np.abs(h - P.h).max() > 1e-6
