"""Pins of the oracle's DOT fluctuations (Eq. path, Eq. DOTjumpN, Eq. jumps)
against closed forms, a LAPACK-based evaluation, the quadrature order of the
3-point Gauss-Legendre rule, mirror symmetry and one-signed spectra."""
import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

G = 9.81


def _lapack_abs(A):
    w, V = np.linalg.eig(A)
    return (V @ np.diag(np.abs(w)) @ np.linalg.inv(V)).real


def _lapack_fluct(O, law, wl, wr, ngl=3):
    """D-/+ with |A| from numpy's eig at the Gauss-Legendre nodes of [0, 1]."""
    s, w = np.polynomial.legendre.leggauss(ngl)
    s, w = 0.5 * (s + 1.0), 0.5 * w
    dW = wr - wl
    Mm, Mp = np.zeros((3, 3)), np.zeros((3, 3))
    for sk, wk in zip(s, w):
        p = wl + sk * dW
        A = O.flux_matrix(law, p[0], p[1])
        X = _lapack_abs(A)
        Mm += 0.5 * wk * (A - X)
        Mp += 0.5 * wk * (A + X)
    return Mm @ dW, Mp @ dW


def test_gl3_rule_is_gauss_legendre(oracle):
    """Row 2 of D- + D+ with h constant along the path is a GL3 quadrature of
    xi d q_s(Psi(s))/ds, a polynomial of degree 2 in s; a wrong node or weight
    breaks exactness. Checked against the exact value xi (q_s(W+) - q_s(W-))."""
    O = oracle
    law = O.grass(0.013, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(1)
    for _ in range(200):
        h = rng.uniform(0.2, 3.0)
        qL, qR = rng.uniform(-3, 3, 2)
        zL, zR = rng.uniform(-0.5, 0.5, 2)
        dm, dp = O.fluct_edge(law, [h, qL, zL], [h, qR, zR])
        tot = dm + dp
        uL, uR = qL / h, qR / h
        exact = np.array([qR - qL,
                          (uL + uR) * (qR - qL) + G * h * (zR - zL),
                          W.XI_P04 * 0.013 * (uR ** 3 - uL ** 3)])
        sc = np.abs(exact).max() + np.sqrt(G * h) * (abs(qR - qL) + abs(zR - zL))
        assert np.abs(tot - exact).max() <= 1e-13 * sc


def test_compatibility_condition_general_path(oracle):
    """Eq. jumps: D- + D+ = int A(Psi) dPsi/ds ds, whose exact value along the
    segment path is [dq, d(q^2/h + g h^2/2) + g (hL+hR)/2 dz, xi d q_s]. GL3
    reproduces it up to its quadrature error, O(|dW|^7) for small jumps."""
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    WL, WR = W.random_edges(300, 2, rel_jump=1e-3, dz_scale=1e-3)
    for k in range(WL.shape[1]):
        wl, wr = WL[:, k], WR[:, k]
        dm, dp = O.fluct_edge(law, wl, wr)
        hL, qL, zL = wl
        hR, qR, zR = wr
        qsL = O.sediment(law, hL, qL)[0]
        qsR = O.sediment(law, hR, qR)[0]
        exact = np.array([qR - qL,
                          (qR ** 2 / hR + 0.5 * G * hR ** 2) - (qL ** 2 / hL + 0.5 * G * hL ** 2)
                          + G * 0.5 * (hL + hR) * (zR - zL),
                          W.XI_P04 * (qsR - qsL)])
        sc = np.abs(dm).max() + np.abs(dp).max()
        assert np.abs(dm + dp - exact).max() <= 1e-11 * sc


def test_gl3_convergence_order(oracle):
    """D+-(GL3) - D+-(exact integral) shrinks like |dW|^7: halving the jump
    divides the error by ~128 (a 2-point or misplaced rule gives at most 2^5)."""
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    wl = np.array([1.3, 0.9, 0.1])
    d = np.array([0.35, 0.5, -0.2])
    errs = []
    for eps in (0.4, 0.2, 0.1):
        wr = wl + eps * d
        dm, dp = O.fluct_edge(law, wl, wr)
        rm, rp = _lapack_fluct(O, law, wl, wr, ngl=40)
        errs.append(max(np.abs(dm - rm).max(), np.abs(dp - rp).max()))
    assert errs[0] / errs[1] > 64 and errs[1] / errs[2] > 64, errs


def test_matches_lapack_fluctuations(oracle):
    O = oracle
    WL, WR = W.random_edges(500, 3)
    rng = np.random.default_rng(3)
    for k in range(WL.shape[1]):
        law = O.grass(rng.uniform(1e-3, 0.03), xi=W.XI_P04, g=G)
        wl, wr = WL[:, k], WR[:, k]
        dm, dp = O.fluct_edge(law, wl, wr)
        rm, rp = _lapack_fluct(O, law, wl, wr)
        sc = np.abs(rm).max() + np.abs(rp).max()
        assert np.abs(dm - rm).max() <= 1e-10 * sc
        assert np.abs(dp - rp).max() <= 1e-10 * sc


@pytest.mark.parametrize("method", [1, 2, 3])
def test_methods_agree_with_analytic(oracle, method):
    """A-DOT (analytic) and the numerical-eigenstructure DOT give the same
    fluctuations (the paper's claim that A-DOT reproduces DOT, Sec. 4.3)."""
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    WL, WR = W.random_edges(2000, 4 + method)
    am, ap = O.fluct(law, WL, WR, 0)
    bm, bp = O.fluct(law, WL, WR, method)
    sc = np.abs(am).max(axis=0) + np.abs(ap).max(axis=0)
    assert (np.abs(am - bm).max(axis=0) <= 1e-11 * sc).all()
    assert (np.abs(ap - bp).max(axis=0) <= 1e-11 * sc).all()


def test_zero_jump_gives_zero(oracle):
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    WL, _ = W.random_edges(100, 9)
    dm, dp = O.fluct(law, WL, WL.copy())
    assert (dm == 0).all() and (dp == 0).all()


def test_mirror_symmetry(oracle):
    """x -> -x maps (h, q, z) to (h, -q, z) and swaps the sides of an edge:
    D-(P W+, P W-) = P D+(W-, W+) and D+(P W+, P W-) = P D-(W-, W+)."""
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    WL, WR = W.random_edges(1000, 10)
    P = np.array([1.0, -1.0, 1.0])[:, None]
    dm, dp = O.fluct(law, WL, WR)
    mm, mp = O.fluct(law, P * WR, P * WL)
    sc = np.abs(dm).max(axis=0) + np.abs(dp).max(axis=0)
    assert (np.abs(mm - P * dp).max(axis=0) <= 1e-12 * sc).all()
    assert (np.abs(mp - P * dm).max(axis=0) <= 1e-12 * sc).all()


def test_one_signed_spectrum_is_pure_upwind(oracle):
    """Fixed bed, supercritical along the whole path: every eigenvalue is >= 0
    (u > 0) or <= 0 (u < 0), so all of sum_k w_k A_k dW goes to one side."""
    O = oracle
    law = O.grass(0.0, xi=1.0, g=G)
    WL, WR = W.random_edges(500, 11, fr_range=(1.6, 3.0), rel_jump=0.1)
    for sign in (1.0, -1.0):
        S = np.array([1.0, sign, 1.0])[:, None]
        dm, dp = O.fluct(law, S * WL, S * WR)
        tot = dm + dp
        sc = np.abs(tot).max(axis=0)
        small, big = (dm, dp) if sign > 0 else (dp, dm)
        assert (np.abs(small).max(axis=0) <= 1e-13 * sc).all()
        assert (np.abs(big - tot).max(axis=0) <= 1e-13 * sc).all()


def test_lake_at_rest_edges(oracle):
    """u = 0 and h + z constant: A dW = 0 and every l_i . dW carries a factor
    that vanishes (Eq. RR-1 with lambda = -c, 0, c), so D+- = 0 up to rounding."""
    O = oracle
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(12)
    for _ in range(500):
        zL, zR = rng.uniform(0, 0.5, 2)
        dm, dp = O.fluct_edge(law, [1.0 - zL, 0.0, zL], [1.0 - zR, 0.0, zR])
        bound = 1e-14 * np.sqrt(G) * abs(zR - zL) * 10
        assert np.abs(dm).max() <= bound and np.abs(dp).max() <= bound
