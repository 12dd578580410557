"""Pins of the oracle's eigenstructure against things other than itself:
numpy/LAPACK eigensolvers, finite differences of the physical flux, matrix
invariants (trace, determinant, principal minors) and the fixed-bed textbook
case. The paper's formulas are Eq. W&A_definition, charPol, lambda,
parameters, parameters_bis, RR, RR-1 and asbA (Sec. 2 and 3.3)."""
import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

G = 9.81


def _law(O, Ag, xi=W.XI_P04):
    return O.grass(Ag, xi=xi, g=G)


def _states(n, seed, fr=(-3.0, 3.0)):
    rng = np.random.default_rng(seed)
    h, q = W.random_states(n, seed, fr_range=fr)
    xiAg = rng.uniform(1e-4, 0.05, size=n)
    return h, q, xiAg


def test_grass_value_and_derivatives_vs_finite_differences(oracle):
    O = oracle
    L = _law(O, 0.01, xi=1.0)
    qs, dh, dq = O.sediment(L, 2.0, 1.0)
    assert qs == pytest.approx(0.01 * 0.5 ** 3, rel=1e-15)  # q_s = A_g u^3, u = 0.5
    h, q = W.random_states(200, 3)
    for hi, qi in zip(h, q):
        _, dh, dq = O.sediment(L, hi, qi)
        eh, eq = 1e-6 * hi, 1e-6 * max(abs(qi), 1e-3)
        fdh = (O.sediment(L, hi + eh, qi)[0] - O.sediment(L, hi - eh, qi)[0]) / (2 * eh)
        fdq = (O.sediment(L, hi, qi + eq)[0] - O.sediment(L, hi, qi - eq)[0]) / (2 * eq)
        sc = abs(fdh) + abs(fdq) + 1e-12
        assert abs(dh - fdh) <= 1e-7 * sc
        assert abs(dq - fdq) <= 1e-7 * sc


def test_mpm_derivatives_vs_finite_differences(oracle):
    O = oracle
    L = O.mpm(2.65, 1e-3, 0.02, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(11)
    h = rng.uniform(0.1, 0.6, 300)
    q = rng.uniform(-1.5, 1.5, 300)
    n_active = 0
    for hi, qi in zip(h, q):
        qs, dh, dq = O.sediment(L, hi, qi)
        # q_s = 8 (theta - 0.047)^1.5 sqrt(g (s-1) d^3), theta = n^2 u^2 / ((s-1) d h^(1/3))
        theta = 0.02 ** 2 * (qi / hi) ** 2 / (1.65 * 1e-3 * hi ** (1 / 3))
        ref = np.sign(qi) * 8 * max(theta - 0.047, 0.0) ** 1.5 * np.sqrt(G * 1.65 * 1e-9)
        assert qs == pytest.approx(ref, rel=1e-12, abs=1e-18)
        if theta < 0.047 * 1.01:
            continue
        n_active += 1
        eh, eq = 1e-6 * hi, 1e-6 * abs(qi)
        fdh = (O.sediment(L, hi + eh, qi)[0] - O.sediment(L, hi - eh, qi)[0]) / (2 * eh)
        fdq = (O.sediment(L, hi, qi + eq)[0] - O.sediment(L, hi, qi - eq)[0]) / (2 * eq)
        sc = abs(fdh) + abs(fdq)
        assert abs(dh - fdh) <= 1e-6 * sc
        assert abs(dq - fdq) <= 1e-6 * sc
    assert n_active > 50


def test_flux_matrix_is_flux_jacobian_plus_bed_term(oracle):
    """A(W) W_x must equal the x-derivative of the conservative flux
    (q, q^2/h + g h^2/2, xi q_s) plus the non-conservative g h z_x (Eq. SV-Ex)."""
    O = oracle
    xi = W.XI_P04
    L = _law(O, 0.02, xi)

    def F(h, q):
        return np.array([q, q * q / h + 0.5 * G * h * h, xi * O.sediment(L, h, q)[0]])

    h, q = W.random_states(100, 5)
    for hi, qi in zip(h, q):
        A = O.flux_matrix(L, hi, qi)
        e = 1e-6
        Jh = (F(hi * (1 + e), qi) - F(hi * (1 - e), qi)) / (2 * e * hi)
        eq = e * max(abs(qi), 1e-3)
        Jq = (F(hi, qi + eq) - F(hi, qi - eq)) / (2 * eq)
        J = np.stack([Jh, Jq, [0.0, G * hi, 0.0]], axis=1)
        assert np.allclose(A, J, rtol=1e-6, atol=1e-9 * np.abs(A).max())


def test_analytic_eigenvalues_match_lapack(oracle):
    O = oracle
    h, q, xiAg = _states(4000, 21)
    worst = 0.0
    for hi, qi, xa in zip(h, q, xiAg):
        L = O.grass(xa, xi=1.0, g=G)
        lam = O.eigvals_analytic(L, hi, qi)
        ref = np.sort(np.linalg.eigvals(O.flux_matrix(L, hi, qi)).real)
        sc = abs(qi / hi) + np.sqrt(G * hi)
        worst = max(worst, np.abs(lam - ref).max() / sc)
    assert worst < 1e-12, worst


def test_qr_eigenvalues_match_lapack(oracle):
    O = oracle
    h, q, xiAg = _states(3000, 22)
    for hi, qi, xa in zip(h, q, xiAg):
        A = O.flux_matrix(O.grass(xa, xi=1.0, g=G), hi, qi)
        lam = O.qr_eigenvalues(A)
        ref = np.sort(np.linalg.eigvals(A).real)
        sc = abs(qi / hi) + np.sqrt(G * hi)
        assert np.abs(lam - ref).max() <= 1e-12 * sc
    # also on general real-spectrum matrices that are not flux matrices
    rng = np.random.default_rng(4)
    for _ in range(300):
        V = rng.standard_normal((3, 3))
        D = np.diag(np.sort(rng.uniform(-5, 5, 3)))
        A = V @ D @ np.linalg.inv(V)
        lam = O.qr_eigenvalues(A)
        assert np.allclose(lam, np.diag(D), atol=1e-9 * np.abs(A).max())


def test_fixed_bed_reduces_to_shallow_water_speeds(oracle):
    """A_g = 0: eigenvalues are exactly u - c, 0, u + c (sorted)."""
    O = oracle
    L = O.grass(0.0, xi=1.0, g=G)
    h, q = W.random_states(500, 8)
    for hi, qi in zip(h, q):
        u, c = qi / hi, np.sqrt(G * hi)
        lam = O.eigvals_analytic(L, hi, qi)
        ref = np.sort([u - c, 0.0, u + c])
        assert np.abs(lam - ref).max() <= 4e-15 * (abs(u) + c) * 10


def test_eigenvalue_invariants(oracle):
    """trace = 2u, product = det A, pair sum = sum of principal 2x2 minors."""
    O = oracle
    h, q, xiAg = _states(2000, 23)
    for hi, qi, xa in zip(h, q, xiAg):
        L = O.grass(xa, xi=1.0, g=G)
        A = O.flux_matrix(L, hi, qi)
        l1, l2, l3 = O.eigvals_analytic(L, hi, qi)
        c2 = G * hi
        sc = abs(qi / hi) + np.sqrt(c2)
        assert abs((l1 + l2 + l3) - 2 * qi / hi) <= 1e-13 * sc
        assert abs(l1 * l2 * l3 - np.linalg.det(A)) <= 1e-12 * sc ** 3
        minors = (A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]) + (A[0, 0] * A[2, 2] - A[0, 2] * A[2, 0]) \
            + (A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1])
        assert abs(l1 * l2 + l2 * l3 + l3 * l1 - minors) <= 1e-12 * sc ** 2


def test_eigenvectors_diagonalise_A(oracle):
    """Eq. RR / RR-1: R^-1 R = I, R L R^-1 = A, A r_i = l_i r_i, l_i A = l_i l_i."""
    O = oracle
    h, q, xiAg = _states(2000, 24)
    for hi, qi, xa in zip(h, q, xiAg):
        L = O.grass(xa, xi=1.0, g=G)
        A = O.flux_matrix(L, hi, qi)
        lam = O.eigvals_analytic(L, hi, qi)
        R, Ri = O.eigvecs_analytic(L, hi, qi, lam)
        cond = np.linalg.cond(R)
        assert np.abs(Ri @ R - np.eye(3)).max() <= 1e-13 * cond
        sA = np.abs(A).max()
        assert np.abs(R @ np.diag(lam) @ Ri - A).max() <= 1e-13 * sA * cond
        for i in range(3):
            assert np.abs(A @ R[:, i] - lam[i] * R[:, i]).max() <= 1e-12 * sA * np.abs(R[:, i]).max()
            assert np.abs(Ri[i] @ A - lam[i] * Ri[i]).max() <= 1e-12 * sA * np.abs(Ri[i]).max()


def test_numeric_eigenstructure_inverts(oracle):
    O = oracle
    h, q, xiAg = _states(1000, 25)
    for hi, qi, xa in zip(h, q, xiAg):
        A = O.flux_matrix(O.grass(xa, xi=1.0, g=G), hi, qi)
        lam, R, Ri = O.eig_numeric(A)
        cond = np.linalg.cond(R)
        assert np.abs(Ri @ R - np.eye(3)).max() <= 1e-13 * cond
        assert np.abs(R @ np.diag(lam) @ Ri - A).max() <= 1e-12 * np.abs(A).max() * cond
    M = np.random.default_rng(2).standard_normal((50, 3, 3))
    for m in M:
        assert np.allclose(O.inverse3(m), np.linalg.inv(m), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_abs_matrix_matches_lapack(oracle, method):
    """|A| = V |L| V^-1 from numpy's eig, for each of the four evaluations."""
    O = oracle
    h, q, xiAg = _states(1500, 26 + method)
    worst = 0.0
    for hi, qi, xa in zip(h, q, xiAg):
        L = O.grass(xa, xi=1.0, g=G)
        A = O.flux_matrix(L, hi, qi)
        w, V = np.linalg.eig(A)
        ref = (V @ np.diag(np.abs(w)) @ np.linalg.inv(V)).real
        got = O.abs_matrix(L, hi, qi, method)
        err = np.abs(got - ref).max() / (np.abs(ref).max() * np.linalg.cond(V))
        worst = max(worst, err)
    assert worst < 1e-12, worst


def test_abs_matrix_squares_to_A_squared(oracle):
    O = oracle
    h, q, xiAg = _states(500, 30)
    for hi, qi, xa in zip(h, q, xiAg):
        L = O.grass(xa, xi=1.0, g=G)
        A = O.flux_matrix(L, hi, qi)
        X = O.abs_matrix(L, hi, qi, 0)
        assert np.abs(X @ X - A @ A).max() <= 1e-11 * np.abs(A @ A).max() * 10


def test_abs_matrix_fixed_bed_supercritical_equals_A(oracle):
    """A_g = 0 and |Fr| > 1: the spectrum is one-signed (plus the zero of the bed
    field), so |A| = sign(u) A."""
    O = oracle
    L = O.grass(0.0, xi=1.0, g=G)
    h, q = W.random_states(300, 31, fr_range=(1.05, 3.0))
    for s in (+1, -1):
        for hi, qi in zip(h, q):
            A = O.flux_matrix(L, hi, s * qi)
            for m in range(4):
                X = O.abs_matrix(L, hi, s * qi, m)
                assert np.abs(X - s * A).max() <= 1e-12 * np.abs(A).max()


def test_newton_form_at_exact_coalescence(oracle):
    """Fixed bed at Fr = 1 has the double eigenvalue 0 and a defective A; the
    Newton form with f[0,0] = 0 gives |A| = A^2 / (2c). Slightly off critical
    it must agree with R|L|R^-1 from LAPACK."""
    O = oracle
    L = O.grass(0.0, xi=1.0, g=G)
    h = 0.7
    c = np.sqrt(G * h)
    A = O.flux_matrix(L, h, c * h)
    for m in range(4):
        X = O.abs_matrix(L, h, c * h, m)
        assert np.allclose(X, A @ A / (2 * c), rtol=0, atol=1e-13 * c)
    for fr in (1 + 1e-3, 1 - 1e-3, 1.2, 0.8):
        A = O.flux_matrix(L, h, fr * c * h)
        w, V = np.linalg.eig(A)
        ref = (V @ np.diag(np.abs(w)) @ np.linalg.inv(V)).real
        assert np.allclose(O.abs_matrix(L, h, fr * c * h, 3), ref, atol=1e-10 * np.abs(ref).max())


def test_nonhyperbolic_state_is_reported(oracle):
    """Eq. parameters needs |k2 / sqrt(4 k1^3)| <= 1. A transport law with
    xi dq_s/dq < -(1 + Fr^2/3) makes k1 < 0; with the Grass law that cannot
    happen, so the check is exercised through a negative A_g."""
    O = oracle
    L = O.grass(-5.0, xi=1.0, g=G)
    with pytest.raises(O.OracleError) as e:
        O.eigvals_analytic(L, 1.0, 2.0)
    assert e.value.status == O.E_NONHYPERBOLIC
