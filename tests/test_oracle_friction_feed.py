"""Pins of the oracle's friction source (Eq. scheme with S = (0, -g h s_f, 0),
Strickler s_f = q|q| / (K_s^2 h^(10/3)), Sec. 2), of its sediment feed through
an end (Sec. 5.1, the Soni case) and of the power law of the velocity
(Eq. Soni_qs), against things other than the oracle itself:

* the paper's printed Soni data, which must be a uniform flow at normal depth
  (textbook Manning-Strickler relation q = K_s h^(5/3) s0^(1/2));
* the closed-form solution of the friction ODE dq/dt = -g q|q| / (K_s^2 h^(7/3))
  on a uniform periodic flow, and forward Euler's first-order convergence to it;
* exact stillness of a uniform flow at the textbook normal slope;
* the bed-volume budget: the bed gains exactly what the feed brings minus what
  leaves, step by step;
* mirror symmetry of a feed from the right with the flow towards -x;
* finite differences, the Grass law it reduces to, and LAPACK eigenvalues for
  the power law.
"""
import numpy as np
import pytest

from paper_1912_04791_gb300 import workloads as W

G = 9.81
KS, H0, Q0 = 49.4, 0.05, 0.02  # Soni case (Eq. Soni0, Sec. 5.1)


def normal_slope(q, h, ks):
    """Manning-Strickler uniform flow q = K_s h^(5/3) s^(1/2), solved for s."""
    return (q / (ks * h ** (5.0 / 3.0))) ** 2


def test_printed_soni_state_is_normal_flow():
    """The paper's h0 = 0.05 m, q0 = 0.02 m^2/s, K_s = 49.4 and s0 = 3.56 per
    mille: the textbook normal slope of that flow rounds to the printed s0, so
    the friction closure q^2 / (K_s^2 h^(10/3)) is the one of the initial
    equilibrium (a different exponent or a missing square would not be)."""
    s = normal_slope(Q0, H0, KS)
    assert round(s * 1e3, 2) == 3.56
    assert abs(s - 3.56e-3) < 0.005 * 3.56e-3


@pytest.mark.parametrize("bc_left,bc_right", [("QS", "HS"), ("Q", "HS")])
def test_uniform_flow_at_normal_slope_stays(oracle, bc_left, bc_right):
    """A fixed bed (no transport) at the textbook normal slope: friction balances
    the path-conservative bed-slope term cell by cell, and the extrapolated
    ghost beds continue the slope at both ends, so nothing moves."""
    O = oracle
    s = normal_slope(Q0, H0, KS)
    P = W.soni_aggradation(n=100, s0=s)
    L = O.power(0.0, 5.0, xi=P.xi, g=G)
    kinds = {"QS": O.BC_INFLOW_QS, "Q": O.BC_INFLOW_Q, "HS": O.BC_OUTFLOW_HS}
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, L, kinds[bc_left], kinds[bc_right],
                     (Q0, 0.0, 0.0), (H0, 0.0, 0.0), ks=KS)
    h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=500)
    assert steps == 500
    assert np.array_equal(z, P.z)
    if bc_left == "QS":
        assert np.abs(h - H0).max() <= 1e-14 and np.abs(q - Q0).max() <= 1e-15
    else:
        # INFLOW_Q copies the bed: the first edge sees no slope, so the first
        # cell is pushed off balance (only the extrapolating kind is balanced)
        assert np.abs(q - Q0).max() > 1e-8


def test_first_step_off_normal_slope(oracle):
    """On 1.2 x the normal slope an inner cell accelerates in the first step by
    exactly dt g h (s0 - s_n): the bed-slope term g h s0 minus the friction at
    the normal state."""
    O = oracle
    sn = normal_slope(Q0, H0, KS)
    s0 = 1.2 * sn
    P = W.soni_aggradation(n=50, s0=s0)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.power(0.0, 5.0, xi=P.xi, g=G),
                     O.BC_INFLOW_QS, O.BC_OUTFLOW_HS, (Q0, 0.0, 0.0), (H0, 0.0, 0.0), ks=KS)
    h, q, z, t, steps, dt = O.run(cfg, P.h, P.q, P.z, max_steps=1)
    dz = P.z[0] - P.z[1]  # the discrete slope times dx
    want = dt * G * H0 * (dz / P.dx - sn)
    assert want > 0
    np.testing.assert_allclose(q[1:-1] - Q0, want, rtol=1e-9)
    assert np.abs(h - H0).max() <= 1e-15


def _decay(O, q0, h, cfl, ks, t_end):
    n = 8
    L = O.grass(0.0, xi=1.0, g=G)
    cfg = O.make_cfg(n, 0.0, 1.0, cfl, L, O.BC_PERIODIC, O.BC_PERIODIC, ks=ks)
    hh, qq, zz, t, steps, _ = O.run(cfg, np.full(n, h), np.full(n, q0), np.zeros(n), t_end=t_end)
    return hh, qq, zz, t, steps


def test_friction_decay_matches_ode(oracle):
    """Uniform periodic flow on a flat bed: every jump is zero, so the scheme is
    forward Euler on dq/dt = -k q|q|, k = g / (K_s^2 h^(7/3)), whose solution is
    q0 / (1 + k q0 t). Euler's global error is first order in dt: bounded by
    dt t max|q''| / 2 with q'' = 2 k^2 q^3, and halving the CFL number halves it."""
    O = oracle
    h, q0, ks, T = 0.3, 0.5, 20.0, 5.0
    k = G / (ks ** 2 * h ** (7.0 / 3.0))
    exact = q0 / (1.0 + k * q0 * T)
    errs = []
    for cfl in (0.8, 0.4):
        hh, qq, zz, t, steps = _decay(O, q0, h, cfl, ks, T)
        assert t == T and np.array_equal(hh, np.full(8, h)) and not zz.any()
        assert np.ptp(qq) == 0.0
        dt = cfl * (1.0 / 8) / np.sqrt(G * h)  # above every step's cfl dx / (|u| + c)
        err = exact - qq[0]
        # the solution is convex, so each Euler step lands below it; the decay
        # is contractive, so the global error is at most the sum of the local
        # errors, t dt max|q''| / 2
        assert 0.0 < err <= dt * T * k * k * q0 ** 3
        errs.append(err)
    assert 1.8 < errs[0] / errs[1] < 2.2
    # friction opposes the flow in both directions: q -> -q mirrors the decay
    _, qn, _, _, _ = _decay(O, -q0, h, 0.8, ks, T)
    _, qp, _, _, _ = _decay(O, q0, h, 0.8, ks, T)
    assert np.array_equal(qn, -qp)


def _flat_feed(O, n, qs_in, steps, h=0.4, q=0.2):
    L = O.grass(0.01, xi=W.XI_P04, g=G)
    cfg = O.make_cfg(n, 0.0, 10.0, 0.9, L, O.BC_INFLOW_QS, O.BC_TRANSMISSIVE, (q, qs_in, 0.0))
    return L, O.run(cfg, np.full(n, h), np.full(n, q), np.zeros(n), max_steps=steps)


def test_feed_equilibrium_and_first_step(oracle):
    """Uniform flow (u = 0.5 m/s) on a flat bed: fed its own discharge
    A_g u^3 it stays exactly; fed d more, the first step changes only the
    first cell's bed, by dt/dx xi d (the edge discharge is the imposed one)."""
    O = oracle
    qs = 0.01 * 0.5 ** 3
    L, (h, q, z, t, steps, dt) = _flat_feed(O, 64, qs, 200)
    assert np.abs(z).max() <= 1e-17 and np.abs(h - 0.4).max() <= 1e-16
    d = 0.37 * qs
    L, (h, q, z, t, steps, dt) = _flat_feed(O, 64, qs + d, 1)
    assert np.array_equal(h, np.full(64, 0.4)) and np.array_equal(q, np.full(64, 0.2))
    assert not z[1:].any()
    assert z[0] == pytest.approx(dt / (10.0 / 64) * W.XI_P04 * d, rel=1e-12)


def test_feed_bed_volume_budget(oracle):
    """Over 1500 steps of aggradation the bed volume grows each step by
    dt xi (q_s,in - q_s(W_last)): the feed minus what leaves through the
    transmissive end (zero jump there, so the edge discharge is xi q_s of the
    last cell). The inner edges telescope up to the three-node Gauss rule's
    error on the rational q_s along each segment (5e-8 of a step's budget
    measured here); a lost, doubled or mis-signed feed term is an O(1) error."""
    O = oracle
    n, dx = 200, 10.0 / 200
    L = O.grass(0.01, xi=W.XI_P04, g=G)
    qin = 3 * 0.01 * 0.5 ** 3
    cfg = O.make_cfg(n, 0.0, 10.0, 0.9, L, O.BC_INFLOW_QS, O.BC_TRANSMISSIVE, (0.2, qin, 0.0))
    h, q, z = np.full(n, 0.4), np.full(n, 0.2), np.zeros(n)
    t, pred, worst = 0.0, 0.0, 0.0
    for _ in range(1500):
        qs_last = O.sediment(L, h[-1], q[-1])[0]
        v0 = z.sum() * dx
        h, q, z, t, _, dt = O.run(cfg, h, q, z, max_steps=1, t0=t)
        dp = dt * W.XI_P04 * (qin - qs_last)
        worst = max(worst, abs(z.sum() * dx - v0 - dp) / dp)
        pred += dp
    assert worst <= 1e-6
    assert abs(z.sum() * dx - pred) <= 1e-6 * pred
    assert z[0] > z[n // 4] > 0.0  # the deposit is thickest at the feed


def test_feed_from_the_right_mirrors(oracle):
    """x -> -x, q -> -q: a feed at the right end with the flow towards -x
    (signed discharge -q_s,in) is the mirror image of the left-fed run."""
    O = oracle
    n, steps = 120, 300
    L = O.grass(0.01, xi=W.XI_P04, g=G)
    qin = 2.5 * 0.01 * 0.5 ** 3
    x = W.cell_centres(n, 0.0, 10.0)
    z0 = 0.02 * np.sin(x)
    a = O.run(O.make_cfg(n, 0.0, 10.0, 0.9, L, O.BC_INFLOW_QS, O.BC_OUTFLOW_HS,
                         (0.2, qin, 0.0), (0.4, 0.0, 0.0), ks=25.0),
              np.full(n, 0.4), np.full(n, 0.2), z0, max_steps=steps)
    b = O.run(O.make_cfg(n, 0.0, 10.0, 0.9, L, O.BC_OUTFLOW_HS, O.BC_INFLOW_QS,
                         (0.4, 0.0, 0.0), (-0.2, -qin, 0.0), ks=25.0),
              np.full(n, 0.4), np.full(n, -0.2), z0[::-1].copy(), max_steps=steps)
    assert a[4] == b[4] == steps and b[3] == pytest.approx(a[3], rel=1e-13)
    for k, sign in ((0, 1), (1, -1), (2, 1)):
        ref = a[k]
        assert np.abs(sign * b[k][::-1] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(a[2] - z0).max() > 1e-4


def test_soni_volume_tends_to_the_fed_volume(oracle):
    """The Soni case (Sec. 5.1) with its printed data: the bed deposits the
    excess feed xi Delta Q_S t_end / B in the limit (the mass balance the paper
    invokes); at 100 and 400 cells the shortfall is the first-order numerical
    bed flux leaving through the outlet and shrinks with the cell size. The
    deposit is thickest at the feed and decays downstream."""
    O = oracle
    V_fed = None
    gaps = []
    for n in (100, 400):
        P = W.soni_aggradation(n=n)
        L = O.power(P.Ag, P.extra["beta"], xi=P.xi, g=P.g)
        cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, L, P.bc_left, P.bc_right, P.bcl, P.bcr,
                         ks=P.extra["ks"])
        h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, t_end=P.t_end)
        assert t == P.t_end
        dz = z - P.z
        V_fed = P.xi * (P.bcl[1] - P.extra["qs0"]) * P.t_end
        gaps.append((V_fed - dz.sum() * P.dx) / V_fed)
        m = int(0.4 * n)
        assert np.all(np.diff(dz[:m]) < 0)  # decays from the feed over the front
        assert dz[0] > 0.03
    assert 0.0 < gaps[1] < gaps[0] < 0.1
    assert gaps[1] < 0.03


def test_power_law_derivatives_and_reductions(oracle):
    O = oracle
    L = O.power(1.45e-3, 5.0, xi=1.0, g=G)
    qs, _, _ = O.sediment(L, 0.05, 0.02)  # u = 0.4: alpha u^5
    assert qs == pytest.approx(1.45e-3 * 0.4 ** 5, rel=1e-14)
    assert O.sediment(L, 0.05, -0.02)[0] == -qs
    rng = np.random.default_rng(11)
    for beta, ucr in ((5.0, 0.0), (2.5, 0.1), (1.0, 0.0)):
        L = O.power(2e-3, beta, u_cr=ucr, xi=1.0, g=G)
        for hi, ui in zip(rng.uniform(0.05, 2.0, 200), rng.choice([-1, 1], 200) * rng.uniform(0.2, 2.0, 200)):
            qi = ui * hi
            _, dh, dq = O.sediment(L, hi, qi)
            eh, eq = 1e-6 * hi, 1e-6 * abs(qi)
            fdh = (O.sediment(L, hi + eh, qi)[0] - O.sediment(L, hi - eh, qi)[0]) / (2 * eh)
            fdq = (O.sediment(L, hi, qi + eq)[0] - O.sediment(L, hi, qi - eq)[0]) / (2 * eq)
            sc = abs(fdh) + abs(fdq)
            assert abs(dh - fdh) <= 1e-7 * sc and abs(dq - fdq) <= 1e-7 * sc
    # beta = 3 is the thresholded Grass law; beta = 3, u_cr = 0 the Grass law
    h, q = W.random_states(300, 12)
    for A, ucr in ((0.02, 0.3), (0.02, 0.0)):
        P3, T3 = O.power(A, 3.0, u_cr=ucr, xi=W.XI_P04), O.grass_thr(A, ucr, xi=W.XI_P04)
        for hi, qi in zip(h, q):
            np.testing.assert_allclose(O.sediment(P3, hi, qi), O.sediment(T3, hi, qi), rtol=1e-14, atol=0)


def test_power_law_eigenvalues_match_lapack(oracle):
    O = oracle
    L = O.power(1.45e-3, 5.0, xi=W.XI_P04, g=G)
    rng = np.random.default_rng(13)
    for hi, fi in zip(rng.uniform(0.02, 1.0, 600), rng.choice([-1, 1], 600) * rng.uniform(0.05, 2.5, 600)):
        u = fi * np.sqrt(G * hi)
        lam = O.eigvals_analytic(L, hi, u * hi)
        ref = np.sort(np.linalg.eigvals(O.flux_matrix(L, hi, u * hi)).real)
        assert np.abs(np.sort(lam) - ref).max() <= 1e-10 * (abs(u) + np.sqrt(G * hi))
