"""Closed-form and exact solutions used to pin the oracle (test infrastructure).

* ``swe_riemann``: exact solution of the fixed-bed shallow-water Riemann problem
  (the A_g = 0, flat-bed special case of the dSVE system, Eq. SV-Ex with q_s = 0
  and z constant). Standard textbook construction: two nonlinear waves, each a
  shock (Rankine-Hugoniot) or a rarefaction (Riemann invariants); the star depth
  solves f_L(h*) + f_R(h*) + u_R - u_L = 0 (Newton), no dry bed.
* ``MovableBedRiemann``: exact self-similar solution of the movable-bed Riemann
  problem with the Grass law, built from the PDE (Eq. SV-Ex): rarefactions
  along integral curves of the eigenvectors (LAPACK), shocks from the
  generalised Rankine-Hugoniot conditions of the segment path (Eq. path) with
  the Lax entropy condition. The paper cites this solution but does not give it.
* ``berthon``: the smooth steady-flow-plus-linear-erosion solution of Test 2
  (Sec. 4.2, Eq. berthon and the initial/boundary data that follow it). The
  paper's form has z_t = -alpha, which solves Eq. SV-Ex3 with xi = 1; for
  general xi the erosion rate is xi*alpha (q_s = alpha x + beta along the flow).
"""
from __future__ import annotations

import numpy as np


def _f_wave(hs, hk, g):
    """Velocity change across one wave as a function of the star depth, and its
    derivative: shock branch (hs > hk) from the Rankine-Hugoniot conditions of
    the mass and momentum equations, rarefaction branch from the Riemann
    invariant u +- 2c."""
    if hs > hk:
        s = np.sqrt(0.5 * g * (hs + hk) / (hs * hk))
        f = (hs - hk) * s
        ds = 0.5 * 0.5 * g * (-hk) / (hs * hs * hk) / s  # d s / d hs
        df = s + (hs - hk) * ds
        return f, df
    cs, ck = np.sqrt(g * hs), np.sqrt(g * hk)
    return 2.0 * (cs - ck), g / cs


def swe_star(hL, uL, hR, uR, g=9.81, tol=1e-15):
    """Star-region depth and velocity of the shallow-water Riemann problem."""
    cL, cR = np.sqrt(g * hL), np.sqrt(g * hR)
    if 2.0 * (cL + cR) <= uR - uL:
        raise ValueError("dry bed generated; not supported")
    hs = ((0.5 * (cL + cR) - 0.25 * (uR - uL)) ** 2) / g  # two-rarefaction guess
    for _ in range(200):
        fL, dL = _f_wave(hs, hL, g)
        fR, dR = _f_wave(hs, hR, g)
        F = fL + fR + uR - uL
        step = F / (dL + dR)
        hn = hs - step
        if hn <= 0:
            hn = 0.5 * hs
        if abs(hn - hs) <= tol * hs:
            hs = hn
            break
        hs = hn
    fL, _ = _f_wave(hs, hL, g)
    fR, _ = _f_wave(hs, hR, g)
    us = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return hs, us


def swe_riemann(hL, uL, hR, uR, x, t, x0=0.0, g=9.81):
    """Exact (h, q) at positions x and time t > 0 for a discontinuity at x0."""
    hs, us = swe_star(hL, uL, hR, uR, g)
    cL, cR, cs = np.sqrt(g * hL), np.sqrt(g * hR), np.sqrt(g * hs)
    xs = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.empty_like(xs)
    u = np.empty_like(xs)
    for idx, S in np.ndenumerate(xs):
        if S <= us:  # left of the contact: left wave
            if hs > hL:  # left shock
                sL = uL - cL * np.sqrt(0.5 * hs * (hs + hL)) / hL
                h[idx], u[idx] = (hL, uL) if S <= sL else (hs, us)
            else:  # left rarefaction
                head, tail = uL - cL, us - cs
                if S <= head:
                    h[idx], u[idx] = hL, uL
                elif S >= tail:
                    h[idx], u[idx] = hs, us
                else:
                    c = (uL + 2.0 * cL - S) / 3.0
                    h[idx], u[idx] = c * c / g, S + c
        else:
            if hs > hR:  # right shock
                sR = uR + cR * np.sqrt(0.5 * hs * (hs + hR)) / hR
                h[idx], u[idx] = (hR, uR) if S >= sR else (hs, us)
            else:
                head, tail = uR + cR, us + cs
                if S >= head:
                    h[idx], u[idx] = hR, uR
                elif S <= tail:
                    h[idx], u[idx] = hs, us
                else:
                    c = (-uR + 2.0 * cR + S) / 3.0
                    h[idx], u[idx] = c * c / g, S - c
    return h, h * u


# ---------------------------------------------------------------------------
# Test 2 (Berthon): smooth steady flow with linear-in-time bed erosion.
# ---------------------------------------------------------------------------

BERTHON = dict(alpha=0.005, beta=0.005, Ag=0.005, C=1.0, L=7.0, t_end=10.0)


def berthon(x, t, q0, alpha=0.005, beta=0.005, Ag=0.005, C=1.0, g=9.81, xi=1.0):
    """(h, q, z) of Eq. berthon at positions x and time t.

    u(x) = ((alpha x + beta)/A_g)^(1/3), h = q0/u, z(x,0) = C - (u^3 + 2 g q0)/(2 g u),
    z(x,t) = z(x,0) - xi*alpha*t (the paper prints -alpha t, its xi = 1 case).
    """
    x = np.asarray(x, dtype=np.float64)
    u = np.cbrt((alpha * x + beta) / Ag)
    h = q0 / u
    z0 = C - (u ** 3 + 2.0 * g * q0) / (2.0 * g * u)
    return h, np.full_like(x, q0), z0 - xi * alpha * t


def berthon_cell_average(n, q0, t, L=7.0, ngl=8, **kw):
    """Cell averages of the Berthon solution on n uniform cells of [0, L]
    (Gauss-Legendre with ngl points per cell)."""
    s, w = np.polynomial.legendre.leggauss(ngl)
    dx = L / n
    xc = (np.arange(n) + 0.5) * dx
    acc = [np.zeros(n), np.zeros(n), np.zeros(n)]
    for sk, wk in zip(s, w):
        vals = berthon(xc + 0.5 * dx * sk, t, q0, **kw)
        for a, v in zip(acc, vals):
            a += 0.5 * wk * v
    return tuple(acc)


def berthon_boundary(q0, L=7.0, alpha=0.005, beta=0.005, Ag=0.005, C=1.0, g=9.81, xi=1.0):
    """Boundary data of Test 2: inflow q(0,t) = q0 with z(0,t) = z0(0) - xi alpha t,
    and outflow depth h(L) fixed. Returns (q0, z0_left, erosion_rate, h_right)."""
    h0, _, z0 = berthon(np.array([0.0]), 0.0, q0, alpha, beta, Ag, C, g, xi)
    hL, _, _ = berthon(np.array([L]), 0.0, q0, alpha, beta, Ag, C, g, xi)
    return q0, float(z0[0]), xi * alpha, float(hL[0])


# ---------------------------------------------------------------------------
# Exact solution of the movable-bed Riemann problem (segment path).
# ---------------------------------------------------------------------------
# The solution of W_t + A(W) W_x = 0 (Eq. quasiLinNC with S = 0) for piecewise
# constant data is self-similar: three waves, one per characteristic family,
# separate constant states W_L, W1, W2, W_R. A wave of family i is either a
# rarefaction, along the integral curve dW/dh = r_i(W) (the eigenvector with
# unit h-entry, from LAPACK here) across which lambda_i increases left to right,
# or a shock moving at sigma with the generalised Rankine-Hugoniot conditions
# of the segment path (Eq. path), which hold exactly for this system:
#     sigma dh = dq,
#     sigma dq = d(q^2/h + g h^2/2) + g (h_l + h_r)/2 dz,
#     sigma dz = xi d(q_s),
# and the Lax condition lambda_i(W_r) < sigma < lambda_i(W_l). Which branch a
# given change of h takes follows from the sign of d(lambda_i)/dh along r_i.

def _flux_matrix(h, q, g, xi, Ag):
    u = q / h
    c2 = g * h
    return np.array([[0.0, 1.0, 0.0],
                     [c2 - u * u, 2.0 * u, c2],
                     [-3.0 * xi * Ag * u ** 3 / h, 3.0 * xi * Ag * u * u / h, 0.0]])


def _eig(h, q, g, xi, Ag):
    w, V = np.linalg.eig(_flux_matrix(h, q, g, xi, Ag))
    o = np.argsort(w.real)
    w, V = w.real[o], V.real[:, o]
    return w, V / V[0]  # unit h-entry


def _lam(W, i, g, xi, Ag):
    return _eig(W[0], W[1], g, xi, Ag)[0][i]


def _grad_lam_dot_r(W, i, g, xi, Ag):
    """d lambda_i / dh along the integral curve of r_i (central difference)."""
    _, V = _eig(W[0], W[1], g, xi, Ag)
    r = V[:, i]
    e = 1e-6 * W[0]
    return (_lam(W + e * r, i, g, xi, Ag) - _lam(W - e * r, i, g, xi, Ag)) / (2 * e)


def _integral_curve(W0, i, h1, g, xi, Ag, rtol=1e-12):
    from scipy.integrate import solve_ivp
    if h1 == W0[0]:
        return np.array(W0, dtype=float)

    def rhs(h, y):
        W = np.array([h, y[0], y[1]])
        r = _eig(W[0], W[1], g, xi, Ag)[1][:, i]
        # continue the eigenvector with a consistent sign (unit h-entry makes it unique)
        return [r[1], r[2]]

    sol = solve_ivp(rhs, (W0[0], h1), [W0[1], W0[2]], method="DOP853", rtol=rtol, atol=1e-14)
    return np.array([h1, sol.y[0, -1], sol.y[1, -1]])


def _rh_residual(Wl, Wr, sigma, g, xi, Ag):
    hl, ql, zl = Wl
    hr, qr, zr = Wr
    F = lambda h, q: q * q / h + 0.5 * g * h * h  # noqa: E731
    qs = lambda h, q: Ag * (q / h) ** 3  # noqa: E731
    return np.array([sigma * (hr - hl) - (qr - ql),
                     sigma * (qr - ql) - (F(hr, qr) - F(hl, ql)) - g * 0.5 * (hl + hr) * (zr - zl),
                     sigma * (zr - zl) - xi * (qs(hr, qr) - qs(hl, ql))])


def _shock(W0, i, h1, g, xi, Ag, left_known=True):
    """State across a family-i shock with depth h1 on the other side, and its speed."""
    from scipy.optimize import fsolve
    lam, V = _eig(W0[0], W0[1], g, xi, Ag)
    guess_W = W0 + (h1 - W0[0]) * V[:, i]
    x0 = [guess_W[1], guess_W[2], lam[i]]

    def F(x):
        W1 = np.array([h1, x[0], x[1]])
        Wl, Wr = (W0, W1) if left_known else (W1, W0)
        return _rh_residual(Wl, Wr, x[2], g, xi, Ag)

    x, info, ier, msg = fsolve(F, x0, xtol=1e-14, full_output=True)
    return np.array([h1, x[0], x[1]]), x[2]


class MovableBedRiemann:
    """Exact solution for left/right states WL, WR = (h, q, z) of the dSVE system
    with the Grass law q_s = A_g u^3 (Eq. SV-Ex, Eq. Grass), frictionless."""

    def __init__(self, WL, WR, Ag, xi=1.0, g=9.81):
        from scipy.optimize import fsolve
        self.WL, self.WR = np.array(WL, float), np.array(WR, float)
        self.Ag, self.xi, self.g = Ag, xi, g

        def waves(p):
            W = self.WL
            out = []
            for i, h1 in ((0, p[0]), (1, p[1])):
                out.append(self._wave(W, i, h1))
                W = out[-1][0]
            out.append(self._wave(W, 2, self.WR[0]))
            return out

        def resid(p):
            W3 = waves(p)[-1][0]
            return [(W3[1] - self.WR[1]) / (abs(self.WR[1]) + 1.0),
                    (W3[2] - self.WR[2]) / (abs(self.WR[2]) + 1.0)]

        # initial guess: SWE star depth on the water surface jump
        hs, _ = swe_star(self.WL[0], self.WL[1] / self.WL[0], self.WR[0] + self.WR[2] - self.WL[2],
                         self.WR[1] / self.WR[0], g)
        p0 = [hs, max(hs - (self.WR[2] - self.WL[2]), 0.05)]
        p, info, ier, msg = fsolve(resid, p0, xtol=1e-13, full_output=True)
        self.converged = ier == 1 and np.abs(resid(p)).max() < 1e-10
        self.params = p
        self.waves = waves(p)
        self.states = [self.WL] + [w[0] for w in self.waves]

    def _wave(self, W0, i, h1):
        """(W1, kind, speeds) for family i from W0 (left) to depth h1 (right)."""
        G = _grad_lam_dot_r(W0, i, self.g, self.xi, self.Ag)
        rare = (h1 - W0[0]) * G > 0
        if rare or abs(G) < 1e-12:
            W1 = _integral_curve(W0, i, h1, self.g, self.xi, self.Ag)
            return W1, "rarefaction", (_lam(W0, i, self.g, self.xi, self.Ag),
                                       _lam(W1, i, self.g, self.xi, self.Ag))
        W1, sigma = _shock(W0, i, h1, self.g, self.xi, self.Ag)
        return W1, "shock", (sigma, sigma)

    def rh_residuals(self):
        """Rankine-Hugoniot residuals of the shocks (scaled), for checking."""
        out = []
        W = self.WL
        for W1, kind, (s0, s1) in self.waves:
            if kind == "shock":
                out.append(np.abs(_rh_residual(W, W1, s0, self.g, self.xi, self.Ag)).max())
            W = W1
        return out

    def lax_ok(self):
        W = self.WL
        for i, (W1, kind, (s0, s1)) in enumerate(self.waves):
            if kind == "shock":
                if not (_lam(W1, i, self.g, self.xi, self.Ag) < s0 < _lam(W, i, self.g, self.xi, self.Ag)):
                    return False
            W = W1
        return True

    def sample(self, x, t, x0=0.0):
        """(h, q, z) at positions x and time t > 0."""
        xs = (np.asarray(x, float) - x0) / t
        out = np.empty((3,) + xs.shape)
        for idx, S in np.ndenumerate(xs):
            W = self.WL
            val = None
            for i, (W1, kind, (s0, s1)) in enumerate(self.waves):
                if S < s0:
                    val = W
                    break
                if kind == "rarefaction" and S < s1:
                    val = self._fan_state(W, i, S)
                    break
                W = W1
            if val is None:
                val = self.WR
            out[(slice(None),) + idx] = val
        return out[0], out[1], out[2]

    def _fan_state(self, W0, i, S):
        """State inside the family-i rarefaction where lambda_i = S (one dense
        integration of the integral curve per wave, then a root solve on it)."""
        from scipy.integrate import solve_ivp
        from scipy.optimize import brentq
        if not hasattr(self, "_dense"):
            self._dense = {}
        h1 = self.waves[i][0][0]
        if i not in self._dense:
            def rhs(h, y):
                r = _eig(h, y[0], self.g, self.xi, self.Ag)[1][:, i]
                return [r[1], r[2]]
            self._dense[i] = solve_ivp(rhs, (W0[0], h1), [W0[1], W0[2]], method="DOP853",
                                       rtol=1e-12, atol=1e-14, dense_output=True).sol
        sol = self._dense[i]
        W = lambda h: np.array([h, *sol(h)])  # noqa: E731
        h = brentq(lambda hh: _lam(W(hh), i, self.g, self.xi, self.Ag) - S,
                   min(W0[0], h1), max(W0[0], h1), xtol=1e-14)
        return W(h)
