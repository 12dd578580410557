"""Closed-form and exact solutions used to pin the oracle (test infrastructure).

* ``swe_riemann``: exact solution of the fixed-bed shallow-water Riemann problem
  (the A_g = 0, flat-bed special case of the dSVE system, Eq. SV-Ex with q_s = 0
  and z constant). Standard textbook construction: two nonlinear waves, each a
  shock (Rankine-Hugoniot) or a rarefaction (Riemann invariants); the star depth
  solves f_L(h*) + f_R(h*) + u_R - u_L = 0 (Newton), no dry bed.
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
