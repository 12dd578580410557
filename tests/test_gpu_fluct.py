"""Parity of the CUDA edge fluctuations (adot_fluctuations, Eq. DOTjumpN)
with the FP64 oracle, element by element, on seeded random edges.

Tolerances. FP64: per edge, max |D_gpu - D_oracle| <= 1e-12 (|D-|_inf + |D+|_inf),
the float64 bar of the method. FP32: the inputs are rounded to float-float and
every node evaluated in float32; the eigen-solve amplifies the float32 unit
roundoff (6e-8) by the conditioning of R (|lambda| / min gap, at most ~1e3
for the edges drawn here), so the per-edge bar is 1e-4 of the same norm."""
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


def _solver(gpu, Ag, xi, prec, law=0, **kw):
    cfg = gpu.make_config(16, 0.0, 1.0, 0.9, Ag, xi, precision=prec, law=law, **kw)
    return gpu.Solver(cfg)


@pytest.mark.parametrize("n", [1, 7, 256, 1000, 20011])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_random_edges_match_oracle(gpu, n, prec, tol):
    WL, WR = W.random_edges(n, 100 + n, fr_range=(-2.5, 2.5))
    Ag, xi = 0.01, W.XI_P04
    rm, rp = O.fluct(O.grass(Ag, xi=xi, g=G), WL, WR)
    with _solver(gpu, Ag, xi, prec) as s:
        dm, dp, rho = s.fluctuations(WL, WR)
    err = _rel_err(dm, dp, rm, rp)
    assert err.max() <= tol, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_jump_and_empty_batch(gpu, prec):
    WL, _ = W.random_edges(333, 5)
    with _solver(gpu, 0.01, W.XI_P04, prec) as s:
        dm, dp, _ = s.fluctuations(WL, WL.copy())
        assert (dm == 0).all() and (dp == 0).all()
        e = np.zeros((3, 0))
        dm, dp, rho = s.fluctuations(e, e.copy())
        assert dm.shape == (3, 0) and rho == 0.0


@pytest.mark.parametrize("prec", [0, 1])
def test_lake_at_rest_edges(gpu, prec):
    rng = np.random.default_rng(3)
    z = rng.integers(0, 512, size=(2, 4000)) / 1024.0
    WL = np.stack([1.0 - z[0], np.zeros(4000), z[0]])
    WR = np.stack([1.0 - z[1], np.zeros(4000), z[1]])
    with _solver(gpu, 0.01, W.XI_P04, prec) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    eps = 1e-16 if prec == 0 else 1.2e-7
    bound = 40 * eps * np.sqrt(G) * np.abs(z[1] - z[0])
    assert (np.abs(dm).max(axis=0) <= bound + 1e-300).all()
    assert (np.abs(dp).max(axis=0) <= bound + 1e-300).all()


def test_spectral_radius_output(gpu):
    WL, WR = W.random_edges(500, 8)
    law = O.grass(0.01, xi=W.XI_P04, g=G)
    s, _ = np.polynomial.legendre.leggauss(3)
    s = 0.5 * (s + 1)
    ref = 0.0
    for k in range(WL.shape[1]):
        for sk in s:
            p = WL[:, k] + sk * (WR[:, k] - WL[:, k])
            ref = max(ref, O.spectral_radius(law, p[0], p[1]))
    with _solver(gpu, 0.01, W.XI_P04, 0) as sv:
        _, _, rho = sv.fluctuations(WL, WR)
    assert rho == pytest.approx(ref, rel=1e-13)


def test_fixed_bed_coalescence_uses_newton_form(gpu):
    """A_g = 0 with a node exactly at Fr = 1: the double root 0 takes the
    coalescence reading in both implementations (FP64)."""
    h = np.array([0.5, 0.7, 1.3])
    c = np.sqrt(G * h)
    WL = np.stack([h, c * h * 0.98, np.zeros(3)])
    WR = np.stack([h, c * h * 1.02, np.zeros(3)])  # midpoint node at Fr = 1 exactly
    rm, rp = O.fluct(O.grass(0.0, xi=1.0, g=G), WL, WR)
    with _solver(gpu, 0.0, 1.0, 0) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    assert _rel_err(dm, dp, rm, rp).max() <= 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_near_critical_edges_use_fp64_root(gpu, prec, tol):
    """Small A_g near |Fr| = 1: two roots nearly coalesce (1 - arg^2 small);
    FP32 redoes those nodes in FP64 and must stay within its bar."""
    n = 3000
    rng = np.random.default_rng(9)
    h = rng.uniform(0.2, 2.0, n)
    fr = rng.uniform(0.97, 1.03, n) * rng.choice([-1, 1], n)
    q = fr * np.sqrt(G * h) * h
    WL = np.stack([h, q, np.zeros(n)])
    WR = np.stack([h * (1 + rng.uniform(-1e-3, 1e-3, n)), q * (1 + rng.uniform(-1e-3, 1e-3, n)),
                   rng.uniform(-1e-3, 1e-3, n)])
    law = O.grass(1e-5, xi=W.XI_P04, g=G)
    rm, rp = O.fluct(law, WL, WR)
    with _solver(gpu, 1e-5, W.XI_P04, prec) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    assert _rel_err(dm, dp, rm, rp).max() <= tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_mpm_law_edges(gpu, prec, tol):
    n = 4000
    rng = np.random.default_rng(10)
    h = rng.uniform(0.1, 0.6, n)
    q = rng.uniform(-1.2, 1.2, n)
    WL = np.stack([h, q, rng.uniform(0, 0.2, n)])
    WR = WL * (1 + rng.uniform(-0.05, 0.05, (3, n)))
    law = O.mpm(2.65, 1e-3, 0.02, xi=W.XI_P04, g=G)
    rm, rp = O.fluct(law, WL, WR)
    with _solver(gpu, 0.0, W.XI_P04, prec, law=1, s_rel=2.65, d50=1e-3, manning_n=0.02) as s:
        dm, dp, _ = s.fluctuations(WL, WR)
    assert _rel_err(dm, dp, rm, rp).max() <= tol


def test_device_pointers(gpu):
    torch = pytest.importorskip("torch")
    WL, WR = W.random_edges(1234, 11)
    rm, rp = O.fluct(O.grass(0.01, xi=W.XI_P04, g=G), WL, WR)
    with _solver(gpu, 0.01, W.XI_P04, 0) as s:
        tl, tr = torch.tensor(WL, device="cuda"), torch.tensor(WR, device="cuda")
        dm, dp, _ = s.fluctuations(tl, tr)
        torch.cuda.synchronize()
        assert _rel_err(dm.cpu().numpy(), dp.cpu().numpy(), rm, rp).max() <= 1e-12


def test_nonhyperbolic_state_reported(gpu):
    """A negative A_g drives k1 below zero: the library reports the state."""
    WL = np.array([[1.0], [2.0], [0.0]])
    WR = np.array([[1.1], [2.1], [0.0]])
    with _solver(gpu, -5.0, 1.0, 0) as s:
        with pytest.raises(gpu.AdotError) as e:
            s.fluctuations(WL, WR)
    assert e.value.status == gpu.E_NONHYPERBOLIC
