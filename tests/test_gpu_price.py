"""PRICE-C (Sec. 3.2, Eq. PRICEjump, AiPRICE, Apsi, Im) on the GPU against the
oracle: the stateless edge fluctuations, whole runs on grids of 1 to 4097
cells with every boundary kind, the friction source and the sediment feed, in
each of the three launch shapes, the still-water drift that places epsilon,
and the 1e7-cell benchmark workload in the launch configuration the benchmark
times.

Tolerances as for the DOT scheme: FP64 every value within 1e-12 of the
variable's scale; FP32 (float-float state, float32 fluctuations) the increment
W^K - W^0 within 1e-5 in L1 relative."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS = 1e-4
MPM = dict(s_rel=2.65, d50=1e-3, manning_n=0.02)
SHAPES = [(256, 64), (256, 40), (256, 32)]


def _laws(gpu, kind, Ag, xi):
    if kind == "grass":
        return O.grass(Ag, xi=xi), {}
    if kind == "mpm":
        return O.mpm(xi=xi, **MPM), dict(law=gpu.LAW_MPM, **MPM)
    return O.grass_thr(Ag, 0.3, xi=xi), dict(law=gpu.LAW_GRASS_THR, u_cr=0.3)


@pytest.mark.parametrize("kind", ["grass", "mpm", "thr"])
@pytest.mark.parametrize("nu,eps", [(0.05, 1e-4), (0.21, 1.0), (0.9, 0.3)])
def test_price_fluctuations_match_oracle(gpu, kind, nu, eps):
    WL, WR = W.random_edges(3001, 11)
    olaw, kw = _laws(gpu, kind, 0.01, W.XI_P04)
    rm, rp = O.price_fluct(olaw, WL, WR, nu, eps)
    sc = np.abs(rm).max(axis=1, keepdims=True) + np.abs(rp).max(axis=1, keepdims=True)
    for prec, tol in ((gpu.FP64, 1e-12), (gpu.FP32, 1e-4)):
        cfg = gpu.make_config(16, 0.0, 1.0, 0.9, 0.01, W.XI_P04, precision=prec,
                              scheme=gpu.SCHEME_PRICE_C, price_eps=eps, **kw)
        with gpu.Solver(cfg) as s:
            dm, dp = gpu.adot_price_fluctuations(s.ctx, WL, WR, nu)
        err = max((np.abs(dm - rm) / sc).max(), (np.abs(dp - rp) / sc).max())
        assert err <= tol, (prec, err)


def _problems():
    out = []
    for n in (1, 2, 31, 33, 257, 1000, 4097):
        out.append(("smooth", W.smooth_periodic(n), {}, {}))
    out.append(("riemann", W.movable_bed_riemann(301), {}, {}))
    P = W.gaussian_bump(500, Ag=0.001)
    out.append(("bump", P, {}, {}))
    out.append(("bump_mpm", P, {"mpm": True}, {}))
    S = W.soni_aggradation()
    out.append(("soni", S, {"power": True}, {"ks": S.extra["ks"]}))
    return out


def _oracle_cfg(P, flags, ks, eps):
    if flags.get("mpm"):
        law = O.mpm(xi=P.xi, **MPM)
    elif flags.get("power"):
        law = O.power(P.Ag, P.extra["beta"], xi=P.xi, g=P.g)
    else:
        law = O.grass(P.Ag, xi=P.xi, g=P.g)
    return O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, law, P.bc_left, P.bc_right, P.bcl, P.bcr,
                      ks=ks, scheme=O.SCHEME_PRICE_C, price_eps=eps)


def _gpu_kw(gpu, P, flags, ks):
    kw = dict(scheme=gpu.SCHEME_PRICE_C, price_eps=EPS, ks=ks)
    if flags.get("mpm"):
        kw.update(law=gpu.LAW_MPM, **MPM)
    elif flags.get("power"):
        kw.update(law=gpu.LAW_POWER, beta=P.extra["beta"])
    return kw


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{b}x{c}" for b, c in SHAPES])
@pytest.mark.parametrize("case", _problems(), ids=lambda c: f"{c[0]}{c[1].n}")
def test_price_runs_match_oracle(gpu, case, shape):
    name, P, flags, extra = case
    ks = extra.get("ks", 0.0)
    K = 40
    ho, qo, zo, to, so, _ = O.run(_oracle_cfg(P, flags, ks, EPS), P.h, P.q, P.z, max_steps=K)
    kw = _gpu_kw(gpu, P, flags, ks)
    for prec in (gpu.FP64, gpu.FP32):
        cfg = gpu.config_for(P, prec, block_threads=shape[0], reg_cap=shape[1], step_kernel=2, **kw)
        with gpu.Solver(cfg) as s:
            s.set_state(P.h, P.q, P.z)
            g0 = s.get_state()
            s.step(K)
            t, steps, _ = s.query()
            got = s.get_state()
        assert steps == so == K
        for a, b, a0, ag in zip(got, (ho, qo, zo), (P.h, P.q, P.z), g0):
            if prec == gpu.FP64:
                assert t == pytest.approx(to, rel=1e-13)
                sc = max(np.abs(b).max(), 1e-300)
                assert np.abs(a - b).max() <= 1e-12 * sc, (name, np.abs(a - b).max() / sc)
            else:
                assert t == pytest.approx(to, rel=1e-5)
                inc, ref = a - ag, b - a0
                assert np.abs(inc - ref).sum() <= 1e-5 * np.abs(ref).sum() + 1e-15 * a.size, \
                    (name, np.abs(inc - ref).sum() / max(np.abs(ref).sum(), 1e-300))


@pytest.mark.parametrize("eps", [1.0, 0.25, 1e-4])
def test_price_still_water_drift(gpu, eps):
    """A^Psi dW vanishes on still water, so a step moves h by a quarter of its
    second difference and z by eps times that of z (the oracle pins this). With
    eps = 1 the free surface stays level and q at rounding; with eps < 1 the
    surface tilts and a flow starts (PRICE-C as printed is not well-balanced),
    the same flow in the oracle and on the GPU."""
    P = W.lake_at_rest(300)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right,
                     scheme=O.SCHEME_PRICE_C, price_eps=eps)
    ho, qo, zo, *_ = O.run(cfg, P.h, P.q, P.z, max_steps=20)
    with gpu.Solver(gpu.config_for(P, gpu.FP64, scheme=gpu.SCHEME_PRICE_C, price_eps=eps)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(20)
        h, q, z = s.get_state()
    for a, b in ((h, ho), (q, qo), (z, zo)):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(ho).max(), np.abs(b).max())
    if eps == 1.0:
        assert np.abs(q).max() <= 1e-14 and np.abs(h + z - 1.0).max() <= 1e-14
    else:
        assert np.abs(h + z - 1.0).max() > 1e-3 and np.abs(q).max() > 1e-2


N_FULL = 10_000_000


@pytest.fixture(scope="module")
def full_price_oracle(oracle):
    P = W.smooth_periodic(N_FULL)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi, g=P.g), P.bc_left,
                     P.bc_right, scheme=O.SCHEME_PRICE_C, price_eps=EPS)
    h, q, z, t, steps, _ = O.run(cfg, P.h, P.q, P.z, max_steps=3)
    return P, (h, q, z, t)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_price_full_size_matches_oracle(gpu, full_price_oracle, prec):
    """The 1e7-cell benchmark workload, autotuned launch shape (as bench.py), 3 steps."""
    P, (ho, qo, zo, to) = full_price_oracle
    with gpu.Solver(gpu.config_for(P, getattr(gpu, prec), scheme=gpu.SCHEME_PRICE_C,
                                   price_eps=EPS)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(3)
        t, steps, _ = s.query()
        got = s.get_state()
    assert steps == 3
    for a, b, a0 in zip(got, (ho, qo, zo), (P.h, P.q, P.z)):
        if prec == "FP64":
            assert t == pytest.approx(to, rel=1e-13)
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        else:
            assert t == pytest.approx(to, rel=1e-5)
            inc, ref = a - a0, b - a0
            err = np.abs(inc - ref)
            assert err.sum() <= 1e-5 * np.abs(ref).sum(), err.sum() / np.abs(ref).sum()
