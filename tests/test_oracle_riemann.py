"""Exact movable-bed Riemann solutions (oracle/exact.py) and the oracle's
convergence to them: the benchmark's Riemann problem (left h = 2, u = 0.25,
z = 0; right h = 1, u = 0.2, z = 0.5; A_g = 0.01, p = 0.4) and the paper's
Test 1 states (tests/golden/paper_test1_states.json, Sec. 4.1)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import exact as X
from paper_1912_04791_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_test1_states.json")


@pytest.fixture(scope="module")
def bench_rp():
    return X.MovableBedRiemann((2.0, 0.5, 0.0), (1.0, 0.2, 0.5), Ag=0.01, xi=W.XI_P04)


@pytest.fixture(scope="module")
def paper_rp():
    d = json.load(open(GOLD))
    return d, X.MovableBedRiemann(d["WL"], d["WR"], Ag=d["Ag"], xi=d["xi"])


def test_fixed_bed_limit_is_textbook_dam_break():
    R = X.MovableBedRiemann((2.0, 0.3, 0.0), (1.0, -0.1, 0.0), Ag=0.0, xi=1.0)
    x = np.linspace(0, 10, 41)
    h, q, z = R.sample(x, 0.5, 5.0)
    he, qe = X.swe_riemann(2.0, 0.15, 1.0, -0.1, x, 0.5, 5.0)
    assert R.converged
    assert np.abs(h - he).max() < 1e-10 and np.abs(q - qe).max() < 1e-10 and np.abs(z).max() < 1e-12


@pytest.mark.parametrize("which", ["bench", "paper"])
def test_exact_solution_is_consistent(which, bench_rp, paper_rp):
    R = bench_rp if which == "bench" else paper_rp[1]
    assert R.converged and R.lax_ok()
    assert all(r < 1e-12 for r in R.rh_residuals())
    assert np.abs(R.states[-1] - R.WR).max() < 1e-9
    # inside each rarefaction fan the solution is self-similar: lambda_i(W(S)) = S
    for i, (W1, kind, (s0, s1)) in enumerate(R.waves):
        if kind == "rarefaction":
            for S in np.linspace(s0, s1, 5)[1:-1]:
                Wm = R._fan_state(R.states[i], i, S)
                assert X._lam(Wm, i, R.g, R.xi, R.Ag) == pytest.approx(S, abs=1e-10)


def _l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_oracle_converges_to_benchmark_riemann_solution(bench_rp):
    law = O.grass(0.01, xi=W.XI_P04)
    errs = []
    for n in (400, 800, 1600):
        P = W.movable_bed_riemann(n)
        h, q, z, t, _, _ = O.run(O.make_cfg(n, 0, 10, 0.9, law), P.h, P.q, P.z, t_end=1.0)
        he, qe, ze = bench_rp.sample(W.cell_centres(n, 0, 10), t, 5.0)
        errs.append([_l1(h, he), _l1(q, qe), _l1(z, ze)])
    errs = np.array(errs)
    assert (errs[1:] < errs[:-1]).all(), errs
    assert (errs[-1] < [1.2e-3, 4e-3, 1.6e-3]).all(), errs


def test_oracle_converges_to_paper_test1(paper_rp):
    d, R = paper_rp
    law = O.grass(d["Ag"], xi=d["xi"])
    errs = []
    for n in (500, 1000, 2000):
        P = W.Problem("test1", n, 0.0, d["length"], 0.9, d["t_end"], d["Ag"], d["xi"],
                      *W.riemann(n, 0.0, d["length"], d["x0"], d["WL"], d["WR"]))
        h, q, z, t, _, _ = O.run(O.make_cfg(n, 0, d["length"], 0.9, law), P.h, P.q, P.z,
                                 t_end=d["t_end"])
        he, qe, ze = R.sample(W.cell_centres(n, 0, d["length"]), t, d["x0"])
        errs.append([_l1(h, he), _l1(q, qe), _l1(z, ze)])
    errs = np.array(errs)
    assert (errs[1:] < errs[:-1]).all(), errs
