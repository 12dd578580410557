"""What the learned |A|_Psi surrogate gives against the analytic A-DOT path it
replaces (the dissipative half of Eq. DOTjumpN), on the smooth periodic
problem.

Accuracy: a network trained on edges the method itself generates (harvested
from the smooth problem at the sweep's sizes) drives the problem to t_end =
0.5 s at N = 1000, 4000 and 16000; its state stays within 1e-3 (L1, relative,
per variable) of the GPU FP64 path, which is parity-tested against the oracle,
and the analytic FP32 path within 1e-5.

Throughput: on the same 2^20-cell state, the increments of both forms over 20
steps against the oracle (1e-5 analytic, 1e-3 surrogate), the fallback
fraction, and cell-updates/s of each, timed with CUDA events. The surrogate
costs 7*128 + 3*128^2 + 128*9 = 51,200 multiply-adds (1.024e5 tensor flops) per
edge against ~700 float32 instructions of the analytic eigen-solve, so even at
the measured bf16 peak its edges per second stay below peak / 1.024e5 (about
1.8e10): on this GPU the network buys no speed over the analytic path, and the
test asserts that measured trade and the ceiling."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLOPS_PER_EDGE = 2 * (7 * 128 + 3 * 128 * 128 + 128 * 9)


@pytest.fixture(scope="module")
def sweep_net(gpu):
    """(parameters, inputs, labels) of a network trained on edges of the smooth
    problem at 1000 to 65536 cells, sampled at several times up to t_end."""
    Xs, Ts = [], []
    for n in (1000, 4000, 16000, 65536):
        P = W.smooth_periodic(n)
        with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
            s.set_state(P.h, P.q, P.z)
            for k in range(5):
                X, T = gpu.adot_harvest(s.ctx, 40000, seed=1000 * n + k)
                Xs.append(X), Ts.append(T)
                s.run_to(P.t_end * (k + 1) / 5)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    with gpu.Mlp(16384) as net:
        net.set_params(W.mlp_init())
        net.set_data(X, T)
        hist = net.train(4000, 16384, lr=2e-3, seed=7)
        theta = net.get_params()
    assert hist[-100:].mean() < 0.2 * hist[:10].mean()
    return theta, X, T


def _with_net(gpu, theta, X, T, fn):
    with gpu.Mlp(16384) as net:
        net.set_params(theta)
        net.set_data(X, T)
        return fn(net)


@pytest.mark.parametrize("n", [1000, 4000, 16000])
def test_surrogate_accuracy_at_t_end(gpu, sweep_net, n):
    theta, X, T = sweep_net
    P = W.smooth_periodic(n)
    out = {}
    for name, prec in (("fp64", gpu.FP64), ("fp32", gpu.FP32)):
        with gpu.Solver(gpu.config_for(P, prec)) as s:
            s.set_state(P.h, P.q, P.z)
            s.run_to(P.t_end)
            out[name] = s.get_state()

    def run(net):
        with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
            s.set_state(P.h, P.q, P.z)
            gpu.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
            s.run_to(P.t_end)
            t, _, _ = s.query()
            edges, fb = gpu.adot_surrogate_stats(s.ctx)
            return s.get_state(), t, fb / edges

    sur, t, fb = _with_net(gpu, theta, X, T, run)
    assert t == P.t_end and fb < 0.05
    for name, a_all, tol in (("fp32", out["fp32"], 1e-5), ("surrogate", sur, 1e-3)):
        for v, a, b in zip("hqz", a_all, out["fp64"]):
            err = np.abs(a - b).sum() / np.abs(b).sum()
            assert err <= tol, (name, v, err)


def test_surrogate_trade_against_analytic(gpu, sweep_net):
    torch = pytest.importorskip("torch")
    theta, X, T = sweep_net
    n, K, KT = 1 << 20, 20, 240
    P = W.smooth_periodic(n)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right)
    ho, qo, zo, *_ = O.run(cfg, P.h, P.q, P.z, max_steps=K)
    stream = torch.cuda.Stream()

    def timed(s):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        gpu.adot_enqueue_steps(s.ctx, KT)
        b.record(stream)
        torch.cuda.synchronize()
        gpu.adot_query(s.ctx)
        return n * KT / (a.elapsed_time(b) * 1e-3)

    def run(net):
        res = {}
        for name in ("analytic", "surrogate"):
            with gpu.Solver(gpu.config_for(P, gpu.FP32), stream=stream) as s:
                s.set_state(P.h, P.q, P.z)
                if name == "surrogate":
                    gpu.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
                s.step(K)
                got = s.get_state()
                edges, fb = gpu.adot_surrogate_stats(s.ctx)
                gpu.adot_step(s.ctx, 6)  # graph phase and capture outside the timed steps
                rate = timed(s)
            err = max(np.abs((a - a0) - (b - a0)).sum() / np.abs(b - a0).sum()
                      for a, b, a0 in zip(got, (ho, qo, zo), (P.h, P.q, P.z)))
            res[name] = {"cell_updates_per_s": rate, "l1_increment_vs_oracle": err,
                         "fallback_fraction": fb / edges if edges else 0.0}
        return res

    res = _with_net(gpu, theta, X, T, run)
    print(json.dumps(res))
    assert res["analytic"]["l1_increment_vs_oracle"] <= 1e-5
    assert res["surrogate"]["l1_increment_vs_oracle"] <= 1e-3
    assert res["surrogate"]["fallback_fraction"] < 0.05
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = json.load(fh)["bf16_tflops"] * 1e12
    except (OSError, ValueError, KeyError):
        peak = 2.25e15  # nominal dense bf16
    ceiling = peak / FLOPS_PER_EDGE  # edges (about one per cell) per second at the tensor peak
    assert res["surrogate"]["cell_updates_per_s"] <= ceiling
    # the measured trade: on this GPU the analytic eigen-solve is the faster form
    assert res["surrogate"]["cell_updates_per_s"] < res["analytic"]["cell_updates_per_s"]
