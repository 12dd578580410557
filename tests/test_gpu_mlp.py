"""The |A|_Psi surrogate on the GPU: tensor-core forward and backward kernels
against the FP64 reference MLP (oracle/mlp.py), training, harvested labels
against the oracle's |A|_Psi, and the surrogate time step.

Tolerances: the GPU holds weights, activations and output gradients in
bfloat16 and accumulates in float32. Against the reference that rounds the
same operands to bfloat16 (everything else float64), outputs agree to 1e-2 of
their scale at worst (a float32/float64 difference can flip one bfloat16
rounding) and 1e-4 typically; gradients to a cosine above 0.999 and a relative
norm error below 2e-2."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in M.layer_shapes():
        parts.append(rng.standard_normal(o * i) * scale * np.sqrt(2.0 / i))
        parts.append(rng.standard_normal(o) * 0.1)
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("train_engine", [0, 1], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("n", [1, 63, 64, 127, 129, 1000, 4099])
def test_forward_matches_reference(gpu, n, train_engine):
    """The training forward pass: on tcgen05 the fused two-group kernel, which
    also stores every hidden layer's Z and H, bit-identical to its inference
    use (fused = 2; tanh.approx GELU, so the median bound of the tcgen05
    inference test); on mma.sync the per-layer kernels, which accumulate like
    the single-kernel mma.sync inference and agree with it to 1e-5."""
    theta = _theta(1)
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 7)).astype(np.float32)
    ref, _ = M.forward(theta, X.astype(np.float64), bf16=True)
    with gpu.Mlp(8192) as net:
        net.set_params(theta)
        net.set_train_engine(train_engine)
        y = net.forward(X, fused=False)
        yf = net.forward(X, fused=True)
        y2 = net.forward(X, fused=2)
    sc = np.abs(ref).max()
    err = np.abs(y - ref)
    med = 1e-4 if train_engine == 1 else 2e-4
    assert err.max() <= 1e-2 * sc, err.max()
    if n >= 64:  # a median over fewer than 576 outputs says little
        assert np.median(err) <= med * sc, np.median(err)
    if train_engine == 1:
        assert np.abs(yf - y).max() <= 1e-5 * sc
    else:
        assert np.array_equal(y, y2)


@pytest.mark.parametrize("fused", [2, 3], ids=["two_groups", "pipeline"])
@pytest.mark.parametrize("n", [1, 127, 128, 129, 256, 257, 385, 1000, 4099, 8192])
def test_forward_tcgen05_matches_reference(gpu, n, fused):
    """The tcgen05/TMEM inference kernel (two 128-row tiles per CTA) against
    the reference with bf16 operands. Its GELU takes tanh.approx (relative error
    below 2^-10.9), which moves a pre-rounding activation by at most about
    2.5e-4 |x|: a bfloat16 rounding flips in a few per cent of activations, the
    same size of effect as the float32/float64 difference; the bound is the
    per-layer-kernel one with the median doubled."""
    theta = _theta(1)
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal((n, 7)).astype(np.float32)
    ref, _ = M.forward(theta, X.astype(np.float64), bf16=True)
    with gpu.Mlp(8192) as net:
        net.set_params(theta)
        y_tc = net.forward(X, fused=fused)
        y_mma = net.forward(X, fused=1)
        y_other = net.forward(X, fused=5 - fused)
    sc = np.abs(ref).max()
    err = np.abs(y_tc - ref)
    print(f"n={n} tcgen05 vs reference: max {err.max() / sc:.2e}, median {np.median(err) / sc:.2e} of scale")
    assert np.isfinite(y_tc).all()
    assert err.max() <= 1e-2 * sc and np.median(err) <= 2e-4 * sc, (err.max() / sc, np.median(err) / sc)
    assert np.abs(y_tc - y_mma).max() <= 1e-2 * sc
    # both tcgen05 kernels do the same arithmetic in the same order
    assert np.array_equal(y_tc, y_other)


def test_tcgen05_bounded_wait_reports_timeout(gpu):
    """Failure detection of the tensor-core pipeline without a GPU fault: the
    test hook withholds one accumulator hand-off in the first CTA, so that the
    epilogue's bounded wait (about a second) runs out; the call reports
    ADOT_E_TIMEOUT, and the same network then gives the same outputs as
    before (the hook clears itself; clearing it explicitly also works)."""
    theta = _theta(1)
    X = np.random.default_rng(7).standard_normal((4099, 7)).astype(np.float32)
    with gpu.Mlp(8192) as net:
        net.set_params(theta)
        ref = net.forward(X, fused=3)
        net.inject_fault(1)
        with pytest.raises(gpu.AdotError) as err:
            net.forward(X, fused=3)
        assert err.value.status == gpu.E_TIMEOUT
        assert np.array_equal(net.forward(X, fused=3), ref)
        net.inject_fault(1)
        net.inject_fault(0)
        assert np.array_equal(net.forward(X, fused=3), ref)
        with pytest.raises(gpu.AdotError):
            net.inject_fault(2)


def test_engine_value_checked(gpu):
    with gpu.Mlp(64) as net:
        for e in (1, 2, 0):
            net.set_engine(e)
        with pytest.raises(gpu.AdotError):
            net.set_engine(3)


@pytest.mark.parametrize("train_engine", [0, 1], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("n", [2048, 1000])
def test_gradient_matches_reference(gpu, n, train_engine):
    """Forward, backward and the weight gradients (the batch rows as the
    reduction dimension; 1000 rows leave ragged 128-row and 512-row chunks)."""
    theta = _theta(2)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 7)).astype(np.float32)
    T = rng.standard_normal((n, 9)).astype(np.float32)
    Y, cache = M.forward(theta, X.astype(np.float64), bf16=True)
    loss_ref, dY = M.mse(Y, T.astype(np.float64))
    g_ref = M.backward(theta, cache, dY, bf16=True)
    with gpu.Mlp(n) as net:
        net.set_params(theta)
        net.set_train_engine(train_engine)
        loss, g = net.gradient(X, T)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    cos = float(g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref)))
    rel = float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref))
    assert cos > 0.999 and rel < 2e-2, (cos, rel)
    # and against the exact float64 gradient (no bfloat16 anywhere)
    Y64, c64 = M.forward(theta, X.astype(np.float64))
    g64 = M.backward(theta, c64, M.mse(Y64, T.astype(np.float64))[1])
    assert float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64))) > 0.99


def test_train_engines_agree(gpu):
    """tcgen05 and mma.sync training on the same batch: bf16 operands, float32
    accumulation in another order, and the tcgen05 forward's GELU through
    tanh.approx (a bf16 rounding flips in a few per cent of activations), so
    the bounds against the reference apply between the engines too."""
    theta = _theta(5)
    rng = np.random.default_rng(9)
    n = 4096
    X = rng.standard_normal((n, 7)).astype(np.float32)
    T = rng.standard_normal((n, 9)).astype(np.float32)
    out = []
    with gpu.Mlp(n) as net:
        for e in (0, 1):
            net.set_params(theta)
            net.set_train_engine(e)
            out.append(net.gradient(X, T))
        with pytest.raises(gpu.AdotError):
            net.set_train_engine(2)
    (l0, g0), (l1, g1) = out
    assert l0 == pytest.approx(l1, rel=1e-3)
    assert float(g0 @ g1 / (np.linalg.norm(g0) * np.linalg.norm(g1))) > 0.999
    assert float(np.linalg.norm(g0 - g1) / np.linalg.norm(g1)) < 2e-2


def test_params_roundtrip_and_padding(gpu):
    theta = _theta(4).astype(np.float32)
    with gpu.Mlp(128) as net:
        net.set_params(theta)
        assert np.array_equal(net.get_params(), theta)


def _edge_dataset(n, seed):
    WL, WR = W.random_edges(n, seed, h_range=(0.5, 2.0), fr_range=(-0.6, 0.6), rel_jump=0.05,
                            dz_scale=0.02)
    rng = np.random.default_rng(seed + 1)
    Ag = rng.uniform(0.001, 0.02, n)
    T = np.stack([O.abs_psi(O.grass(a, xi=W.XI_P04), WL[:, k:k + 1], WR[:, k:k + 1])[0]
                  for k, a in enumerate(Ag)])
    X = np.concatenate([WL.T, WR.T, Ag[:, None]], axis=1)
    return X.astype(np.float32), T.astype(np.float32)


@pytest.mark.parametrize("train_engine", [0, 1], ids=["tcgen05", "mma_sync"])
def test_training_reduces_loss(gpu, train_engine):
    X, T = _edge_dataset(3000, 5)
    with gpu.Mlp(1024) as net:
        net.set_train_engine(train_engine)
        net.set_params(_theta(6, 0.5))
        net.set_data(X, T)
        st, box = net.stats()
        assert np.allclose(st[:7], X.mean(0), rtol=1e-4, atol=1e-5)
        assert np.allclose(st[7:14], X.std(0), rtol=1e-3)
        h = net.train(400, 1024, lr=2e-3, seed=7)
    assert np.isfinite(h).all()
    assert h[-20:].mean() < 0.1 * h[:5].mean(), (h[:5], h[-20:])


def test_harvest_labels_match_oracle(gpu):
    P = W.smooth_periodic(5000)
    for prec in (0, 1):
        with gpu.Solver(gpu.config_for(P, prec)) as s:
            s.set_state(P.h, P.q, P.z)
            s.step(20)
            X, T = gpu.adot_harvest(s.ctx, 3000, seed=11)
        WL = X[:, 0:3].T.astype(np.float64)
        WR = X[:, 3:6].T.astype(np.float64)
        assert (X[:, 6] == np.float32(P.Ag)).all()
        ref = O.abs_psi(O.grass(P.Ag, xi=P.xi), WL, WR)
        sc = np.abs(ref).max(axis=1, keepdims=True)
        assert (np.abs(T - ref) <= 1e-5 * sc).all()


@pytest.mark.parametrize("engine", [0, 1, 2])
def test_surrogate_all_fallback_equals_analytic_path(gpu, engine):
    """With the fallback band covering every Froude number each edge takes the
    analytic eigenstructure: the surrogate step equals the plain float32 step."""
    P = W.smooth_periodic(3000)
    X, T = _edge_dataset(500, 8)
    with gpu.Mlp(512) as net:
        net.set_engine(engine)
        net.set_params(_theta(9))
        net.set_data(X, T)
        with gpu.Solver(gpu.config_for(P, gpu.FP32, block_threads=256, reg_cap=64)) as s:
            s.set_state(P.h, P.q, P.z)
            gpu.adot_set_surrogate(s.ctx, net, 0.0, 100.0)
            s.step(30)
            a = s.get_state()
            edges, fb = gpu.adot_surrogate_stats(s.ctx)
        assert edges == fb == 30 * 3001
    with gpu.Solver(gpu.config_for(P, gpu.FP32, block_threads=256, reg_cap=64)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(30)
        b = s.get_state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.fixture(scope="module")
def trained_smooth_net(gpu):
    """Parameters, data and oracle run of a network trained on edges harvested
    from the smooth periodic problem (N = 4096)."""
    P = W.smooth_periodic(4096)
    with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
        s.set_state(P.h, P.q, P.z)
        Xs, Ts = [], []
        for k in range(6):
            X, T = gpu.adot_harvest(s.ctx, 20000, seed=100 + k)
            Xs.append(X), Ts.append(T)
            s.step(40)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    with gpu.Mlp(8192) as net:
        net.set_params(_theta(10, 0.5))
        net.set_data(X, T)
        h = net.train(1500, 8192, lr=2e-3, seed=3)
        theta = net.get_params()
    return P, X, T, theta, h


@pytest.mark.parametrize("engine", [0, 2])
def test_trained_surrogate_engines_agree(gpu, trained_smooth_net, engine):
    """The tcgen05 engines and the mma.sync engine drive the same trained
    network through 30 surrogate steps: same fallback count, increments within
    1e-3 (L1, relative) of each other."""
    P, X, T, theta, _ = trained_smooth_net
    out = []
    for eng in (engine, 1):
        with gpu.Mlp(512) as net:
            net.set_engine(eng)
            net.set_params(theta)
            net.set_data(X, T)
            with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
                s.set_state(P.h, P.q, P.z)
                gpu.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
                s.step(30)
                out.append((s.get_state(), gpu.adot_surrogate_stats(s.ctx)))
    (a, sa), (b, sb) = out
    assert sa == sb
    for x, y, x0 in zip(a, b, (P.h, P.q, P.z)):
        assert np.abs((x - x0) - (y - x0)).sum() <= 1e-3 * np.abs(y - x0).sum()


def test_surrogate_eval_matches_network_on_state_edges(gpu, trained_smooth_net):
    """adot_surrogate_eval (tcgen05 engine) on every edge of a periodic state
    equals the per-layer forward kernels applied to the same edge inputs built
    on the host (left cell (e-1) mod n, right cell e mod n, the hi words of the
    float-float state, A_g, standardised with the network's statistics), to the
    bf16 bound of the forward tests; NaN rows match the fallback count, and the
    evaluation leaves the step statistics alone."""
    P, X, T, theta, _ = trained_smooth_net
    with gpu.Mlp(8192) as net:
        net.set_params(theta)
        net.set_data(X, T)
        st, _ = net.stats()
        with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
            s.set_state(P.h, P.q, P.z)
            s.step(10)
            gpu.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
            s.step(3)
            before = gpu.adot_surrogate_stats(s.ctx)
            absA, fb = gpu.adot_surrogate_eval(s.ctx, P.n + 1)
            assert gpu.adot_surrogate_stats(s.ctx) == before
            h, q, z = (a.astype(np.float32) for a in s.get_state())
            gpu.adot_set_surrogate(s.ctx, net, 0.0, 100.0)
            all_fb, fb_all = gpu.adot_surrogate_eval(s.ctx, P.n + 1)
        n = P.n
        e = np.arange(n + 1)
        L, R = (e - 1) % n, e % n
        Xe = np.stack([h[L], q[L], z[L], h[R], q[R], z[R], np.full(n + 1, P.Ag, np.float32)], axis=1)
        Zs = (Xe - st[:7]) / st[7:14]
        Y = np.concatenate([net.forward(Zs[i:i + 8192], fused=False) for i in range(0, n + 1, 8192)])
    assert fb == int(np.isnan(absA[0]).sum())
    assert fb_all == n + 1 and np.isnan(all_fb[0]).all()
    ok = ~np.isnan(absA[0])
    assert ok.sum() > 0.9 * (n + 1)
    got = (absA.T[ok] - st[14:23]) / st[23:32]
    ref = Y[ok]
    assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_trained_surrogate_step(gpu):
    """A network trained briefly (1500 steps) on edges harvested from the smooth
    periodic problem drives the same problem: the state stays finite, few edges
    fall back, and the increment over 50 steps stays within 5e-2 (L1, relative)
    of the oracle's, while the analytic FP32 path's increment, computed on the
    same state, stays within 1e-5. The trained-to-convergence network is held
    to 1e-3 at t_end in tests/test_gpu_surrogate_gain.py."""
    P = W.smooth_periodic(4096)
    with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
        s.set_state(P.h, P.q, P.z)
        Xs, Ts = [], []
        for k in range(6):
            X, T = gpu.adot_harvest(s.ctx, 20000, seed=100 + k)
            Xs.append(X), Ts.append(T)
            s.step(40)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right)
    ho, qo, zo, *_ = O.run(cfg, P.h, P.q, P.z, max_steps=50)
    with gpu.Mlp(8192) as net:
        net.set_params(_theta(10, 0.5))
        net.set_data(X, T)
        h = net.train(1500, 8192, lr=2e-3, seed=3)
        assert h[-50:].mean() < 1e-2
        with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
            s.set_state(P.h, P.q, P.z)
            gpu.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
            s.step(50)
            hs, qs, zs = s.get_state()
            edges, fb = gpu.adot_surrogate_stats(s.ctx)
    assert np.isfinite(hs).all() and edges == 50 * 4097
    assert fb / edges < 0.05
    with gpu.Solver(gpu.config_for(P, gpu.FP32)) as s:
        s.set_state(P.h, P.q, P.z)
        s.step(50)
        ha, qa, za = s.get_state()
    for a, c, b, a0 in ((hs, ha, ho, P.h), (qs, qa, qo, P.q), (zs, za, zo, P.z)):
        assert np.abs((a - a0) - (b - a0)).sum() <= 5e-2 * np.abs(b - a0).sum()
        assert np.abs((c - a0) - (b - a0)).sum() <= 1e-5 * np.abs(b - a0).sum()


def test_adam_update_matches_reference(gpu):
    """The update kernel of the training graph (Adam with the cosine-decayed
    step size) against oracle/mlp.py's adam and cosine_lr, element by element,
    on the same gradients, at t = 1, 2, mid-schedule and after the schedule's
    end. The kernel holds beta1, beta2, eps and lr0 as float32 constants, so
    the reference takes those float32 values; what remains is float32 rounding:
    a few ulp of each step's update plus half an ulp of each stored parameter."""
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    b1, b2, eps, lr0, T = f32(0.9), f32(0.999), f32(1e-8), f32(1e-3), 200
    rng = np.random.default_rng(21)
    theta0 = _theta(3)
    P = theta0.size
    th, m, v = theta0.copy(), np.zeros(P), np.zeros(P)
    S = np.zeros(P)  # sum of the reference's step magnitudes
    checked = []
    with gpu.Mlp(256) as net:
        net.set_params(theta0)
        for t in range(1, 261):
            g = (rng.standard_normal(P) * 10.0 ** rng.uniform(-3, 1, P)).astype(np.float32)
            net.apply_gradient(g, lr0, T)
            prev = th
            th, m, v = M.adam(th, g.astype(np.float64), m, v, t, lr=M.cosine_lr(t, T, lr0),
                              b1=b1, b2=b2, eps=eps)
            S += np.abs(th - prev)
            if t in (1, 2, 101, 260):
                got = net.get_params().astype(np.float64)
                bound = 2e-6 * S + t * 2.0 ** -24 * (np.abs(th) + S)
                err = np.abs(got - th)
                assert (err <= bound).all(), (t, (err / bound).max())
                assert np.abs(got - theta0).max() > 0.5 * t * lr0 * 0.05  # the parameters moved
                checked.append(t)
    assert checked == [1, 2, 101, 260]
