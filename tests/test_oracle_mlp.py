"""Pins of the surrogate's FP64 reference (oracle/mlp.py) and of the label
|A|_Psi, against finite differences, closed forms and library routines."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_1912_04791_gb300 import workloads as W


def test_gelu_against_erf_form_and_derivative():
    from scipy.special import erf
    x = np.linspace(-6, 6, 2001)
    exact = 0.5 * x * (1 + erf(x / np.sqrt(2)))
    assert np.abs(mlp.gelu(x) - exact).max() < 1e-3  # published accuracy of the tanh form
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    e = 1e-6
    fd = (mlp.gelu(x + e) - mlp.gelu(x - e)) / (2 * e)
    assert np.abs(mlp.gelu_prime(x) - fd).max() < 1e-8


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(mlp.n_params()) * 0.1
    X = rng.standard_normal((6, 7))
    T = rng.standard_normal((6, 9))
    Y, cache = mlp.forward(theta, X)
    L0, dY = mlp.mse(Y, T)
    g = mlp.backward(theta, cache, dY)
    idx = rng.choice(theta.size, 300, replace=False)
    for i in idx:
        e = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += e
        tm[i] -= e
        fd = (mlp.mse(mlp.forward(tp, X)[0], T)[0] - mlp.mse(mlp.forward(tm, X)[0], T)[0]) / (2 * e)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9, (i, g[i], fd)  # 1e-9: loss rounding / step


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    t1, m1, v1 = mlp.adam(th, g, m, v, 1, lr=1e-3)
    # with t = 1 the bias corrections give m_hat = g, v_hat = g^2
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each step
    moves theta by lr_t g / (|g| + eps): after T steps the sum of the step sizes."""
    rng = np.random.default_rng(5)
    th0 = rng.standard_normal(40)
    g = rng.standard_normal(40)
    th, m, v = th0.copy(), np.zeros(40), np.zeros(40)
    lrs = [mlp.cosine_lr(t, 30, 2e-3) for t in range(1, 41)]
    for t, lr in enumerate(lrs, start=1):
        th, m, v = mlp.adam(th, g, m, v, t, lr=lr)
        assert np.allclose(m, (1 - 0.9 ** t) * g, rtol=1e-13, atol=0)
        assert np.allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12, atol=0)
    ref = th0 - sum(lrs) * g / (np.abs(g) + 1e-8)
    assert np.abs(th - ref).max() <= 1e-13


def test_cosine_schedule_closed_forms():
    lr0, T = 1e-3, 200
    assert mlp.cosine_lr(1, T, lr0) == lr0
    assert abs(mlp.cosine_lr(T // 2 + 1, T, lr0) - 0.525 * lr0) <= 1e-18  # cos(pi/2) = 0
    assert abs(mlp.cosine_lr(T + 1, T, lr0) - 0.05 * lr0) <= 1e-18
    assert mlp.cosine_lr(T + 50, T, lr0) == mlp.cosine_lr(T + 1, T, lr0)
    # cos(pi f) + cos(pi (1 - f)) = 0: steps symmetric about the middle sum to 1.05 lr0
    for t in (2, 17, 64, 150):
        assert abs(mlp.cosine_lr(t, T, lr0) + mlp.cosine_lr(T + 2 - t, T, lr0) - 1.05 * lr0) <= 1e-18
    lr = [mlp.cosine_lr(t, T, lr0) for t in range(1, T + 2)]
    assert all(a > b for a, b in zip(lr, lr[1:]))
    assert mlp.cosine_lr(7, 0, lr0) == lr0  # no schedule length: constant


def test_label_is_gl3_average_of_lapack_abs():
    law = O.grass(0.01, xi=W.XI_P04)
    WL, WR = W.random_edges(200, 3)
    got = O.abs_psi(law, WL, WR)
    s, w = np.polynomial.legendre.leggauss(3)
    s, w = 0.5 * (s + 1), 0.5 * w
    for k in range(WL.shape[1]):
        ref = np.zeros((3, 3))
        for sk, wk in zip(s, w):
            p = WL[:, k] + sk * (WR[:, k] - WL[:, k])
            ev, V = np.linalg.eig(O.flux_matrix(law, p[0], p[1]))
            ref += wk * (V @ np.diag(np.abs(ev)) @ np.linalg.inv(V)).real
        assert np.abs(got[k] - ref.ravel()).max() <= 1e-10 * np.abs(ref).max()
