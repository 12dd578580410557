"""FP64 reference of the learned |A|_Psi surrogate (test infrastructure).

A multilayer perceptron 7 -> 128 -> 128 -> 128 -> 128 -> 9 with GELU after
each hidden layer, mean-squared-error loss on standardised outputs and the
Adam update (Kingma & Ba 2015). GELU uses the tanh form of Hendrycks & Gimpel
(2016), gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).

Parameters are one packed float vector, layer by layer: W_l (out x in,
row-major) then b_l. With bf16=True the forward and backward passes round
the operands of every matrix product (weights, activations, output
gradients) to bfloat16 (round to nearest even), the points where the CUDA
kernels hold bfloat16 values; all other arithmetic stays in float64.
"""
from __future__ import annotations

import numpy as np

SIZES = (7, 128, 128, 128, 128, 9)
C_GELU = np.sqrt(2.0 / np.pi)


def layer_shapes():
    return [(SIZES[i + 1], SIZES[i]) for i in range(len(SIZES) - 1)]


def n_params() -> int:
    return sum(o * i + o for o, i in layer_shapes())


def unpack(theta: np.ndarray):
    """[(W, b), ...] views into the packed vector."""
    out, k = [], 0
    for o, i in layer_shapes():
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + 0.044715 * x ** 3)))


def gelu_prime(x):
    t = np.tanh(C_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * x * x)


def forward(theta, X, bf16=False):
    """Y [n, 9] and the cache (pre-activations, activations) for backward."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = unpack(np.asarray(theta, dtype=np.float64))
    a = np.asarray(X, dtype=np.float64)
    acts, pres = [a], []
    for li, (W, b) in enumerate(layers):
        z = rnd(a) @ rnd(W).T + b
        pres.append(z)
        a = gelu(z) if li < len(layers) - 1 else z
        acts.append(a)
    return a, (pres, acts)


def mse(Y, T):
    """Mean over all entries of (Y - T)^2 and its gradient with respect to Y."""
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(theta, cache, dY, bf16=False):
    """Packed gradient of the loss with respect to theta, given dL/dY."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = unpack(np.asarray(theta, dtype=np.float64))
    pres, acts = cache
    grads = []
    g = np.asarray(dY, dtype=np.float64)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        dz = g
        dW = rnd(dz).T @ rnd(acts[li])
        db = dz.sum(axis=0)
        grads.append((dW, db))
        if li > 0:
            g = (rnd(dz) @ rnd(W)) * gelu_prime(pres[li - 1])
    grads.reverse()
    return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_lr(t, total, lr0, floor=0.05):
    """Step size of Adam step t (counting from 1) under the training schedule
    (a reading: the paper's surrogate is not in the paper): cosine decay from
    lr0 at t = 1 to floor * lr0 at t = total + 1, constant after that,
    lr_t = lr0 (floor + (1 - floor) (1 + cos(pi f)) / 2), f = min(1, (t - 1) / total)."""
    f = min(1.0, (t - 1) / total) if total > 0 else 0.0
    return lr0 * (floor + (1.0 - floor) * 0.5 * (1.0 + np.cos(np.pi * f)))


def features(WL, WR, Ag):
    """Raw surrogate inputs [n, 7]: h_L, q_L, z_L, h_R, q_R, z_R, A_g."""
    WL, WR = np.asarray(WL), np.asarray(WR)
    n = WL.shape[1]
    return np.stack([WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], np.broadcast_to(Ag, (n,))], axis=1)
