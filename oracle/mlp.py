"""FP64 oracle of the learned drag closure (not part of the paper).

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline use this module; the CUDA library never does.

The closure is a small multilayer perceptron c = f(features) that scales
the drag computed from stale bulk fields, F = c F_stale, standing in for a
fresh fine-to-bulk average.  Network (features padded to K0 = 16):

    Z1 = X W1 + b1,   A1 = act(Z1)            X: [B, 16], W1: [16, H]
    Z2 = A1 W2 + b2,  A2 = act(Z2)            W2: [H, H]
    c  = A2 w3 + b3                           w3: [H]
    loss = mean (c - c*)^2

The activation is one of two: GELU, the exact form x Phi(x) with Phi the
standard normal CDF (Hendrycks & Gimpel), or ReLU, max(x, 0) (its
derivative taken as 0 at x = 0).  Training is Adam (Kingma & Ba) on FP32-style master
weights.  With ``bf16=True`` the inputs of the two forward matrix products
(X, W1, A1, W2) and of the backward product dZ2 W2^T are rounded to
bfloat16 (round to nearest even) exactly where the tensor-core kernels round
them; all arithmetic is then done in float64, so the oracle isolates the
kernels' accumulation error from their input quantisation.

Written from the definitions above as plain numpy; the gradients are the
chain rule written out layer by layer (pinned against central differences).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

K0 = 16          # padded feature width
NFEAT = 7        # eps, log10(1+Re), |s|, grad eps (3), sigma^2


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest, ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + erf(x / np.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)
    return cdf + x * pdf


def relu(x):
    """max(x, 0); for complex x (a complex step) the branch follows the real
    part, so the step differentiates the piece it lies on."""
    x = np.asarray(x)
    return np.where(x.real > 0, x, 0.0 * x)


def relu_grad(x):
    return (np.asarray(x).real > 0).astype(np.float64)


ACTIVATIONS = {"gelu": (gelu, gelu_grad), "relu": (relu, relu_grad)}


def init_params(hidden: int = 64, seed: int = 0) -> dict:
    """He-style uniform init from a Philox stream (the same numbers are
    handed to the GPU; the GPU never draws its own)."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 77]))
    def u(shape, fan_in):
        b = np.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, shape)
    return dict(W1=u((K0, hidden), NFEAT), b1=np.zeros(hidden),
                W2=u((hidden, hidden), hidden), b2=np.zeros(hidden),
                w3=u((hidden,), hidden) * 0.1, b3=np.array([1.0]))


def _exact(a):
    """float64, or complex128 for complex values (so that the forward pass
    can be differentiated by a complex step)."""
    return np.asarray(a, dtype=np.result_type(a, np.float64))


def forward(p: dict, X: np.ndarray, bf16_inputs: bool = False, act: str = "gelu"):
    q = (lambda a: bf16(a)) if bf16_inputs else _exact
    f = ACTIVATIONS[act][0]
    Z1 = q(X) @ q(p["W1"]) + p["b1"]
    A1 = f(Z1)
    Z2 = q(A1) @ q(p["W2"]) + p["b2"]
    A2 = f(Z2)
    c = A2 @ p["w3"] + p["b3"][0]
    return c, dict(X=X, Z1=Z1, A1=A1, Z2=Z2, A2=A2)


def loss_and_grads(p: dict, X: np.ndarray, target: np.ndarray, bf16_inputs: bool = False, act: str = "gelu"):
    q = (lambda a: bf16(a)) if bf16_inputs else (lambda a: np.asarray(a, np.float64))
    dact = ACTIVATIONS[act][1]
    B = X.shape[0]
    c, s = forward(p, X, bf16_inputs, act)
    r = c - target
    loss = float(np.mean(r * r))
    dc = 2.0 * r / B
    g = {}
    g["w3"] = s["A2"].T @ dc
    g["b3"] = np.array([dc.sum()])
    dA2 = np.outer(dc, p["w3"])
    dZ2 = dA2 * dact(s["Z2"])
    g["W2"] = q(s["A1"]).T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dA1 = q(dZ2) @ q(p["W2"]).T
    dZ1 = dA1 * dact(s["Z1"])
    g["W1"] = q(X).T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


ADAM = dict(beta1=0.9, beta2=0.999, eps=1e-8)


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float):
    """One Adam update (t counts from 1); returns new (p, m, v)."""
    b1, b2, e = ADAM["beta1"], ADAM["beta2"], ADAM["eps"]
    P, M, V = {}, {}, {}
    for k in p:
        M[k] = b1 * m[k] + (1 - b1) * g[k]
        V[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = p[k] - lr * mh / (np.sqrt(vh) + e)
    return P, M, V
