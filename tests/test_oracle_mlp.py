"""Pins of the learned-closure oracle (oracle/mlp.py, or_mlp_features).

The closure is not in the paper; these pins tie the oracle to definitions
it does not share code with: torch's own bfloat16 conversion, closed-form
GELU values, the linear closed forms and the positive homogeneity of the
ReLU network, central differences and complex steps of the loss, the closed
form of the first Adam step, and closed-form closure targets in the Stokes
regime.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp


def test_bf16_rounding_matches_torch_conversion():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=2000) * 10 ** rng.uniform(-8, 8, 2000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gelu_closed_forms_and_derivative():
    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    # GELU(1) = Phi(1) = 0.841344746068543 (standard normal CDF at 1)
    assert mlp.gelu(1.0) == pytest.approx(0.841344746068543, rel=1e-13)
    assert mlp.gelu(-1.0) == pytest.approx(-(1 - 0.841344746068543), rel=1e-12)
    assert mlp.gelu(10.0) == pytest.approx(10.0, rel=1e-15)
    assert abs(mlp.gelu(-10.0)) < 1e-20
    x = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, rtol=1e-7, atol=1e-9)


def test_relu_network_closed_forms():
    """With every input, weight and bias of the hidden layers non-negative
    no unit is cut, and the network is the affine map
    ((X W1 + b1) W2 + b2) w3 + b3; with b2 far below zero every second-layer
    unit is cut and c = b3; with zero biases the network is positively
    homogeneous, c(a X) - b3 = a (c(X) - b3) for a > 0."""
    rng = np.random.default_rng(6)
    p = mlp.init_params(hidden=16, seed=2)
    X = np.zeros((21, mlp.K0))
    X[:, :mlp.NFEAT] = rng.random((21, mlp.NFEAT))
    q = dict(p)
    q["W1"] = np.abs(p["W1"])
    q["W2"] = np.abs(p["W2"])
    q["b1"] = rng.random(16)
    q["b2"] = rng.random(16)
    c, _ = mlp.forward(q, X, act="relu")
    affine = ((X @ q["W1"] + q["b1"]) @ q["W2"] + q["b2"]) @ q["w3"] + q["b3"][0]
    assert np.allclose(c, affine, rtol=1e-13, atol=1e-13)
    q["b2"] = np.full(16, -1e3)
    c, _ = mlp.forward(q, X, act="relu")
    assert np.all(c == q["b3"][0])
    z = dict(p)
    z["b1"] = np.zeros(16)
    z["b2"] = np.zeros(16)
    z["b3"] = np.array([0.7])
    c1, _ = mlp.forward(z, X, act="relu")
    c3, _ = mlp.forward(z, 3.5 * X, act="relu")
    assert np.allclose(c3 - 0.7, 3.5 * (c1 - 0.7), rtol=1e-12, atol=1e-14)
    # the GELU network is not homogeneous: the pin would catch a swapped activation
    g1, _ = mlp.forward(z, X)
    g3, _ = mlp.forward(z, 3.5 * X)
    assert not np.allclose(g3 - 0.7, 3.5 * (g1 - 0.7), rtol=1e-3)
    assert mlp.relu(-2.0) == 0.0 and mlp.relu(3.0) == 3.0
    assert mlp.relu_grad(-2.0) == 0.0 and mlp.relu_grad(3.0) == 1.0 and mlp.relu_grad(0.0) == 0.0


@pytest.mark.parametrize("act", ["gelu", "relu"])
def test_backprop_matches_central_differences(act):
    rng = np.random.default_rng(1)
    p = mlp.init_params(hidden=8, seed=3)
    p["b1"] = rng.normal(size=8) * 0.1
    p["b2"] = rng.normal(size=8) * 0.1
    X = np.zeros((13, mlp.K0))
    X[:, :mlp.NFEAT] = rng.random((13, mlp.NFEAT))
    t = 1.0 + 0.3 * rng.normal(size=13)
    loss, g = mlp.loss_and_grads(p, X, t, act=act)
    h = 1e-6
    for k, v in p.items():
        flat = v.reshape(-1)
        for idx in range(flat.size):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].reshape(-1)[idx] += h
            lp, _ = mlp.loss_and_grads(q, X, t, act=act)
            q[k].reshape(-1)[idx] -= 2 * h
            lm, _ = mlp.loss_and_grads(q, X, t, act=act)
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_bf16_mode_is_fp64_on_rounded_inputs():
    rng = np.random.default_rng(2)
    p = mlp.init_params(hidden=64, seed=5)
    X = np.zeros((32, mlp.K0))
    X[:, :mlp.NFEAT] = rng.random((32, mlp.NFEAT))
    c16, s16 = mlp.forward(p, X, bf16_inputs=True)
    q = dict(p)
    q["W1"] = mlp.bf16(p["W1"])
    q["W2"] = mlp.bf16(p["W2"])
    Z1 = mlp.bf16(X) @ q["W1"] + p["b1"]
    A1 = mlp.gelu(Z1)
    Z2 = mlp.bf16(A1) @ q["W2"] + p["b2"]
    c = mlp.gelu(Z2) @ p["w3"] + p["b3"][0]
    assert np.allclose(c16, c, rtol=1e-15, atol=1e-15)


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so every parameter
    moves by -lr g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    z = {"w": np.zeros(3)}
    P, M, V = mlp.adam_step(p, g, z, z, 1, 0.01)
    want = p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(P["w"], want, rtol=1e-14)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(4)
    p = mlp.init_params(hidden=16, seed=1)
    X = np.zeros((256, mlp.K0))
    X[:, :mlp.NFEAT] = rng.random((256, mlp.NFEAT))
    t = 1.0 + 0.4 * X[:, 0] - 0.2 * X[:, 2] ** 2
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    l0, _ = mlp.loss_and_grads(p, X, t)
    for it in range(1, 301):
        loss, g = mlp.loss_and_grads(p, X, t)
        p, m, v = mlp.adam_step(p, g, m, v, it, 3e-3)
    assert loss < 0.05 * l0


# ----------------------------------------------------------- features and targets
def _uniform_fields(nb, eps, u):
    n = int(np.prod(nb))
    return np.full(n, eps), np.tile(np.asarray(u, float)[:, None], (1, n))


def test_target_is_one_when_fields_are_fresh():
    w = synth.tiny(seed=7, n=3000)
    o = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine)
    f, t, Fs = oracle.mlp_features(w.desc, w.pos_d, w.vel, o["eps_bulk"], o["u_bulk"], o["var_bulk"], o["u_bulk"])
    assert np.all(t == 1.0)
    assert np.array_equal(Fs, o["force"])
    assert np.allclose(f[:, 6], [oracle.gather(w.desc, o["var_bulk"], x)[0] for x in w.pos_d[:, :3]])


def test_target_in_stokes_regime_is_velocity_ratio():
    """eps = 1, particles at rest, tiny flow (Wen-Yu Stokes limit F = 3 pi mu d u):
    doubling the fresh fluid velocity doubles the drag, so c* = 2; the
    features are eps = 1, zero porosity gradient, Re and |s| of the stale flow."""
    desc = synth.make_desc((0, 0, 0), (1, 1, 1), (8, 8, 8), 2, fp64=True, law=1)
    nb = (4, 4, 4)
    eps, us = _uniform_fields(nb, 1.0, [1e-9, 0.0, 0.0])
    _, uf = _uniform_fields(nb, 1.0, [2e-9, 0.0, 0.0])
    var = np.full(int(np.prod(nb)), 0.25)
    rng = np.random.default_rng(0)
    n = 40
    pos = np.zeros((n, 4))
    pos[:, :3] = rng.random((n, 3))
    pos[:, 3] = 0.003
    vel = np.zeros((n, 4))
    f, t, Fs = oracle.mlp_features(desc, pos, vel, eps, us, var, uf)
    # Wen-Yu at eps = 1 is Stokes drag times the Schiller-Naumann factor
    re1 = 1000.0 * 0.003 * 1e-9 / 1e-3
    want = 2.0 * (1 + 0.15 * (2 * re1) ** 0.687) / (1 + 0.15 * re1 ** 0.687)
    assert np.allclose(t, want, rtol=1e-12) and abs(want - 2.0) < 1e-4
    # interpolating a constant carries one rounding
    assert np.allclose(f[:, 0], 1.0, rtol=0, atol=1e-15) and np.allclose(f[:, 3:6], 0.0, atol=1e-13)
    assert np.allclose(f[:, 6], 0.25)
    re = 1000.0 * 0.003 * 1e-9 / 1e-3
    assert np.allclose(f[:, 1], math.log10(1 + re), rtol=1e-12)
    assert np.allclose(f[:, 2], 1e-9)
    assert np.allclose(Fs[0], 3 * math.pi * 1e-3 * 0.003 * 1e-9 * (1 + 0.15 * re ** 0.687), rtol=1e-12)


@pytest.mark.parametrize("act", ["gelu", "relu"])
def test_backprop_matches_complex_step_derivatives(act):
    """The FP64 backprop against complex-step derivatives of the oracle's
    own forward pass (Squire & Trapp 1998: f'(x) = Im f(x + ih) / h with no
    subtractive cancellation, so h = 1e-30 gives the derivative to machine
    precision; the GELU's erf and the matrix products are analytic, and the
    ReLU is linear on the piece each pre-activation lies on).  Every
    parameter of a small network agrees to 1e-10 relative: the FP64
    reference mode of the closure's gradient."""
    rng = np.random.default_rng(4)
    p = mlp.init_params(hidden=8, seed=5)
    p["b1"] = rng.normal(size=8) * 0.1
    p["b2"] = rng.normal(size=8) * 0.1
    X = np.zeros((17, mlp.K0))
    X[:, :mlp.NFEAT] = rng.random((17, mlp.NFEAT))
    t = 1.0 + 0.3 * rng.normal(size=17)
    _, g = mlp.loss_and_grads(p, X, t, act=act)
    h = 1e-30
    worst = 0.0
    for k, v in p.items():
        flat = v.reshape(-1)
        for idx in range(flat.size):
            q = {kk: vv.astype(np.complex128) for kk, vv in p.items()}
            q[k].reshape(-1)[idx] += 1j * h
            c, _ = mlp.forward(q, X, act=act)
            d = np.mean((c - t) ** 2).imag / h
            ref = g[k].reshape(-1)[idx]
            err = abs(ref - d) / max(abs(d), 1e-12)
            worst = max(worst, err)
            assert err <= 1e-10, (k, idx, ref, d)
    print("worst relative difference from the complex step", worst)
