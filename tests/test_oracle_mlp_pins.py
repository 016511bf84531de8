"""Pins of the FP64 MLP oracle (oracle/mlp.py) to facts outside itself:
finite differences of its own forward pass and loss (which share no code
with the chain-rule formulas they check), closed forms of SiLU and of the
first Adam step, and the bfloat16 rounding rule checked by brute force."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _theta(seed, scale=0.5):
    r = synth.rng(seed)
    return np.concatenate([r.normal(scale=scale, size=mlp.N_PARAMS - 1), [0.3]])


def test_parameter_count_and_layout():
    assert mlp.N_PARAMS == 3 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4481
    t = np.arange(mlp.N_PARAMS, dtype=float)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(t)
    assert W1.shape == (64, 3) and W2.shape == (64, 64) and w3.shape == (64,)
    assert W1[1, 0] == 3 and b1[0] == 192 and W2[0, 1] == 257 and b3 == 4480
    assert np.array_equal(mlp.pack(W1, b1, W2, b2, w3, b3), t)


def test_silu_closed_forms():
    assert mlp.silu(0.0) == 0.0 and mlp.silu_d1(0.0) == 0.5 and mlp.silu_d2(0.0) == 0.5
    z = np.linspace(-6, 6, 25)
    h = 1e-5
    assert np.allclose((mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), mlp.silu_d1(z), atol=1e-9)
    assert np.allclose((mlp.silu_d1(z + h) - mlp.silu_d1(z - h)) / (2 * h), mlp.silu_d2(z), atol=1e-9)
    assert abs(mlp.silu(40.0) - 40.0) < 1e-12 and abs(mlp.silu(-40.0)) < 1e-12


def test_constant_network():
    """All weights zero but b3: y = b3 everywhere, zero input gradient."""
    t = np.zeros(mlp.N_PARAMS)
    t[-1] = 1.25
    y, u = mlp.forward(t, synth.rng(1).normal(size=(5, 3)))
    assert np.all(y == 1.25) and np.all(u == 0)


def test_single_path_network_closed_form():
    """One hidden path x0 -> unit 0 -> unit 0 -> y: y = w3 silu(W2 silu(W1 x0))."""
    t = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(t.copy())
    W1[0, 0], W2[0, 0], w3[0] = 0.7, -1.3, 2.0
    t = mlp.pack(W1, b1, W2, b2, w3, b3)
    x = np.array([[0.4, 9.0, -3.0]])
    y, u = mlp.forward(t, x)
    a = 0.4 * 0.7 / (1 + np.exp(-0.4 * 0.7))
    z2 = -1.3 * a
    assert abs(y[0] - 2.0 * z2 / (1 + np.exp(-z2))) < 1e-15
    assert u[0, 1] == 0 and u[0, 2] == 0


def test_input_gradient_matches_finite_differences():
    t = _theta(3)
    X = synth.rng(4).normal(size=(7, 3))
    _, u = mlp.forward(t, X)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (mlp.forward(t, X + e)[0] - mlp.forward(t, X - e)[0]) / (2 * h)
        assert np.allclose(fd, u[:, k], rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("lam", [0.0, 0.5])
def test_sobolev_weight_gradient_matches_finite_differences(lam):
    t = _theta(5)
    r = synth.rng(6)
    X, V, G = r.normal(size=(9, 3)), r.normal(size=9), r.normal(size=(9, 3))
    L, g = mlp.loss_grad(t, X, V, G, lam)
    assert abs(L - mlp.loss(t, X, V, G, lam)) <= 1e-13 * abs(L)
    # every parameter block, including the last bias
    idx = [0, 1, 100, 191, 192, 200, 255, 256, 300, 1000, 4351, 4352, 4400, 4415, 4416, 4450, 4479, 4480]
    h = 1e-6
    for i in idx:
        tp, tm = t.copy(), t.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, V, G, lam) - mlp.loss(tm, X, V, G, lam)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_first_adam_step_closed_form():
    """With bias correction the first step is -lr g / (|g| + eps)."""
    r = synth.rng(7)
    t, g = r.normal(size=50), r.normal(size=50)
    t1, m, v = mlp.adam(t, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    assert np.allclose(t1, t - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    t = np.array([3.0, -2.0])
    m = v = np.zeros(2)
    for k in range(1, 3001):
        t, m, v = mlp.adam(t, m, v, 2 * t, k, lr=1e-2)
    assert np.all(np.abs(t) < 1e-3)


def _bf16_brute(x):
    """Nearest bfloat16 by enumerating the two neighbours of x's FP32 value."""
    f = np.float32(x)
    u = int(np.array([f]).view(np.uint32)[0])
    lo = u & 0xFFFF0000
    hi = lo + 0x10000
    vlo = float(np.array([lo], np.uint32).view(np.float32)[0])
    vhi = float(np.array([hi], np.uint32).view(np.float32)[0])
    dlo, dhi = abs(float(f) - vlo), abs(vhi - float(f))
    if dlo < dhi:
        return vlo
    if dhi < dlo:
        return vhi
    return vlo if ((lo >> 16) & 1) == 0 else vhi


def test_bf16_rounding():
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1 + 2 ** -8) == 1.0                      # tie -> even
    assert mlp.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6           # tie -> even (up)
    assert mlp.bf16_round(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7    # above the tie
    assert mlp.bf16_round(-(1 + 2 ** -8 + 2 ** -20)) == -(1 + 2 ** -7)
    xs = synth.rng(8).normal(scale=3.0, size=400)
    got = mlp.bf16_round(xs)
    assert all(got[i] == _bf16_brute(xs[i]) for i in range(xs.size))


def test_surrogate_bias_normalisation():
    """V_nn = Vs y((xi - mu) inv_s) + Vm, chain rule through the affine map."""
    t = _theta(9)
    norm = (np.array([1.0, -2.0, 0.5]), np.array([2.0, 0.5, 4.0]), 3.0, 7.0)
    xi = synth.rng(10).normal(size=(4, 2))
    V, dV = mlp.bias(t, norm, xi)
    h = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (mlp.bias(t, norm, xi + e)[0] - mlp.bias(t, norm, xi - e)[0]) / (2 * h)
        assert np.allclose(fd, dV[:, k], rtol=1e-6, atol=1e-7)
    X = np.zeros((4, 3))
    X[:, :2] = (xi - norm[0][:2]) * norm[1][:2]
    assert np.allclose(V, 7.0 * mlp.forward(t, X)[0] + 3.0, rtol=1e-15)
