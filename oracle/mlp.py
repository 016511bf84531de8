"""FP64 CPU oracle of the MLP surrogate of the hills sum.

TEST INFRASTRUCTURE ONLY (same rule as the rest of `oracle/`): called by
`tests/` and nothing else; shares no code with the CUDA library.

The paper points to neural-network bias representations (its ANN and FUNN
methods, Secs. 2.1.7 and 2.1.8) but prints no network for metadynamics; the surrogate
here is a plain 3 -> 64 -> 64 -> 1 perceptron with SiLU activations,
z -> z * sigmoid(z), written from those definitions:

    z1 = W1 x + b1,  a1 = silu(z1)
    z2 = W2 a1 + b2, a2 = silu(z2)
    y  = w3 . a2 + b3

Parameters are one flat vector of 4481 numbers in the order
W1 [64][3] (row j = hidden unit j), b1 [64], W2 [64][64] (row i = output
unit i), b2 [64], w3 [64], b3.  The GPU keeps an FP32 master copy and runs
the network with the weights rounded to bfloat16 (round to nearest, ties
to even); `bf16_round` emulates that rounding so that the oracle evaluates
the very same network in FP64.

Training loss (Sobolev: values and input gradients), over a batch of B
samples (x_b, V_b, G_b):

    L = 1/B sum_b [ (y(x_b) - V_b)^2 + lam |grad_x y(x_b) - G_b|^2 ]

Its weight gradient needs the derivative of grad_x y with respect to the
weights (double backward); `loss_grad` writes that chain rule out term by
term.  Adam (Kingma & Ba 2015, with bias correction) updates the master
copy.

The surrogate of the bias maps a CV point xi to y through a fixed affine
normalisation: V_nn(xi) = Vs * y((xi - mu) * inv_s) + Vm and
dV_nn/dxi_k = Vs * inv_s_k * dy/dx_k.
"""
from __future__ import annotations

import numpy as np

H1, H2, DIN = 64, 64, 3
N_PARAMS = H1 * DIN + H1 + H2 * H1 + H2 + H2 + 1  # 4481

_O_W1 = 0
_O_B1 = _O_W1 + H1 * DIN
_O_W2 = _O_B1 + H1
_O_B2 = _O_W2 + H2 * H1
_O_W3 = _O_B2 + H2
_O_B3 = _O_W3 + H2


def unpack(theta):
    t = np.asarray(theta, dtype=np.float64)
    assert t.shape == (N_PARAMS,)
    return (t[_O_W1:_O_B1].reshape(H1, DIN), t[_O_B1:_O_W2], t[_O_W2:_O_B2].reshape(H2, H1), t[_O_B2:_O_W3],
            t[_O_W3:_O_B3], t[_O_B3])


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, np.atleast_1d(b3)]).astype(np.float64)


def bf16_round(a):
    """FP32 value of `a` rounded to bfloat16 (8 exponent, 7 stored
    mantissa bits), nearest with ties to even, returned as float64.  The
    input is first rounded to FP32, as the GPU's master copy is FP32."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_d1(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def silu_d2(z):
    s = sigmoid(z)
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


def forward(theta, X):
    """y [B] and its input gradient grad_x y [B][3] at inputs X [B][3]."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    z1 = X @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    y = a2 @ w3 + b3
    g2 = silu_d1(z2) * w3          # dy/dz2
    g1 = silu_d1(z1) * (g2 @ W2)   # dy/dz1
    return y, g1 @ W1


def loss(theta, X, V, G, lam):
    y, u = forward(theta, X)
    return float(np.mean((y - V) ** 2) + lam * np.mean(np.sum((u - G) ** 2, axis=1)))


def loss_grad(theta, X, V, G, lam):
    """(L, dL/dtheta [4481]) of the Sobolev loss, by the chain rule through
    the forward pass and through the input gradient."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    B = X.shape[0]
    z1 = X @ W1.T + b1
    a1, d1, dd1 = silu(z1), silu_d1(z1), silu_d2(z1)
    z2 = a1 @ W2.T + b2
    a2, d2, dd2 = silu(z2), silu_d1(z2), silu_d2(z2)
    y = a2 @ w3 + b3
    g2 = d2 * w3            # [B][64]
    h1 = g2 @ W2            # [B][64]  W2^T g2
    g1 = d1 * h1
    u = g1 @ W1             # [B][3]   grad_x y
    r = y - V
    e = u - G
    L = float(np.mean(r ** 2) + lam * np.mean(np.sum(e ** 2, axis=1)))
    dy = 2.0 * r / B                       # upstream of y
    du = 2.0 * lam * e / B                 # upstream of grad_x y
    # through u = W1^T g1, g1 = d1 * h1, h1 = W2^T g2, g2 = d2 * w3
    gb1 = du @ W1.T                        # upstream of g1 [B][64]
    hb1 = gb1 * d1                         # upstream of h1
    gb2 = hb1 @ W2.T                       # upstream of g2
    # z2 receives the value path and the d2 = silu'(z2) path
    zb2 = dy[:, None] * w3 * d2 + gb2 * w3 * dd2
    dw3 = dy @ a2 + np.sum(gb2 * d2, axis=0)
    db3 = np.sum(dy)
    dW2 = zb2.T @ a1 + g2.T @ hb1
    db2 = zb2.sum(axis=0)
    ab1 = zb2 @ W2
    zb1 = ab1 * d1 + gb1 * h1 * dd1
    dW1 = zb1.T @ X + g1.T @ du
    db1 = zb1.sum(axis=0)
    return L, pack(dW1, db1, dW2, db2, dw3, db3)


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t = 1, 2, ...): returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bias(theta, norm, xi):
    """Surrogate bias V_nn and dV_nn/dxi at CV points xi [P][d] (d <= 3),
    norm = (mu[3], inv_s[3], Vm, Vs), or the same 8 numbers flat; unused
    inputs are 0."""
    if np.ndim(norm[0]) == 0:
        norm = (norm[0:3], norm[3:6], norm[6], norm[7])
    mu, inv_s, Vm, Vs = np.asarray(norm[0], float), np.asarray(norm[1], float), float(norm[2]), float(norm[3])
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    d = xi.shape[1]
    X = np.zeros((xi.shape[0], DIN))
    X[:, :d] = (xi - mu[:d]) * inv_s[:d]
    y, u = forward(theta, X)
    return Vs * y + Vm, Vs * u[:, :d] * inv_s[:d]
