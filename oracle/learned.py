"""Learned proposal correction: a small network that shifts each conditional logit.

Test infrastructure: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use this module; the CUDA path never imports it.

The paper's sampler (Sec. 3.3, Eq. 5, Eq. 9) draws spin i with probability
sigmoid(l_i), l_i the conditional logit that the chi-MPS environments give.
This extension (not in the paper) draws it with sigmoid(l_i + Delta_i) where
Delta_i = f_theta(x_i) is a 7 -> 64 -> 64 -> 1 network of local features. The
draw and log q (Eq. 9) both use the corrected logit, so q stays a normalised
distribution over configurations and the independence Metropolis-Hastings
test (Eq. 10) keeps sampling the Boltzmann distribution exactly, whatever
theta is.

Features of site i = (r, c), in this order (0 where the neighbour is absent):

    x0 = l_i clamped to [-32, 32]  conditional logit of the chi-MPS (Eq. 5)
    x1 = 2 beta Jv[r-1, c] s(r-1, c)   field of the spin above
    x2 = beta Jh[r, c-1] s(r, c-1)     field of the spin on the left
    x3 = Jh[r, c]                  coupling to the right (spin not yet drawn)
    x4 = Jv[r, c]                  coupling below (row not yet drawn)
    x5 = s(r-1, c+1)               spin above-right, +-1
    x6 = beta

Network (weights and biases stored as bfloat16, arithmetic in float32 on the
GPU, float64 here): the features are rounded to bfloat16, then
h1 = g(W1 x + b1) rounded to bfloat16, h2 = g(W2 h1 + b2), Delta = w3 . h2 + b3,
with g the smooth ReLU: 0 for z <= -1, (z + 1)^2 / 4 for |z| < 1, z for
z >= 1 (continuous with a continuous first derivative).

Training loss: per-site binary cross entropy of sigmoid(x0 + Delta) against a
target probability p (the conditional of a larger chi on the same
configuration), mean over examples. Backward treats the bfloat16 roundings as
the identity (straight-through). Optimiser: Adam (Kingma & Ba, 2015) with
bias correction.

Parameter vector layout (element offsets, the same for the float32 master copy
and the bfloat16 copy): W1 (64 x 16, output-major, input columns 7..15 zero),
b1 (64), W2 (64 x 64, output-major), b2 (64), w3 (64), b3 (1), 7 zeros.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 7
IN_PAD = 16
HIDDEN = 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + HIDDEN * IN_PAD
OFF_W2 = OFF_B1 + HIDDEN
OFF_B2 = OFF_W2 + HIDDEN * HIDDEN
OFF_W3 = OFF_B2 + HIDDEN
OFF_B3 = OFF_W3 + HIDDEN
N_PARAM = OFF_B3 + 8
LOGIT_CLAMP = 32.0


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32; returned as float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of
    a float32, so rounding is done on the low 16 bits of the float32 pattern.
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def act(z):
    """Smooth ReLU g(z)."""
    z = np.asarray(z, dtype=np.float64)
    return np.where(z >= 1.0, z, np.where(z <= -1.0, 0.0, 0.25 * (z + 1.0) ** 2))


def act_grad(z):
    """g'(z)."""
    z = np.asarray(z, dtype=np.float64)
    return np.where(z >= 1.0, 1.0, np.where(z <= -1.0, 0.0, 0.5 * (z + 1.0)))


def unpack(theta):
    """Parameter vector -> (W1 (64, 7), b1, W2 (64, 64), b2, w3, b3)."""
    t = np.asarray(theta, dtype=np.float64)
    W1 = t[OFF_W1:OFF_B1].reshape(HIDDEN, IN_PAD)[:, :N_FEAT]
    b1 = t[OFF_B1:OFF_W2]
    W2 = t[OFF_W2:OFF_B2].reshape(HIDDEN, HIDDEN)
    b2 = t[OFF_B2:OFF_W3]
    w3 = t[OFF_W3:OFF_B3]
    b3 = t[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    t = np.zeros(N_PARAM)
    t[OFF_W1:OFF_B1].reshape(HIDDEN, IN_PAD)[:, :N_FEAT] = W1
    t[OFF_B1:OFF_W2] = b1
    t[OFF_W2:OFF_B2] = np.asarray(W2).reshape(-1)
    t[OFF_B2:OFF_W3] = b2
    t[OFF_W3:OFF_B3] = w3
    t[OFF_B3] = b3
    return t


def init_params(seed: int):
    """Seeded start: W1, W2 ~ N(0, 1/fan_in) and zero w3, b3, so Delta = 0 (plain TNMC)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((HIDDEN, N_FEAT)) / np.sqrt(N_FEAT)
    W2 = rng.standard_normal((HIDDEN, HIDDEN)) / np.sqrt(HIDDEN)
    return pack(W1, np.zeros(HIDDEN), W2, np.zeros(HIDDEN), np.zeros(HIDDEN), 0.0).astype(np.float32)


def features(Jh, Jv, beta, sigma, logits):
    """Features of every site of S configurations: (S, L*L, 7) float64.

    sigma : (S, L, L) spin bits (1 = +1); logits : (S, L*L) uncorrected conditional logits.
    """
    sigma = np.asarray(sigma)
    S, L, _ = sigma.shape
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    s = 2.0 * sigma.astype(np.float64) - 1.0
    X = np.zeros((S, L, L, N_FEAT))
    X[..., 0] = np.clip(np.asarray(logits, dtype=np.float64).reshape(S, L, L), -LOGIT_CLAMP, LOGIT_CLAMP)
    if L > 1:
        X[:, 1:, :, 1] = 2.0 * beta * Jv[None, :, :] * s[:, :-1, :]
        X[:, :, 1:, 2] = beta * Jh[None, :, :] * s[:, :, :-1]
        X[:, :, :-1, 3] = Jh[None, :, :]
        X[:, :-1, :, 4] = Jv[None, :, :]
        X[:, 1:, :-1, 5] = s[:, :-1, 1:]
    X[..., 6] = beta
    return X.reshape(S, L * L, N_FEAT)


def forward(theta, X, rounding=True):
    """Delta for each row of X (..., 7). Returns (Delta, cache for backward)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    x = to_bf16(X) if rounding else np.asarray(X, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = act(z1)
    h1r = to_bf16(h1) if rounding else h1
    z2 = h1r @ W2.T + b2
    h2 = act(z2)
    delta = h2 @ w3 + b3
    return delta, (x, z1, h1r, z2, h2)


def loss(theta, X, target_p, rounding=True):
    """Mean binary cross entropy of sigmoid(x0 + Delta) against target_p."""
    delta, _ = forward(theta, X, rounding)
    z = np.asarray(X, dtype=np.float64)[..., 0] + delta
    lp = -(np.maximum(-z, 0.0) + np.log1p(np.exp(-np.abs(z))))     # log sigmoid(z)
    lm = -(np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z))))      # log sigmoid(-z)
    p = np.asarray(target_p, dtype=np.float64)
    return float(np.mean(-(p * lp + (1.0 - p) * lm)))


def grad(theta, X, target_p, rounding=True):
    """(loss, d loss / d theta) by backpropagation (straight-through over the roundings)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_FEAT)
    p = np.asarray(target_p, dtype=np.float64).reshape(-1)
    N = X.shape[0]
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    delta, (x, z1, h1r, z2, h2) = forward(theta, X, rounding)
    z = X[:, 0] + delta
    sig = np.exp(-(np.maximum(-z, 0.0) + np.log1p(np.exp(-np.abs(z)))))
    dz = (sig - p) / N                          # d loss / d Delta per example
    g_b3 = dz.sum()
    g_w3 = h2.T @ dz
    dz2 = np.outer(dz, w3) * act_grad(z2)
    g_W2 = dz2.T @ h1r
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * act_grad(z1)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    return loss(theta, X, p, rounding), pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1). Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


class Correction:
    """Delta_i for the oracle sampler: features of the current site, then the network.

    theta must hold the bfloat16 values the GPU uses (``to_bf16`` of the master copy).
    """

    def __init__(self, theta, Jh, Jv, beta):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.Jh, self.Jv, self.beta = Jh, Jv, float(beta)

    def site_features(self, sigma, r, c, logit):
        """Features of site (r, c) for all S chains; sigma holds the spins drawn so far."""
        S, L, _ = sigma.shape
        x = np.zeros((S, N_FEAT))
        x[:, 0] = np.clip(logit, -LOGIT_CLAMP, LOGIT_CLAMP)
        if r > 0:
            x[:, 1] = 2.0 * self.beta * float(self.Jv[r - 1, c]) * (2.0 * sigma[:, r - 1, c] - 1.0)
            if c < L - 1:
                x[:, 5] = 2.0 * sigma[:, r - 1, c + 1] - 1.0
        if c > 0:
            x[:, 2] = self.beta * float(self.Jh[r, c - 1]) * (2.0 * sigma[:, r, c - 1] - 1.0)
        if c < L - 1:
            x[:, 3] = float(self.Jh[r, c])
        if r < L - 1:
            x[:, 4] = float(self.Jv[r, c])
        x[:, 6] = self.beta
        return x

    def __call__(self, sigma, r, c, logit):
        delta, _ = forward(self.theta, self.site_features(sigma, r, c, logit))
        return delta
