"""FP64 oracle of the filter-parameter predictor: a 64-128-128-3 perceptron
with GELU activations, mean-squared-error loss and Adam updates.

The paper has no learned component (its Sec. 2 chooses intervals from Lehmann
intervals and grows the degree as they shrink); this network maps kernel-
polynomial density-of-states moments (Sec. 4.1) and the target window to the
degree constant and window margins of the interval heuristic.  Definitions:

    gelu(x)   = x/2 (1 + erf(x / sqrt 2))            (Hendrycks & Gimpel 2016)
    gelu'(x)  = (1 + erf(x / sqrt 2))/2 + x phi(x),   phi = standard normal pdf
    h1 = gelu(x W1 + b1), h2 = gelu(h1 W2 + b2), y = h2 W3 + b3
    loss = mean over the batch and the 3 outputs of (y - t)^2
    Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    p <- p - lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)

Parameters are one flat vector in the order W1 (64x128, row-major), b1, W2
(128x128), b2, W3 (128x3), b3 -- 25219 numbers.
"""
import numpy as np
from scipy.special import erf

SIZES = [(64, 128), (128, 128), (128, 3)]
N_PARAMS = sum(i * o + o for i, o in SIZES)


def unpack(p):
    out, o = [], 0
    for i, n in SIZES:
        W = p[o:o + i * n].reshape(i, n); o += i * n
        b = p[o:o + n]; o += n
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def init(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in SIZES:
        parts.append(rng.standard_normal(i * o) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def forward(p, X):
    (W1, b1), (W2, b2), (W3, b3) = unpack(p)
    z1 = X @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, T):
    y, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    r = y - T
    loss = np.mean(r * r)
    dy = 2.0 * r / (B * 3)
    (W1, b1), (W2, b2), (W3, b3) = unpack(p)
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dz2 = (dy @ W3.T) * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(p, g, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
