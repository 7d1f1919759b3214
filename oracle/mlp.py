"""FP64 oracle of the learned-lambda network (test infrastructure only).

The network reads 36 features from the first 12 steps of c-LSQR and predicts
the Tikhonov parameter and the stopping index. It replaces the per-iteration
GCV search and the L-curve / k_opt choice of §3.3, with GCV kept as fallback.
The paper has no such network; its architecture is fixed here:
  x (36) -> GELU(x W1 + b1) (64) -> GELU(h1 W2 + b2) (64) -> h2 W3 + b3 (2)
with GELU(z) = z/2 (1 + erf(z / sqrt 2)) and the loss
  L = (1 / 2B) sum_b sum_j (out_bj - t_bj)^2
over a batch of B samples. Weights are row-major (in x out). The features of a
solve (log-normalised alpha, beta and |phibar|) are defined by `features` below.

Plain NumPy with hand-written backward; pinned by finite differences.
"""
import math

import numpy as np

SIZES = (36, 64, 64, 2)
NFEAT_STEPS = 12


def gelu(z):
    return 0.5 * z * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def unpack(theta):
    """Split a flat parameter vector into W1, b1, W2, b2, W3, b3 (this order)."""
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        out.append(theta[o:o + a * b].reshape(a, b))
        o += a * b
        out.append(theta[o:o + b])
        o += b
    return out


def nparams():
    return sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64)
    z1 = X @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    out = h2 @ W3 + b3
    return out, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T):
    """L and dL/dtheta (flat, same order as theta)."""
    out, (X, z1, h1, z2, h2) = forward(theta, X)
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64))
    B = X.shape[0]
    d = (out - np.asarray(T, np.float64)) / B
    L = 0.5 * float(np.sum((out - T) ** 2)) / B
    gW3 = h2.T @ d
    gb3 = d.sum(0)
    dz2 = (d @ W3.T) * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1). Returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(alpha, beta, phibar):
    """36 inputs from the first 12 c-LSQR steps (§3.3 quantities):
    log(alpha_i / beta_1), log(beta_{i+1} / beta_1), log(|phibar_{i+1}| / beta_1),
    for i = 1..12; alpha[0] = alpha_1, beta[0] = beta_1, phibar[i-1] = |phibar_{i+1}|."""
    b1 = beta[0]
    a = np.log(np.asarray(alpha[:NFEAT_STEPS], np.float64) / b1)
    b = np.log(np.asarray(beta[1:NFEAT_STEPS + 1], np.float64) / b1)
    p = np.log(np.abs(np.asarray(phibar[:NFEAT_STEPS], np.float64)) / b1)
    return np.concatenate([a, b, p])
