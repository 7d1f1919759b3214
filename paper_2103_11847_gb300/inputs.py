"""Seeded synthetic inputs shaped like the experiments of §4 (arXiv 2103.11847).

This module holds no arithmetic of the method: it builds the blur factors,
clean images and videos, and raw Gaussian noise. Forming the observation
C = M(X_true) + N needs the operator, so callers do that step themselves
(the CUDA library in the benchmark, the FP64 oracle in the tests); the noise
scaling of §4 is ``scale_noise`` below.

Layout: every tensor is a float64 array of shape (n3, rows, cols), slice k is
the frontal slice X(:, :, k).

Stand-ins (the paper's test images are not available):
  * image(n, rng): per channel a smooth field (offset + two ramps + a separable
    sinusoid) with 20 constant axis-aligned rectangles painted over it, clipped
    to [0, 1].
  * video(n, frames, rng): one smooth grey field plus three rectangles moving
    at constant sub-2-pixel-per-frame velocities, clipped to [0, 1].
  * gaussian_blur(n, sigma, r): §4's banded Gaussian Toeplitz matrix
    a_{kl} = exp(-(k-l)^2 / (2 sigma^2)) / (sigma sqrt(2 pi)) for |k-l| <= r,
    divided by the interior row sum so that an interior row sums to one
    (one scalar per matrix, which keeps the matrix symmetric Toeplitz).
  * noise: i.i.d. N(0, 1) entries; scale_noise gives exactly the relative level
    nu = ||N||_F / ||C_hat||_F of §4.
"""
import math

import numpy as np


def rng_for(seed):
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_blur(n, sigma, r):
    d = np.arange(-r, r + 1)
    pdf = np.exp(-(d.astype(np.float64) ** 2) / (2.0 * sigma * sigma)) / (sigma * math.sqrt(2.0 * math.pi))
    norm = pdf.sum()
    A = np.zeros((n, n))
    for k in range(n):
        for off, w in zip(d, pdf):
            l = k + off
            if 0 <= l < n:
                A[k, l] = w / norm
    return A


def image(n, rng, channels=3, rects=20):
    i = np.arange(n)[:, None] / n
    j = np.arange(n)[None, :] / n
    X = np.empty((channels, n, n))
    for c in range(channels):
        a = rng.uniform(0.1, 0.5)
        b, d = rng.uniform(-0.3, 0.3, size=2)
        e = rng.uniform(0.0, 0.2)
        f, g = rng.integers(1, 4, size=2)
        X[c] = a + b * i + d * j + e * np.sin(2 * np.pi * f * i) * np.cos(2 * np.pi * g * j)
    for _ in range(rects):
        h = int(rng.integers(max(1, n // 20), max(2, (2 * n) // 5) + 1))
        w = int(rng.integers(max(1, n // 20), max(2, (2 * n) // 5) + 1))
        r0 = int(rng.integers(0, n - h + 1))
        c0 = int(rng.integers(0, n - w + 1))
        val = rng.uniform(0.0, 1.0, size=channels)
        X[:, r0:r0 + h, c0:c0 + w] = val[:, None, None]
    return np.clip(X, 0.0, 1.0)


def video(n, frames, rng, movers=3):
    i = np.arange(n)[:, None] / n
    j = np.arange(n)[None, :] / n
    a = rng.uniform(0.1, 0.4)
    b, d = rng.uniform(-0.2, 0.2, size=2)
    e = rng.uniform(0.0, 0.2)
    bg = a + b * i + d * j + e * np.sin(2 * np.pi * i) * np.cos(2 * np.pi * 2 * j)
    X = np.broadcast_to(bg, (frames, n, n)).copy()
    for _ in range(movers):
        h = int(rng.integers(n // 16, n // 4 + 1))
        w = int(rng.integers(n // 16, n // 4 + 1))
        y0 = rng.uniform(0, n - h)
        x0 = rng.uniform(0, n - w)
        vy, vx = rng.uniform(-2.0, 2.0, size=2)
        val = rng.uniform(0.3, 1.0)
        for t in range(frames):
            yy = int(round(min(max(y0 + vy * t, 0), n - h)))
            xx = int(round(min(max(x0 + vx * t, 0), n - w)))
            X[t, yy:yy + h, xx:xx + w] = val
    return np.clip(X, 0.0, 1.0)


def gaussian_noise(shape, rng):
    return rng.standard_normal(shape)


def scale_noise(C_clean, G, nu):
    """C_clean + N with N = nu ||C_clean||_F G / ||G||_F (§4's noise level)."""
    return C_clean + nu * np.linalg.norm(C_clean.ravel()) / np.linalg.norm(G.ravel()) * G


# ---------------------------------------------------------------- workloads --
# Each returns dict(A, B, X_true, G, nu, name) in float64; B is None for the
# one-sided operator A *c X.

def colour_deblur(n=64, sigma=2.0, r=4, weights=(1.0, 0.7, 0.4), nu=1e-3, seed=0):
    """Colour image (n x n x 3), one-sided: slice k of A is weights[k] G_{sigma,r}."""
    rng = rng_for(seed)
    G = gaussian_blur(n, sigma, r)
    A = np.stack([w * G for w in weights])
    X = image(n, rng, channels=len(weights))
    return dict(A=A, B=None, X_true=X, G=gaussian_noise(X.shape, rng), nu=nu,
                name=f"colour_deblur_{n}x{n}x{len(weights)}")


def two_sided_deblur(n=256, n3=3, sigma_a=3.0, sigma_b=2.0, r=8, nu=1e-3, seed=1):
    """Two-sided A *c X *c B (n x n x n3): every slice of A is G_{sigma_a,r},
    every slice of B is G_{sigma_b,r}."""
    rng = rng_for(seed)
    GA = gaussian_blur(n, sigma_a, r)
    GB = gaussian_blur(n, sigma_b, r)
    A = np.stack([GA] * n3)
    B = np.stack([GB] * n3)
    X = image(n, rng, channels=n3)
    return dict(A=A, B=B, X_true=X, G=gaussian_noise(X.shape, rng), nu=nu,
                name=f"two_sided_{n}x{n}x{n3}")


def paper_deblur(n=256, nu=1e-3, sigma=4.0, r=6, weights=(1.0, 0.7, 0.7), seed=7):
    """Paper-shaped colour deblur, the shapes of Tables 1-4 (§4): two-sided
    A *c X *c B (n x n x 3) with the within-channel Gaussian G_{4,6} on both
    sides. Slice k of A is weights[k] G (the eigenvalues 1, 0.7, 0.7 of the
    paper's cross-channel matrix, placed on the slices directly), every slice
    of B is G."""
    rng = rng_for(seed)
    G = gaussian_blur(n, sigma, r)
    A = np.stack([w * G for w in weights])
    B = np.stack([G] * len(weights))
    X = image(n, rng, channels=len(weights))
    return dict(A=A, B=B, X_true=X, G=gaussian_noise(X.shape, rng), nu=nu,
                name=f"paper_{n}x{n}x{len(weights)}")


def video_deblur(n=512, frames=64, sigma0=1.5, sigma1=3.5, nu=1e-3, seed=2):
    """Video (n x n x frames), one-sided: frame k of A is G_{s_k, ceil(3 s_k)}
    with s_k linear from sigma0 to sigma1."""
    rng = rng_for(seed)
    A = np.empty((frames, n, n))
    for k in range(frames):
        s = sigma0 + (sigma1 - sigma0) * (k / max(frames - 1, 1))
        A[k] = gaussian_blur(n, s, int(math.ceil(3 * s)))
    X = video(n, frames, rng)
    return dict(A=A, B=None, X_true=X, G=gaussian_noise(X.shape, rng), nu=nu,
                name=f"video_{n}x{n}x{frames}")


def batch_sizes(count=128, lo=64, hi=512, step=32, seed=3):
    rng = rng_for(seed)
    return [int(v) for v in rng.integers(0, (hi - lo) // step + 1, size=count) * step + lo]


def batch_problem(index, n, seed=3):
    """Problem `index` of the uneven batch: n x n x 3 colour image, slice k of A
    is (1, 0.7, 0.4)[k] G_{sigma, ceil(3 sigma)}, sigma ~ U[1, 4],
    nu ~ U[1e-4, 1e-2]."""
    rng = rng_for(seed * 100003 + index)
    sigma = float(rng.uniform(1.0, 4.0))
    nu = float(rng.uniform(1e-4, 1e-2))
    G = gaussian_blur(n, sigma, int(math.ceil(3 * sigma)))
    A = np.stack([w * G for w in (1.0, 0.7, 0.4)])
    X = image(n, rng)
    return dict(A=A, B=None, X_true=X, G=gaussian_noise(X.shape, rng), nu=nu,
                sigma=sigma, name=f"batch[{index}]_{n}x{n}x3")


def random_problem(n1, n2, s, n3, two_sided=False, seed=0):
    """Dense random operator and operand for algebra tests (no structure)."""
    rng = rng_for(seed)
    A = rng.standard_normal((n3, n1, n2))
    B = rng.standard_normal((n3, s, s)) if two_sided else None
    X = rng.standard_normal((n3, n2, s))
    Y = rng.standard_normal((n3, n1, s))
    return dict(A=A, B=B, X=X, Y=Y)
