"""FP64 FISTA with an L1 prior -- TEST INFRASTRUCTURE ONLY.

The paper names deconvolution on its convolutional model as the model's use
(abstract, introduction, conclusion) without fixing an algorithm; this is the
textbook FISTA of Beck and Teboulle (2009) for
    min_x F(x) = 1/2 ||H x - b||^2 + lam ||x||_1,
written step by step in numpy with H and H^T passed in as callables.
"""
import numpy as np


def soft(z, t):
    """Proximal map of t ||.||_1 (soft thresholding)."""
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def objective(H, x, b, lam):
    r = H(x) - b
    return 0.5 * float(np.vdot(r, r)) + lam * float(np.abs(x).sum())


def fista(H, Ht, b, lam, L, iters, x0=None):
    x = np.zeros_like(Ht(b), dtype=np.float64) if x0 is None else np.array(x0, np.float64)
    y = x.copy()
    t = 1.0
    for _ in range(iters):
        g = Ht(H(y) - b)
        x_new = soft(y - g / L, lam / L)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        y = x_new + ((t - 1.0) / t_new) * (x_new - x)
        x, t = x_new, t_new
    return x


def power_iteration(H, Ht, v0, iters):
    """Largest eigenvalue of H^T H by the power method from v0."""
    v = np.array(v0, np.float64)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = Ht(H(v))
        lam = np.linalg.norm(w)
        v = w / lam
    return lam, v
