"""FP64 reference of the kernel-generator MLP -- TEST INFRASTRUCTURE ONLY.

Four linear layers with ReLU after the first three, y = W4 relu(W3 relu(W2
relu(W1 x + b1) + b2) + b3) + b4, mean-squared error over the first `used`
output columns, and its gradients by the chain rule, in numpy FP64.  Pinned
against central finite differences.
"""
import numpy as np


def forward(params, x):
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    for l, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        h = np.maximum(z, 0.0) if l < len(params) - 1 else z
        acts.append(h)
    return acts  # [x, h1, h2, h3, y]


def mse(y, target, used):
    d = y[:, :used] - target[:, :used]
    return float(np.mean(d * d))


def backward(params, acts, target, used):
    """Gradients of mse(...) with respect to every (W, b)."""
    y = acts[-1]
    rows = y.shape[0]
    g = np.zeros_like(y)
    g[:, :used] = 2.0 * (y[:, :used] - target[:, :used]) / (rows * used)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (g.T @ acts[l], g.sum(axis=0))
        if l > 0:
            g = (g @ W) * (acts[l] > 0)
    return grads
