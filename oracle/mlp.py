"""FP64 reference of the kernel-generator MLP -- TEST INFRASTRUCTURE ONLY.

Four linear layers with ReLU after the first three, y = W4 relu(W3 relu(W2
relu(W1 x + b1) + b2) + b3) + b4, mean-squared error over the first `used`
output columns, and its gradients by the chain rule, in numpy FP64.  Pinned
against central finite differences and torch's FP64 linear layers.

Optional rounding hooks let a test apply a lower-precision implementation's
rounding points (a callable mapping an array to its rounded FP64 values)
without changing the arithmetic between them:
  act_round   applied to every hidden activation after the ReLU (the value
              the next layer multiplies);
  grad_round  applied to the output-side gradient of every layer before it
              multiplies the activations (weight gradient) and the weights
              (back-propagation); the bias gradient sums the unrounded one.
The ReLU mask of the backward pass is read from the stored activations, so
act_round must keep positive values positive (BF16 rounding does: it keeps
FP32's exponent range).  With no hooks the functions are the exact FP64
chain rule.
"""
import numpy as np


def forward(params, x, act_round=None):
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    for l, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if l < len(params) - 1:
            h = np.maximum(z, 0.0)
            if act_round is not None:
                h = act_round(h)
        else:
            h = z
        acts.append(h)
    return acts  # [x, h1, h2, h3, y]


def mse(y, target, used):
    d = y[:, :used] - target[:, :used]
    return float(np.mean(d * d))


def backward(params, acts, target, used, grad_round=None):
    """Gradients of mse(...) with respect to every (W, b)."""
    y = acts[-1]
    rows = y.shape[0]
    g = np.zeros_like(y)
    g[:, :used] = 2.0 * (y[:, :used] - target[:, :used]) / (rows * used)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        gq = g if grad_round is None else grad_round(g)
        grads[l] = (gq.T @ acts[l], g.sum(axis=0))
        if l > 0:
            g = (gq @ W) * (acts[l] > 0)
    return grads
