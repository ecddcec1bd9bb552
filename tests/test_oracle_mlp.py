"""Pin of the FP64 MLP reference: its backward pass against central finite
differences of its own loss (a dropped term, a transposed weight or a wrong
ReLU mask changes the gradient by O(1) and fails)."""
import numpy as np

from oracle import mlp


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [(7, 4), (9, 7), (6, 9), (5, 6)]
    params = [(rng.standard_normal(s) * 0.7, rng.standard_normal(s[0]) * 0.1) for s in sizes]
    x = rng.standard_normal((11, 4))
    t = rng.standard_normal((11, 5))
    used = 4
    grads = mlp.backward(params, mlp.forward(params, x), t, used)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in [tuple(rng.integers(0, n) for n in arr.shape) for _ in range(6)]:
                old = arr[idx]
                arr[idx] = old + eps
                fp = mlp.mse(mlp.forward(params, x)[-1], t, used)
                arr[idx] = old - eps
                fm = mlp.mse(mlp.forward(params, x)[-1], t, used)
                arr[idx] = old
                fd = (fp - fm) / (2 * eps)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, g[idx])
    # the unused output column gets no gradient
    assert np.all(grads[-1][0][used:] == 0) and np.all(grads[-1][1][used:] == 0)


def test_mlp_forward_matches_library_linear_layers():
    # the forward pass against torch's CPU linear layers in FP64 (y = x W^T + b,
    # ReLU after every layer but the last): a library routine, not a retyping
    import torch
    rng = np.random.default_rng(1)
    sizes = [(16, 4), (12, 16), (12, 12), (5, 12)]
    params = [(rng.standard_normal(s) * 0.5, rng.standard_normal(s[0]) * 0.2) for s in sizes]
    x = rng.standard_normal((9, 4))
    acts = mlp.forward(params, x)
    h = torch.from_numpy(x)
    for l, (W, b) in enumerate(params):
        h = torch.nn.functional.linear(h, torch.from_numpy(W), torch.from_numpy(b))
        if l < len(params) - 1:
            h = torch.relu(h)
        np.testing.assert_allclose(acts[l + 1], h.numpy(), rtol=1e-13, atol=1e-14)
