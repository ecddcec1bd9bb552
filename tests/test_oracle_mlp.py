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


def test_mlp_rounding_hooks_match_autograd_with_the_same_rounding_points():
    # the hooked chain rule against torch autograd in FP64: the hidden
    # activations are rounded in the forward pass with a straight-through
    # gradient, and a hook rounds the gradient that reaches each matmul output
    # (so the weight gradient and the back-propagated gradient see the rounded
    # value while the bias, added after the matmul, sums the unrounded one)
    import torch
    rng = np.random.default_rng(2)
    sizes = [(16, 4), (12, 16), (12, 12), (5, 12)]
    params = [(rng.standard_normal(s) * 0.5, rng.standard_normal(s[0]) * 0.2) for s in sizes]
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal((9, 5))
    used = 4

    # a relative rounding to 4 significant bits (BF16 keeps 8): coarse enough
    # to move every value, and like BF16 it keeps positive values positive
    def rnd(a):
        m, e = np.frexp(np.asarray(a, np.float64))
        return np.ldexp(np.round(m * 16.0) / 16.0, e)

    def trnd(a):
        return torch.from_numpy(rnd(a.detach().numpy()))

    acts = mlp.forward(params, x, act_round=rnd)
    grads = mlp.backward(params, acts, t, used, grad_round=rnd)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True))
          for W, b in params]
    h = torch.from_numpy(x)
    for l, (W, b) in enumerate(tp):
        mm = h @ W.T
        mm.register_hook(trnd)
        z = mm + b
        if l < len(tp) - 1:
            a = torch.relu(z)
            h = a + (trnd(a) - a).detach()
        else:
            h = z
    loss = ((h[:, :used] - torch.from_numpy(t[:, :used])) ** 2).mean()
    loss.backward()
    np.testing.assert_allclose(acts[-1], h.detach().numpy(), rtol=1e-13, atol=1e-14)
    for l, (W, b) in enumerate(tp):
        np.testing.assert_allclose(grads[l][0], W.grad.numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(grads[l][1], b.grad.numpy(), rtol=1e-12, atol=1e-14)
    # and the rounding does change the gradients (the hooks are not no-ops)
    exact = mlp.backward(params, mlp.forward(params, x), t, used)
    assert np.abs(exact[0][0] - grads[0][0]).max() > 1e-3
