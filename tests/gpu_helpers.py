"""Shared helpers of the GPU parity tests (imported only by tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64) if t.dtype in (
        torch.float16, torch.bfloat16) else t.detach().cpu().numpy()


def dot64(a, b):
    return float(np.dot(np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()))


def dot_test(hx, y, x, hty, tol=1e-6):
    """Adjoint dot test: |<Hx, y> - <x, H^T y>| <= tol * ||Hx|| ||y||."""
    lhs, rhs = dot64(hx, y), dot64(x, hty)
    scale = np.linalg.norm(np.asarray(hx, np.float64)) * np.linalg.norm(np.asarray(y, np.float64))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)
