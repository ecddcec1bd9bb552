"""Pins of the FP64 FISTA oracle: the identity operator reduces one step to
soft thresholding; the power method matches numpy's eigensolver; the
solution matches scikit-learn's coordinate-descent Lasso; the objective gap
obeys the O(1/k^2) bound of FISTA."""
import numpy as np
import pytest

from oracle import fista as F


def test_identity_operator_one_step_is_soft_threshold():
    rng = np.random.default_rng(0)
    b = rng.standard_normal((16, 16))
    x = F.fista(lambda v: v, lambda v: v, b, lam=0.3, L=1.0, iters=1)
    ref = np.where(np.abs(b) > 0.3, b - 0.3 * np.sign(b), 0.0)
    np.testing.assert_array_equal(x, ref)


def test_power_iteration_matches_eigvalsh():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 30))
    lam, _ = F.power_iteration(lambda v: A @ v, lambda v: A.T @ v, rng.standard_normal(30), 300)
    assert lam == pytest.approx(np.linalg.eigvalsh(A.T @ A).max(), rel=1e-8)


def _problem(seed=2):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((60, 40))
    x_true = rng.standard_normal(40) * (rng.random(40) < 0.2)
    b = A @ x_true + 0.01 * rng.standard_normal(60)
    return A, b


def test_solution_matches_coordinate_descent_lasso():
    sk = pytest.importorskip("sklearn.linear_model")
    A, b = _problem()
    lam = 0.5
    L = np.linalg.eigvalsh(A.T @ A).max()
    x = F.fista(lambda v: A @ v, lambda v: A.T @ v, b, lam, L, 5000)
    # scikit-learn minimises 1/(2 n) ||b - A w||^2 + alpha ||w||_1
    ref = sk.Lasso(alpha=lam / A.shape[0], fit_intercept=False, tol=1e-14,
                   max_iter=200000).fit(A, b).coef_
    assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)


def test_objective_gap_obeys_fista_rate():
    A, b = _problem(3)
    lam = 0.2
    L = np.linalg.eigvalsh(A.T @ A).max()
    H, Ht = (lambda v: A @ v), (lambda v: A.T @ v)
    x_star = F.fista(H, Ht, b, lam, L, 20000)
    f_star = F.objective(H, x_star, b, lam)
    for k in (5, 20, 80):
        xk = F.fista(H, Ht, b, lam, L, k)
        gap = F.objective(H, xk, b, lam) - f_star
        assert -1e-9 <= gap <= 2 * L * np.linalg.norm(x_star) ** 2 / (k + 1) ** 2
