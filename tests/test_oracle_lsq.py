"""Pins of the oracle's least squares over the join (Section 1: the closed-form
solution of linear regression through QR), none of which re-calls lstsq."""
import numpy as np

import oracle


def _tiny_join(A, kA, B, kB):
    """J by explicit loops (independent of the oracle's materialisation)."""
    rows = []
    for i in range(len(kA)):
        for j in range(len(kB)):
            if kA[i] == kB[j]:
                rows.append(np.concatenate([A[i], B[j]]))
    return np.array(rows)


def test_exact_fit_recovers_the_coefficients():
    """y = B_x w exactly: beta = (0 for A's columns, w for B's), residual 0."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((60, 3))
    kA = rng.integers(0, 8, 60).astype(np.int32)
    Bx = rng.standard_normal((50, 2))
    w = np.array([1.5, -0.25])
    B = np.column_stack([Bx, Bx @ w])
    kB = rng.integers(0, 8, 50).astype(np.int32)
    beta, res = oracle.join_least_squares(A, kA, B, kB)
    assert np.allclose(beta, [0, 0, 0, 1.5, -0.25], atol=1e-10)
    assert res < 1e-9


def test_normal_equations_on_a_tiny_join():
    """beta solves J_x^T J_x beta = J_x^T y (J from explicit loops)."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((7, 2))
    kA = np.array([0, 1, 1, 2, 2, 2, 3], np.int32)
    B = rng.standard_normal((6, 3))
    kB = np.array([1, 2, 2, 0, 3, 3], np.int32)
    J = _tiny_join(A, kA, B, kB)
    X, y = J[:, :-1], J[:, -1]
    expect = np.linalg.solve(X.T @ X, X.T @ y)
    beta, res = oracle.join_least_squares(A, kA, B, kB)
    assert np.allclose(beta, expect, rtol=1e-10, atol=1e-12)
    # Pythagoras: y splits into its projection and the residual
    assert np.isclose(np.dot(y, y), np.dot(X @ beta, X @ beta) + res * res, rtol=1e-10)
