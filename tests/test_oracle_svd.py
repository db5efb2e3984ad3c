"""Pins of the oracle's singular vectors (oracle.jacobi_svd): the properties
that define V (orthonormal columns, ||R v_j|| = sigma_j, R v_j orthogonal to
R v_k), LAPACK's V where the values are separated (the vectors are unique up
to sign there), the closed form of a diagonal R, and a planted mistake (the
rotations not applied to V) that these pins catch."""
import numpy as np
import pytest

import oracle


def signed(V):
    idx = np.argmax(np.abs(V), axis=0)
    return V * np.sign(V[idx, np.arange(V.shape[1])])


def upper(rng, n, rows=None):
    return np.linalg.qr(rng.standard_normal((rows or 3 * n + 2, n)), mode="r")


def v_pins_hold(R, s, V, tol=1e-12):
    n = R.shape[0]
    U = R @ V
    ok = np.max(np.abs(V.T @ V - np.eye(n))) <= tol * max(n, 1)
    ok &= np.max(np.abs(np.linalg.norm(U, axis=0) - s)) <= tol * max(s[0], 1e-300)
    G = U.T @ U
    off = G - np.diag(np.diag(G))
    ok &= np.max(np.abs(off)) <= tol * max(s[0], 1e-300) ** 2 * max(n, 1)
    return bool(ok)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33, 70])
def test_v_defining_properties(n):
    rng = np.random.default_rng(8100 + n)
    R = upper(rng, n)
    s, V = oracle.jacobi_svd(R)
    assert np.max(np.abs(s - np.linalg.svd(R, compute_uv=False))) <= 1e-12 * s[0]
    assert v_pins_hold(R, s, V)
    # the sign convention: each column's largest-magnitude component is positive
    assert np.all(V[np.argmax(np.abs(V), axis=0), np.arange(n)] > 0)


@pytest.mark.parametrize("n", [4, 16, 32])
def test_v_matches_lapack_for_separated_values(n):
    rng = np.random.default_rng(8200 + n)
    # prescribed, well separated values: U diag(s) W^T, then its R
    s_true = np.linspace(3.0, 1.0, n)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    R = np.linalg.qr(Q1 @ np.diag(s_true) @ Q2.T, mode="r")
    s, V = oracle.jacobi_svd(R)
    _, sv, Vt = np.linalg.svd(R)
    assert np.max(np.abs(s - sv)) <= 1e-13 * sv[0]
    assert np.max(np.abs(V - signed(Vt.T))) <= 1e-10


def test_diagonal_closed_form():
    d = np.array([0.5, -3.0, 2.0, -1.0, 4.0])
    s, V = oracle.jacobi_svd(np.diag(d))
    order = np.argsort(-np.abs(d), kind="stable")
    assert np.array_equal(s, np.abs(d)[order])
    assert np.array_equal(V, np.eye(len(d))[:, order])


def test_planted_unrotated_v_is_caught():
    rng = np.random.default_rng(8300)
    R = upper(rng, 12)
    s, V = oracle.jacobi_svd(R)
    assert v_pins_hold(R, s, V)
    oracle.set_mutation(8)
    try:
        s8, V8 = oracle.jacobi_svd(R)
        assert not v_pins_hold(R, s8, V8), "unrotated V went unnoticed"
    finally:
        oracle.set_mutation(0)
