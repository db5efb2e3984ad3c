"""Pins for the FP64 oracle: each check comes from outside the oracle itself
(LAPACK, brute-force joins built here, closed forms, invariants of the paper).

Paper: "Figaro on GPUs: Two Tables" (arXiv 2503.23385).
  Section 1  Cartesian product, QR head H and QR tail T, Claim 1, the
             O((m1+m2)(n1+n2)^2) finish; R is the Cholesky factor of J^T J and
             prod diag(R) = |det J| = prod sigma for square J.
  Section 3  sigma(J) = sigma(R) (SVD through QR then SVD of R).
"""
import numpy as np
import pytest

import oracle
from workloads import make_pair


def brute_join(A, kA, B, kB):
    """J built with Python loops: one row [A_i, B_j] per pair with equal keys."""
    rows = []
    for i in range(A.shape[0]):
        for j in range(B.shape[0]):
            if kA[i] == kB[j]:
                rows.append(np.concatenate([A[i], B[j]]))
    n = A.shape[1] + B.shape[1]
    return np.array(rows, dtype=np.float64).reshape(-1, n)


def lapack_r(X):
    n = X.shape[1]
    if X.shape[0] == 0:
        return np.zeros((n, n))
    R = np.linalg.qr(X, mode="r")
    R = np.vstack([R, np.zeros((n - R.shape[0], n))]) if R.shape[0] < n else R[:n]
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return R * s[:, None]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---------------------------------------------------------------- grouping --

def test_stable_sort_matches_numpy_stable_argsort():
    rng = np.random.default_rng(1)
    key = rng.integers(-50, 50, size=3000).astype(np.int32)
    key[:5] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0, -1, np.iinfo(np.int32).min]
    g = oracle.group(key)
    perm = np.argsort(key, kind="stable")
    assert np.array_equal(g["perm"], perm)
    assert np.array_equal(g["sorted_key"], key[perm])
    u, first, cnt = np.unique(key, return_index=False, return_counts=True), None, None
    uq, idx, counts = np.unique(key[perm], return_index=True, return_counts=True)
    assert np.array_equal(g["uniq"], uq)
    assert np.array_equal(g["offset"][:-1], idx)
    assert g["offset"][-1] == key.shape[0]
    assert np.array_equal(g["count"], counts)


def test_group_edge_cases():
    for key in [np.zeros(0, np.int32), np.array([7], np.int32), np.full(100, 3, np.int32),
                np.arange(100, 0, -1).astype(np.int32)]:
        g = oracle.group(key)
        assert np.array_equal(g["perm"], np.argsort(key, kind="stable"))
        assert g["count"].sum() == key.shape[0]


def test_match_is_key_intersection():
    rng = np.random.default_rng(2)
    kA = rng.integers(0, 40, 500).astype(np.int32)
    kB = rng.integers(20, 60, 300).astype(np.int32)
    mt = oracle.match(oracle.group(kA), oracle.group(kB))
    common = np.intersect1d(kA, kB)
    assert np.array_equal(mt["key"], common)
    for t, k in enumerate(common):
        assert mt["m1"][t] == np.sum(kA == k) and mt["m2"][t] == np.sum(kB == k)


# ------------------------------------------------------------ Householder --

@pytest.mark.parametrize("shape", [(50, 7), (8, 8), (3, 6), (200, 32), (1, 4)])
def test_householder_matches_lapack(shape):
    X = np.random.default_rng(3).standard_normal(shape)
    R = oracle.qr_r(X)
    assert rel(R, lapack_r(X)) < 1e-13


def test_householder_blocked_equals_one_shot():
    X = np.random.default_rng(4).standard_normal((1000, 9))
    assert rel(oracle.qr_r(X, block_rows=17), oracle.qr_r(X, block_rows=100000)) < 1e-13


# ---------------------------------------------------------------- Jacobi --

@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_jacobi_matches_lapack_svd(n):
    R = np.triu(np.random.default_rng(5 + n).standard_normal((n, n)))
    s = oracle.jacobi_sigma(R)
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(s - ref) / ref[0]) < 1e-13


def test_jacobi_closed_forms():
    d = np.array([3.0, -7.0, 0.5, 0.0])
    assert np.allclose(oracle.jacobi_sigma(np.diag(d)), [7.0, 3.0, 0.5, 0.0], rtol=0, atol=1e-15)
    # [[1, 1], [0, 1]]: sigma = (1 +- sqrt 5) / 2 in absolute value (golden ratio pair)
    s = oracle.jacobi_sigma(np.array([[1.0, 1.0], [0.0, 1.0]]))
    phi = (1 + np.sqrt(5)) / 2
    assert np.allclose(s, [phi, 1 / phi], rtol=1e-15)


# ------------------------------------------------------- head/tail (Sec. 1) --

@pytest.mark.parametrize("m", [1, 2, 3, 10, 57])
def test_head_tail_form_an_orthogonal_matrix(m):
    """[H(I_m); T(I_m)] is the m x m matrix of the transform; it must be
    orthogonal (Claim 1 is a product of Givens rotations)."""
    I = np.eye(m)
    Hm = np.vstack([oracle.qr_head(I)[None, :], oracle.qr_tail(I)])
    assert Hm.shape == (m, m)
    assert np.allclose(Hm @ Hm.T, np.eye(m), atol=1e-14)


def test_head_tail_special_cases():
    X = np.array([[1.0, 2.0, -3.0], [4.0, 6.0, 5.0]])
    # m = 2: H = (x1 + x2)/sqrt 2, T = (x2 - x1)/sqrt 2 (a single Givens rotation)
    assert np.allclose(oracle.qr_head(X), (X[0] + X[1]) / np.sqrt(2), rtol=1e-15)
    assert np.allclose(oracle.qr_tail(X), ((X[1] - X[0]) / np.sqrt(2))[None, :], rtol=1e-15)
    # constant columns: all of the mass goes to the head, the tails vanish
    C = np.ones((9, 2)) * np.array([2.0, -5.0])
    assert np.allclose(oracle.qr_head(C), np.sqrt(9) * np.array([2.0, -5.0]), rtol=1e-15)
    assert np.allclose(oracle.qr_tail(C), 0.0, atol=1e-14)


def test_head_tail_preserve_gram():
    X = np.random.default_rng(6).standard_normal((40, 5))
    h, T = oracle.qr_head(X), oracle.qr_tail(X)
    assert np.allclose(np.outer(h, h) + T.T @ T, X.T @ X, rtol=1e-13, atol=1e-12)


# --------------------------------------------------------- Claim 1 / joins --

@pytest.mark.parametrize("m1,m2,n1,n2", [(1, 1, 1, 1), (2, 3, 1, 2), (5, 7, 2, 3), (8, 8, 4, 4), (1, 6, 1, 3),
                                         (6, 1, 3, 1)])
def test_claim1_cartesian_products_bruteforce(m1, m2, n1, n2):
    rng = np.random.default_rng(10 + m1 * 10 + m2)
    A, B = rng.standard_normal((m1, n1)), rng.standard_normal((m2, n2))
    kA, kB = np.zeros(m1, np.int32), np.zeros(m2, np.int32)
    J = brute_join(A, kA, B, kB)
    assert J.shape[0] == m1 * m2
    Rref = lapack_r(J)
    for route in ("materialized", "reduced"):
        R, s = oracle.join_r_sigma(A, kA, B, kB, route=route)
        assert rel(R, Rref) < 1e-12, route
        sref = np.linalg.svd(J, compute_uv=False)
        sref = np.concatenate([sref, np.zeros(n1 + n2 - sref.shape[0])])
        assert np.max(np.abs(s - sref)) < 1e-12 * max(sref[0], 1)


@pytest.mark.parametrize("seed", range(5))
def test_natural_join_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    m1, m2 = rng.integers(5, 60, 2)
    n1, n2 = rng.integers(1, 5, 2)
    kA = rng.integers(0, 12, m1).astype(np.int32)
    kB = rng.integers(4, 16, m2).astype(np.int32)   # keys 0..3 only in A, 12..15 only in B
    A, B = rng.uniform(-1, 1, (m1, n1)), rng.uniform(-1, 1, (m2, n2))
    J = brute_join(A, kA, B, kB)
    assert oracle.join_rows(kA, kB) == J.shape[0]
    assert np.allclose(oracle.materialize(A, kA, B, kB)[np.lexsort(oracle.materialize(A, kA, B, kB).T[::-1])],
                       J[np.lexsort(J.T[::-1])])
    Rref = lapack_r(J)
    for route in ("materialized", "reduced"):
        R = (oracle.join_r_materialized if route == "materialized" else oracle.join_r_reduced)(A, kA, B, kB)
        assert rel(R, Rref) < 1e-12, route
    assert rel(oracle.join_gram(A, kA, B, kB), J.T @ J) < 1e-14


def test_reduced_rows_gram_equals_join_gram():
    A, B = make_pair(300, 3, 200, 4, 25, np.float64, "uniform_pm1", seed=5)
    red = oracle.reduce(A.x, A.key, B.x, B.key)
    n1, n2 = 3, 4
    M = np.vstack([red["Hd"], np.hstack([red["TA"], np.zeros((red["TA"].shape[0], n2))]),
                   np.hstack([np.zeros((red["TB"].shape[0], n1)), red["TB"]])])
    J = brute_join(A.x, A.key, B.x, B.key)
    assert rel(M.T @ M, J.T @ J) < 1e-13
    # row count of the reduced matrix: sum_g (m1g + m2g - 1)
    mt = oracle.match(oracle.group(A.key), oracle.group(B.key))
    assert M.shape[0] == int(np.sum(mt["m1"] + mt["m2"] - 1))


# -------------------------------------------------------------- invariants --

def test_invariants_square_join():
    """m1 = m2 = 2 Cartesian with n1 = n2 = 2: J is 4 x 4, so
    prod diag(R) = |det J| = prod sigma (Section 1, applications)."""
    rng = np.random.default_rng(7)
    A, B = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    kA = kB = np.zeros(2, np.int32)
    J = brute_join(A, kA, B, kB)
    assert J.shape == (4, 4)
    R, s = oracle.join_r_sigma(A, kA, B, kB)
    d = abs(np.linalg.det(J))
    # J has rank <= 3 here (the Cartesian block structure makes it singular)
    assert abs(np.prod(np.diag(R)) - d) < 1e-12 and abs(np.prod(s) - d) < 1e-12


def test_invariants_square_nonsingular_join():
    """Keys chosen so J is square and non-singular: two 1x1 groups and one 1x2."""
    rng = np.random.default_rng(8)
    A, B = rng.standard_normal((3, 2)), rng.standard_normal((4, 2))
    kA = np.array([1, 2, 3], np.int32)
    kB = np.array([1, 2, 3, 3], np.int32)
    J = brute_join(A, kA, B, kB)
    assert J.shape == (4, 4)
    d = abs(np.linalg.det(J))
    assert d > 1e-3
    R, s = oracle.join_r_sigma(A, kA, B, kB)
    assert abs(np.prod(np.diag(R)) - d) < 1e-12 * max(d, 1)
    assert abs(np.prod(s) - d) < 1e-12 * max(d, 1)


def test_invariants_random_join():
    A, B = make_pair(400, 4, 300, 3, 30, np.float64, "normal", seed=9)
    J = brute_join(A.x, A.key, B.x, B.key)
    R, s = oracle.join_r_sigma(A.x, A.key, B.x, B.key)
    assert rel(R.T @ R, J.T @ J) < 1e-13
    assert abs(np.sum(s ** 2) - np.sum(J ** 2)) < 1e-12 * np.sum(J ** 2)
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)


def test_ones_closed_form():
    """A = ones(m1 x 1), B = ones(m2 x 1): J = ones(m1 m2 x 2), so
    R = [[sqrt(m1 m2), sqrt(m1 m2)], [0, 0]] and sigma = (sqrt(2 m1 m2), 0)."""
    for m1, m2 in [(1, 1), (3, 5), (40, 17)]:
        A, B = np.ones((m1, 1)), np.ones((m2, 1))
        k1, k2 = np.full(m1, 4, np.int32), np.full(m2, 4, np.int32)
        for route in ("materialized", "reduced"):
            R, s = oracle.join_r_sigma(A, k1, B, k2, route=route)
            r = np.sqrt(m1 * m2)
            assert np.allclose(R, [[r, r], [0, 0]], atol=1e-12)
            assert np.allclose(s, [np.sqrt(2 * m1 * m2), 0], atol=1e-12)


def test_one_to_one_join_is_plain_qr_of_paired_rows():
    rng = np.random.default_rng(11)
    m = 50
    A, B = rng.standard_normal((m, 3)), rng.standard_normal((m, 2))
    kA = rng.permutation(m).astype(np.int32)
    kB = rng.permutation(m).astype(np.int32)
    # pair rows by key explicitly
    ia, ib = np.argsort(kA), np.argsort(kB)
    X = np.hstack([A[ia], B[ib]])
    assert rel(oracle.join_r_reduced(A, kA, B, kB), lapack_r(X)) < 1e-12


def test_empty_and_short_joins():
    rng = np.random.default_rng(12)
    A, B = rng.standard_normal((5, 3)), rng.standard_normal((4, 2))
    R = oracle.join_r_reduced(A, np.zeros(5, np.int32), B, np.ones(4, np.int32))
    assert np.all(R == 0)
    # a short join: 2 rows, 5 columns -> rows 2..4 of R are zero
    kA = np.array([0, 1, 2, 3, 4], np.int32)
    kB = np.array([0, 9, 9, 1], np.int32)
    J = brute_join(A, kA, B, kB)
    assert J.shape[0] == 2
    for route in ("materialized", "reduced"):
        R = (oracle.join_r_materialized if route == "materialized" else oracle.join_r_reduced)(A, kA, B, kB)
        assert rel(R, lapack_r(J)) < 1e-12
        assert np.allclose(R[2:], 0)


# -------------------------------------------------------- planted mistakes --

def _pins_pass():
    """A compact set of the pins above; False if any fails."""
    rng = np.random.default_rng(13)
    A, B = rng.standard_normal((7, 2)), rng.standard_normal((6, 3))
    kA = np.array([0, 1, 1, 2, 2, 2, 3], np.int32)
    kB = np.array([2, 1, 2, 1, 1, 4], np.int32)   # group sizes differ: (2, 3) and (3, 2)
    J = brute_join(A, kA, B, kB)
    ok = True
    for route in ("materialized", "reduced"):
        try:
            R, s = oracle.join_r_sigma(A, kA, B, kB, route=route)
        except RuntimeError:  # e.g. Jacobi stops converging
            return False
        ok &= rel(R, lapack_r(J)) < 1e-12
        sref = np.linalg.svd(J, compute_uv=False)
        ok &= np.max(np.abs(s - sref)) < 1e-12 * sref[0]
    g = oracle.group(kA)
    ok &= np.array_equal(g["perm"], np.argsort(kA, kind="stable"))
    I = np.eye(5)
    Hm = np.vstack([oracle.qr_head(I)[None, :], oracle.qr_tail(I)])
    ok &= np.allclose(Hm @ Hm.T, np.eye(5), atol=1e-14)
    return bool(ok)


@pytest.mark.parametrize("code", [1, 2, 3, 4, 5, 6, 7])
def test_planted_mistakes_are_caught(code):
    assert _pins_pass()
    oracle.set_mutation(code)
    try:
        assert not _pins_pass(), f"mutation {code} went unnoticed"
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()
