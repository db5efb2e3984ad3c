"""figaro_join_svd: sigma and the right singular vectors V of the join,
against the FP64 oracle (sigma, and V of the oracle's R by the oracle's
Jacobi with accumulated rotations, pinned by LAPACK in test_oracle_svd.py;
J = Q R)."""
import numpy as np
import pytest

import oracle
from workloads import Table, make_pair

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
VTOL = {"fp64": 1e-9, "mixed": 1e-4}


@pytest.fixture(scope="module")
def fg():
    import paper_2503_23385_gb300 as fg
    fg.library()
    return fg


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def dev(torch, T):
    return (torch.from_numpy(np.ascontiguousarray(T.x)).cuda(), torch.from_numpy(np.ascontiguousarray(T.key)).cuda())


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape", [(3000, 4, 2500, 4, 60), (20000, 16, 15000, 16, 500), (3000, 100, 2000, 60, 40)],
                         ids=["8", "32", "160-wide"])
def test_svd_matches_oracle(fg, torch, shape):
    m1, n1, m2, n2, keys = shape
    A, B = make_pair(m1, n1, m2, n2, keys, np.float32, "normal", seed=900 + n1)
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    # V of R (right singular vectors of J, the largest component of each column positive)
    sv, Vref = oracle.jacobi_svd(Rref)
    gaps = np.min(np.abs(np.diff(sv)) / sv[0])
    for path in ("fp64", "mixed"):
        s, V, R = fg.join_svd(dev(torch, A), dev(torch, B), path=path)
        s, V, R = s.cpu().numpy(), V.cpu().numpy(), R.cpu().numpy()
        assert rel(s, sref) <= TOL[path] and rel(R, Rref) <= TOL[path]
        n = V.shape[0]
        assert np.linalg.norm(V.T @ V - np.eye(n)) <= VTOL[path] * np.sqrt(n)
        # R v_j = sigma_j u_j: the column norms of R V are the singular values
        assert rel(np.linalg.norm(Rref @ V, axis=0), sref) <= 10 * TOL[path]
        if gaps > 1e-3:  # well separated: the vectors themselves are unique up to sign
            assert np.max(np.abs(V - Vref)) <= VTOL[path] / gaps, (path, np.max(np.abs(V - Vref)))


def test_svd_on_the_materialised_join(fg, torch):
    """||J v_j|| = sigma_j and J^T J v_j = sigma_j^2 v_j on a small join."""
    A, B = make_pair(300, 3, 250, 2, 12, np.float64, "normal", seed=930)
    J = oracle.materialize(A.x, A.key, B.x, B.key)
    s, V, _ = fg.join_svd(dev(torch, A), dev(torch, B), path="fp64")
    s, V = s.cpu().numpy(), V.cpu().numpy()
    assert np.allclose(np.linalg.norm(J @ V, axis=0), s, rtol=1e-10)
    G = J.T @ J
    assert np.linalg.norm(G @ V - V * s ** 2) <= 1e-9 * np.linalg.norm(G)
