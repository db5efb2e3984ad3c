"""figaro_join_least_squares (B's last column is the label) against the FP64
oracle's least squares over the materialised join."""
import numpy as np
import pytest

import oracle
from workloads import Table, make_pair

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("shape", [(3000, 4, 2500, 5, 60), (20000, 16, 15000, 17, 500), (800, 1, 900, 2, 40)])
def test_least_squares_matches_oracle(fg, torch, shape):
    m1, n1, m2, n2, keys = shape
    A, B = make_pair(m1, n1, m2, n2, keys, np.float64, "normal", seed=800 + n1)
    x = B.x.copy()
    x[:, -1] += 0.7 * x[:, 0] - 0.2 * (x[:, 1] if n2 > 2 else 0.0)  # the label depends on some features
    B = Table(x, B.key)
    beta_ref, res_ref = oracle.join_least_squares(A.x, A.key, B.x, B.key)
    for path, tol in (("fp64", 1e-9), ("mixed", 2e-5)):
        Ar, Br = A, B
        if path == "mixed":
            Ar = Table(A.x.astype(np.float32).astype(np.float64), A.key)
            Br = Table(B.x.astype(np.float32).astype(np.float64), B.key)
            beta_ref, res_ref = oracle.join_least_squares(Ar.x, Ar.key, Br.x, Br.key)
        beta, res = fg.join_least_squares(dev(torch, A), dev(torch, B), path=path)
        beta, res = beta.cpu().numpy(), float(res.cpu().numpy()[0])
        assert rel(beta, beta_ref) <= tol, (path, rel(beta, beta_ref))
        assert abs(res - res_ref) <= tol * res_ref, (path, res, res_ref)


def test_exact_fit_and_dependent_feature(fg, torch):
    """The label is an exact combination of B's features (residual at rounding
    level, coefficients recovered); with a duplicated feature column beta is
    not unique, so the fitted values J_x beta and the residual are compared."""
    A, B = make_pair(5000, 3, 4000, 3, 80, np.float64, "normal", seed=820)
    w = np.array([2.0, -1.0])
    x = np.column_stack([B.x[:, :2], B.x[:, :2] @ w])
    B = Table(x, B.key)
    for path, tol in (("fp64", 1e-9), ("mixed", 2e-5)):
        beta, res = fg.join_least_squares(dev(torch, A), dev(torch, B), path=path)
        beta, res = beta.cpu().numpy(), float(res.cpu().numpy()[0])
        assert np.allclose(beta, [0, 0, 0, 2.0, -1.0], atol=tol * 10)
        J = oracle.materialize(A.x, A.key, B.x, B.key)
        assert res <= tol * np.linalg.norm(J[:, -1])
    # a feature duplicated: column 1 of A copied into column 2
    A2 = Table(np.column_stack([A.x[:, :2], A.x[:, 1]]), A.key)
    B2 = Table(np.column_stack([B.x[:, :2], B.x[:, 2] + np.sin(B.x[:, 0])]), B.key)
    J = oracle.materialize(A2.x, A2.key, B2.x, B2.key)
    beta_ref, res_ref = oracle.join_least_squares(A2.x, A2.key, B2.x, B2.key)
    beta, res = fg.join_least_squares(dev(torch, A2), dev(torch, B2), path="fp64",
                                      flags=fg.FLAG_ALLOW_RANK_DEFICIENT)
    beta, res = beta.cpu().numpy(), float(res.cpu().numpy()[0])
    assert rel(J[:, :-1] @ beta, J[:, :-1] @ beta_ref) <= 1e-9
    assert abs(res - res_ref) <= 1e-9 * res_ref
