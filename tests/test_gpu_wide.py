"""Wide joins (n1 + n2 in (128, 512]) through the C ABI against the FP64 oracle.

Above 128 columns the library switches to its multi-CTA path: Q = X W
written out, tiled Gram partials, a blocked Cholesky and a block one-sided
Jacobi.  The bars are those of the narrow path: relative Frobenius error
<= 1e-10 (plain FP64 path) and <= 1e-6 (mixed path) for R and sigma on
well-conditioned inputs.  The geometrically column-scaled case (condition
number 1e8) is checked on the error after undoing the column scaling.
"""
import numpy as np
import pytest

import oracle
from workloads import config, make_pair, Table

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}


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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run(fg, torch, A, B, path, **opts):
    R, s = fg.join_qr_svd(dev(torch, A), dev(torch, B), path=path, **opts)
    torch.cuda.synchronize()
    return R.cpu().numpy(), s.cpu().numpy()


@pytest.mark.parametrize("shape", [(3000, 128, 2500, 64, 30), (2000, 200, 1500, 57, 40), (1500, 3, 1200, 130, 20),
                                   (4000, 256, 4000, 256, 100)],
                         ids=["192", "257-ragged", "133", "512"])
def test_wide_widths_match_oracle(fg, torch, shape):
    m1, n1, m2, n2, keys = shape
    A, B = make_pair(m1, n1, m2, n2, keys, np.float32, "normal", seed=600 + n1 + n2)
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    for path in ("fp64", "mixed"):
        R, s = run(fg, torch, A, B, path)
        eR, es = rel(R, Rref), rel(s, sref)
        assert eR <= TOL[path] and es <= TOL[path], f"{path}: err_R={eR:.3e} err_sigma={es:.3e}"
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)
        assert np.all(np.diff(s) <= 0)


def test_wide_rank_deficient(fg, torch):
    """Two copies of a column of A: R is not unique then (any R with
    R^T R = J^T J), so the check is on what is: R^T R against the oracle's
    J^T J (per-group sums), sigma against the oracle's, the dependent
    column's row of R zero and the smallest singular value at rounding level."""
    A, B = make_pair(3000, 100, 2500, 60, 30, np.float64, "normal", seed=610)
    x = A.x.copy()
    x[:, 7] = x[:, 3]
    A = Table(x, A.key)
    for path, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        Ar, Br = A, B
        if path == "mixed":
            Ar, Br = Table(A.x.astype(np.float32).astype(np.float64), A.key), Table(B.x.astype(np.float32).astype(np.float64), B.key)
        G = oracle.join_gram(Ar.x, Ar.key, Br.x, Br.key)
        _, sref = oracle.join_r_sigma(Ar.x, Ar.key, Br.x, Br.key, route="reduced")
        R, s = run(fg, torch, A, B, path, flags=fg.FLAG_ALLOW_RANK_DEFICIENT)
        assert np.all(R[7] == 0)
        assert s[-1] <= 10 * tol * s[0]
        assert rel(s, sref) <= tol
        assert rel(R.T @ R, G) <= tol


def test_c4_shape_column_scaled(fg, torch):
    """The wide, ill-conditioned workload at 2% of its rows: B's columns are
    scaled by 10^(-8 j / 255), condition number 1e8.  Column scaling does not
    change the relative accuracy Cholesky and one-sided Jacobi can reach, so
    the error is measured after undoing it: ||(R - R*) D^-1|| / ||R* D^-1||
    and the largest relative error of a singular value."""
    A, B = config("c4", scale=0.02)
    assert A.n + B.n == 512
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    d = np.concatenate([np.ones(A.n), 10.0 ** (-8.0 * np.arange(B.n) / (B.n - 1))])
    # per-sigma bars: the FP64 path reaches ~1e-13, the mixed path ~2e-5 here
    for path, tol, tol_sv in (("fp64", 1e-10, 1e-8), ("mixed", 1e-6, 2e-4)):
        R, s = run(fg, torch, A, B, path)
        assert rel(R, Rref) <= tol and rel(s, sref) <= tol
        escaled = rel(R / d, Rref / d)
        esv = np.max(np.abs(s - sref) / sref)
        assert escaled <= 100 * tol, f"{path}: column-scaled err_R={escaled:.3e}"
        assert esv <= tol_sv, f"{path}: max per-sigma relative error {esv:.3e}"


def test_wide_results_are_deterministic(fg, torch):
    A, B = make_pair(20000, 160, 15000, 96, 200, np.float32, "normal", seed=620)
    for path in ("fp64", "mixed"):
        R1, s1 = run(fg, torch, A, B, path)
        R2, s2 = run(fg, torch, A, B, path)
        assert np.array_equal(R1, R2) and np.array_equal(s1, s2)
