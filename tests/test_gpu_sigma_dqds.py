"""Singular values by bidiagonalisation and dqds (figaro_triangular_singular_values
and FIGARO_FLAG_SIGMA_DQDS), against the FP64 oracle: its one-sided Jacobi on
the same R (oracle.jacobi_sigma) and, for joins, oracle.join_r_sigma.  Inputs
with a prescribed spectrum (R from the QR of U diag(s) V^T with Haar U, V) are
also checked against s itself.  The argument checks at the end call nothing
on the device and run without a GPU."""
import numpy as np
import pytest

import oracle
from workloads import config, make_pair

EPS = np.finfo(np.float64).eps
KINDS = ["graded", "clustered", "repeated", "rank2", "diag"]


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


def haar(rng, n):
    Q, Rq = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(Rq))


def prescribed(rng, s):
    n = len(s)
    return np.linalg.qr(haar(rng, n) @ np.diag(s) @ haar(rng, n).T, mode="r")


FF_U = 2.0**-46  # roundoff of the float-float arithmetic of the dqds stage


def bound(n, smax):
    """Absolute error allowed on every value: the FP64 bidiagonalisation's
    backward error (a few n eps ||R||), the float-float dqds's (a few n u_ff
    relative) and the reference's own, with margin."""
    return 64.0 * n * (EPS + FF_U) * smax


def run(fg, torch, R):
    s, info = fg.triangular_singular_values(torch.from_numpy(np.ascontiguousarray(R)).cuda())
    return s.cpu().numpy(), info.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 32, 33, 64, 100, 128])
def test_gaussian_triangular_matches_oracle(fg, torch, n):
    rng = np.random.default_rng(7000 + n)
    R = np.linalg.qr(rng.standard_normal((3 * n + 4, n)), mode="r")
    s, info = run(fg, torch, R)
    ref = oracle.jacobi_sigma(R)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - ref)) <= bound(n, ref[0])
    # high relative accuracy on these well-conditioned R
    assert np.max(np.abs(s - ref) / ref) <= 32 * n * FF_U
    assert info[0] >= (1 if n > 1 else 0) and info[0] <= 30 * n + 64


@pytest.mark.gpu
@pytest.mark.parametrize("n", [32, 128])
@pytest.mark.parametrize("kind", KINDS)
def test_prescribed_spectra(fg, torch, n, kind):
    rng = np.random.default_rng(7500 + 10 * n + KINDS.index(kind))
    if kind == "graded":  # condition 1e8, log-spaced
        s = np.logspace(0, -8, n)
    elif kind == "clustered":  # half the values 1, half within 1e-12 of 1
        s = np.ones(n)
        s[n // 2:] += 1e-12 * np.arange(n - n // 2)
    elif kind == "repeated":  # every value the same: B is diagonal at once
        s = np.full(n, 3.0)
    elif kind == "rank2":  # two zero singular values
        s = np.linspace(2.0, 1.0, n)
        s[[3, n - 5]] = 0.0
    else:
        s = np.arange(1, n + 1, dtype=np.float64)
    R = np.diag(s) if kind == "diag" else prescribed(rng, s)
    out, info = run(fg, torch, R)
    ref = np.sort(s)[::-1]
    assert np.all(np.diff(out) <= 0)
    assert np.max(np.abs(out - ref)) <= bound(n, ref[0])
    assert np.max(np.abs(out - oracle.jacobi_sigma(R))) <= bound(n, ref[0])
    assert 0 <= info[0] <= 30 * n + 64


@pytest.mark.gpu
def test_special_matrices(fg, torch):
    # zero matrix, a single entry, a lower triangle that must not be read
    n = 20
    out, info = run(fg, torch, np.zeros((n, n)))
    assert np.all(out == 0) and info[0] == 0
    out, info = run(fg, torch, np.array([[-2.5]]))
    assert out[0] == 2.5 and info[0] == 0
    rng = np.random.default_rng(5)
    R = np.triu(rng.standard_normal((n, n)))
    M = R.copy()
    M[np.tril_indices(n, -1)] = np.nan
    out, _ = run(fg, torch, M)
    ref = oracle.jacobi_sigma(R)
    assert np.max(np.abs(out - ref)) <= bound(n, ref[0])
    # huge and tiny scales: exact power-of-two scaling inside
    for scale in (2.0**600, 2.0**-600):
        out, _ = run(fg, torch, R * scale)
        assert np.max(np.abs(out / scale - ref)) <= bound(n, ref[0])


@pytest.mark.gpu
def test_non_finite_input_is_reported(fg, torch):
    R = np.triu(np.ones((6, 6)))
    R[2, 4] = np.nan
    out, info = run(fg, torch, R)
    assert np.all(np.isnan(out)) and info[0] == -1


@pytest.mark.gpu
def test_many_matrices_one_launch(fg, torch):
    rng = np.random.default_rng(11)
    n, count = 48, 37
    Rs = np.stack([np.linalg.qr(rng.standard_normal((2 * n, n)) * rng.uniform(0.1, 10.0), mode="r")
                   for _ in range(count)])
    s, info = fg.triangular_singular_values(torch.from_numpy(Rs).cuda())
    s, info = s.cpu().numpy(), info.cpu().numpy()
    for b in range(count):
        ref = oracle.jacobi_sigma(Rs[b])
        assert np.max(np.abs(s[b] - ref)) <= bound(n, ref[0])
        assert info[b] > 0


@pytest.mark.gpu
@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(4000, 4, 3000, 4, 70), (30000, 16, 20000, 16, 900), (5000, 70, 4000, 58, 60)],
                         ids=["8", "32", "128"])
def test_join_flag_matches_oracle(fg, torch, path, shape):
    m1, n1, m2, n2, keys = shape
    A, B = make_pair(m1, n1, m2, n2, keys, np.float32, "normal", seed=4100 + n1)
    _, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    d = [(torch.from_numpy(np.ascontiguousarray(T.x)).cuda(), torch.from_numpy(np.ascontiguousarray(T.key)).cuda())
         for T in (A, B)]
    solver = fg.Solver(d[0], d[1], path=path, flags=fg.FLAG_SIGMA_DQDS)
    R, s = solver(d[0], d[1])
    assert solver.status() == 0
    s = s.cpu().numpy()
    tol = 1e-10 if path == "fp64" else 1e-6
    assert np.linalg.norm(s - sref) / np.linalg.norm(sref) <= tol
    # the R that the call returns gives the same values through the direct
    # call (the accurate form; the mixed path's stages run in FP32)
    s2, _ = fg.triangular_singular_values(R)
    agree = bound(len(s), s[0]) if path == "fp64" else 1e-6 * s[0]
    assert np.max(np.abs(s - s2.cpu().numpy())) <= agree
    assert solver.info()["jacobi_sweeps"] > 0  # dqds transforms


@pytest.mark.gpu
def test_batch_flag_matches_single_calls(fg, torch):
    pairs, refs = [], []
    # (100, 100): a wide instance, which the batch runs as a call of its own (the wide form)
    for i, (n1, n2) in enumerate([(4, 4), (16, 16), (30, 34), (8, 24), (100, 100)]):
        A, B = make_pair(3000 + 500 * i, n1, 2500 + 300 * i, n2, 50 + 10 * i, np.float32, "normal", seed=4200 + i)
        refs.append(oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")[1])
        pairs.append(tuple((torch.from_numpy(np.ascontiguousarray(T.x)).cuda(),
                            torch.from_numpy(np.ascontiguousarray(T.key)).cuda()) for T in (A, B)))
    outs, _ = fg.batch_join(pairs, flags=fg.FLAG_SIGMA_DQDS)
    for (R, s), sref in zip(outs, refs):
        s = s.cpu().numpy()
        assert np.linalg.norm(s - sref) / np.linalg.norm(sref) <= 1e-6
        if len(s) <= 128:  # the direct call's limit
            s2, _ = fg.triangular_singular_values(R)
            assert np.max(np.abs(s - s2.cpu().numpy())) <= 1e-6 * s[0]  # FP32 stages on the mixed path


@pytest.mark.gpu
def test_wide_c4_shape_graded(fg, torch):
    """n = 512 (the wide form: one CTA, FP64 bidiagonalisation in global
    scratch, float-float dqds) on the c4 shape at 2 % of its rows, B's columns
    scaled to condition 1e8, both paths, against O2.  Householder
    bidiagonalisation keeps the values to absolute accuracy (of order
    n u ||R||), not to relative accuracy for graded columns: the per-value
    bound is relative to sigma_max."""
    A, B = config("c4", scale=0.02)
    assert A.n + B.n == 512
    _, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    d = [(torch.from_numpy(np.ascontiguousarray(T.x)).cuda(), torch.from_numpy(np.ascontiguousarray(T.key)).cuda())
         for T in (A, B)]
    for path, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        solver = fg.Solver(d[0], d[1], path=path, flags=fg.FLAG_SIGMA_DQDS)
        _, s = solver(d[0], d[1])
        assert solver.status() == 0
        s = s.cpu().numpy()
        assert np.all(np.diff(s) <= 0)
        assert np.linalg.norm(s - sref) / np.linalg.norm(sref) <= tol
        assert np.max(np.abs(s - sref)) <= tol * sref[0]
        assert solver.info()["jacobi_sweeps"] > 512  # dqds transforms


def test_argument_checks_need_no_device():
    """Rejected before any device call (null pointers are never dereferenced)."""
    import ctypes
    import paper_2503_23385_gb300 as fg
    lib = fg.library()
    f = lib.figaro_triangular_singular_values
    one = ctypes.c_void_p(16)
    assert f(None, 4, 0, 4, 1, one, None, None) == 1          # R missing
    assert f(one, 4, 0, 4, 1, None, None, None) == 1          # sigma missing
    assert f(one, 4, 0, 0, 1, one, None, None) == 1           # n < 1
    assert f(one, 3, 0, 4, 1, one, None, None) == 1           # ldr < n
    assert f(one, 4, -1, 4, 1, one, None, None) == 1          # negative stride
    assert f(one, 4, 0, 4, -1, one, None, None) == 1          # negative count
    assert f(one, 129, 0, 129, 1, one, None, None) == 7       # n > 128: unsupported
    assert f(one, 4, 0, 4, 0, one, None, None) == 0           # nothing to do


def test_flag_rejected_where_it_cannot_apply():
    """The dqds flag is accepted at every supported width (a 200-column join
    sizes its workspace) and refused by figaro_join_svd, which needs the
    rotations (argument checks only, no device call)."""
    import ctypes
    import paper_2503_23385_gb300 as fg
    lib = fg.library()
    A = fg.Table(ctypes.c_void_p(16), ctypes.c_void_p(16), 10, 100, 100, fg.F32, fg.MEM_DEVICE, 0)
    B = fg.Table(ctypes.c_void_p(16), ctypes.c_void_p(16), 10, 100, 100, fg.F32, fg.MEM_DEVICE, 0)
    o = fg._options(flags=fg.FLAG_SIGMA_DQDS)
    one = ctypes.c_void_p(16)
    sz = ctypes.c_size_t(0)
    assert lib.figaro_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(sz)) == 0
    assert sz.value > 0
    A.n = B.n = 8
    A.ld = B.ld = 8
    assert lib.figaro_join_svd(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), one, one, 16, None, 16, one, 1 << 20,
                               None) == 7


def test_binding_rejects_what_the_call_cannot_take():
    """The Python wrapper refuses CPU tensors, other dtypes and non-square
    matrices before calling the library (no device needed)."""
    import torch
    import paper_2503_23385_gb300 as fg
    for bad in (torch.zeros((4, 4), dtype=torch.float64),        # host memory
                torch.zeros((4, 4), dtype=torch.float32),        # not FP64
                torch.zeros((3, 4, 5), dtype=torch.float64)):    # not square
        with pytest.raises(fg.FigaroError):
            fg.triangular_singular_values(bad)
