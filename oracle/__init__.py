"""Figaro two-table oracle (Python side): plain FP64 CPU reference.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  It shares no code with the CUDA path: the arithmetic lives in
``figaro_oracle.c`` (compiled here with gcc, no CUDA) and this module only
marshals numpy arrays.

Functions (paper: "Figaro on GPUs: Two Tables", arXiv 2503.23385):

* :func:`group` -- stable sort by key, runs, matched keys (inner natural join).
* :func:`join_r_materialized` (O1) -- Householder QR of the materialised join.
* :func:`join_r_reduced` (O2) -- Householder QR of the per-group head/tail
  rows (Section 1, H and T operators and Claim 1).
* :func:`reduce` -- the head/tail rows themselves, in group order.
* :func:`join_gram` (O3) -- J^T J from per-group sums.
* :func:`jacobi_sigma` -- one-sided Jacobi singular values of a square matrix.
* :func:`join_least_squares` -- least squares over the materialised join.
* :func:`qr_r` -- Householder R of a dense matrix (sign-normalised).
* :func:`materialize` -- rows of J, for brute-force checks on small inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "figaro_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_figaro.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle C library with gcc (IEEE arithmetic, no contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    lib.oracle_set_mutation.argtypes = [_int]
    lib.oracle_set_mutation.restype = None
    lib.oracle_stable_sort.argtypes = [_i32p, _i64, _i32p, _i32p]
    lib.oracle_runs.argtypes = [_i32p, _i64, _i32p, _i32p]
    lib.oracle_runs.restype = _i64
    lib.oracle_match.argtypes = [_i32p, _i32p, _i64, _i32p, _i32p, _i64, _i32p, _i32p, _i32p, _i32p, _i32p]
    lib.oracle_match.restype = _i64
    lib.oracle_qr_update.argtypes = [_f64p, _int, _f64p, _i64, _i64]
    lib.oracle_sign_normalise.argtypes = [_f64p, _int]
    lib.oracle_jacobi_sigma.argtypes = [_f64p, _int, _f64p, _int]
    lib.oracle_jacobi_sigma.restype = _int
    lib.oracle_jacobi_svd.argtypes = [_f64p, _int, _f64p, _f64p, _int]
    lib.oracle_jacobi_svd.restype = _int
    lib.oracle_join_rows.argtypes = [_i32p, _i64, _i32p, _i64]
    lib.oracle_join_rows.restype = _i64
    tab = [_f64p, _i64, _int, _i64, _i32p]
    lib.oracle_join_materialize.argtypes = tab + tab + [_i64, _i64, _f64p]
    lib.oracle_join_materialize.restype = _i64
    lib.oracle_join_r_materialized.argtypes = tab + tab + [_i64, _f64p]
    lib.oracle_join_r_reduced.argtypes = tab + tab + [_i64, _f64p]
    lib.oracle_reduce_sizes.argtypes = [_i32p, _i64, _i32p, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    lib.oracle_reduce_sizes.restype = _i64
    lib.oracle_reduce.argtypes = tab + tab + [_f64p, _f64p, _f64p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    lib.oracle_reduce.restype = _i64
    lib.oracle_join_gram.argtypes = tab + tab + [_f64p]
    lib.oracle_qr_head.argtypes = [ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), _i64, _int, _f64p]
    lib.oracle_qr_tail.argtypes = [ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), _i64, _int, _f64p]
    _lib = lib
    return lib


def set_mutation(code: int) -> None:
    """Plant a known mistake in the oracle (tests only; 0 turns it off)."""
    _load().oracle_set_mutation(int(code))


def _table(x, key):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if x.ndim != 2:
        raise ValueError("features must be 2-D")
    key = np.ascontiguousarray(np.asarray(key, dtype=np.int32))
    if key.shape[0] != x.shape[0]:
        raise ValueError("one key per row")
    m, n = x.shape
    buf = x if m > 0 else np.zeros((1, max(n, 1)), dtype=np.float64)
    kbuf = key if m > 0 else np.zeros(1, dtype=np.int32)
    return [buf, m, n, max(n, 1), kbuf]


def group(key):
    """Stable sort by key and its runs.

    Returns dict(perm, sorted_key, uniq, offset (U+1 entries), count)."""
    lib = _load()
    key = np.ascontiguousarray(np.asarray(key, dtype=np.int32))
    m = key.shape[0]
    perm = np.zeros(max(m, 1), dtype=np.int32)
    sk = np.zeros(max(m, 1), dtype=np.int32)
    kbuf = key if m > 0 else np.zeros(1, dtype=np.int32)
    lib.oracle_stable_sort(kbuf, m, perm, sk)
    uniq = np.zeros(max(m, 1), dtype=np.int32)
    off = np.zeros(m + 1, dtype=np.int32)
    U = lib.oracle_runs(sk, m, uniq, off)
    return {"perm": perm[:m], "sorted_key": sk[:m], "uniq": uniq[:U], "offset": off[:U + 1],
            "count": np.diff(off[:U + 1])}


def match(ga, gb):
    """Keys present in both groupings: dict(key, offA, m1, offB, m2)."""
    lib = _load()
    UA, UB = ga["uniq"].shape[0], gb["uniq"].shape[0]
    gm = max(min(UA, UB), 1)
    out = [np.zeros(gm, dtype=np.int32) for _ in range(5)]
    ua = ga["uniq"] if UA else np.zeros(1, np.int32)
    ub = gb["uniq"] if UB else np.zeros(1, np.int32)
    G = lib.oracle_match(ua, np.ascontiguousarray(ga["offset"]), UA, ub, np.ascontiguousarray(gb["offset"]), UB,
                         *out)
    names = ["key", "offA", "m1", "offB", "m2"]
    return {k: v[:G] for k, v in zip(names, out)}


def join_rows(kA, kB) -> int:
    lib = _load()
    ta, tb = _table(np.zeros((len(kA), 1)), kA), _table(np.zeros((len(kB), 1)), kB)
    return int(lib.oracle_join_rows(ta[4], ta[1], tb[4], tb[1]))


def materialize(A, kA, B, kB, first: int = 0, count: int | None = None):
    """Rows [first, first+count) of J (key ascending, then A order, then B order)."""
    lib = _load()
    ta, tb = _table(A, kA), _table(B, kB)
    if count is None:
        count = join_rows(kA, kB) - first
    n = ta[2] + tb[2]
    X = np.zeros((max(count, 1), max(n, 1)), dtype=np.float64)
    w = lib.oracle_join_materialize(*ta, *tb, first, count, X)
    return X[:w, :n]


def join_r_materialized(A, kA, B, kB, block_rows: int = 65536):
    """O1: R of QR(J) by Householder over the materialised join (sign-normalised)."""
    lib = _load()
    ta, tb = _table(A, kA), _table(B, kB)
    n = ta[2] + tb[2]
    R = np.zeros((n, n), dtype=np.float64)
    lib.oracle_join_r_materialized(*ta, *tb, block_rows, R)
    return R


def join_r_reduced(A, kA, B, kB, block_rows: int = 65536):
    """O2: R of QR(J) by Householder over the head/tail rows (sign-normalised)."""
    lib = _load()
    ta, tb = _table(A, kA), _table(B, kB)
    n = ta[2] + tb[2]
    R = np.zeros((n, n), dtype=np.float64)
    lib.oracle_join_r_reduced(*ta, *tb, block_rows, R)
    return R


def reduce(A, kA, B, kB):
    """Head/tail rows in group order: dict(Hd (G x n), TA (.. x n1), TB (.. x n2))."""
    lib = _load()
    ta, tb = _table(A, kA), _table(B, kB)
    n1, n2 = ta[2], tb[2]
    nta, ntb = _i64(), _i64()
    G = lib.oracle_reduce_sizes(ta[4], ta[1], tb[4], tb[1], ctypes.byref(nta), ctypes.byref(ntb))
    Hd = np.zeros((max(G, 1), max(n1 + n2, 1)))
    TA = np.zeros((max(nta.value, 1), max(n1, 1)))
    TB = np.zeros((max(ntb.value, 1), max(n2, 1)))
    lib.oracle_reduce(*ta, *tb, Hd, TA, TB, ctypes.byref(nta), ctypes.byref(ntb))
    return {"Hd": Hd[:G, :n1 + n2], "TA": TA[:nta.value, :n1], "TB": TB[:ntb.value, :n2]}


def join_gram(A, kA, B, kB):
    """O3: J^T J from per-group sums (no QR)."""
    lib = _load()
    ta, tb = _table(A, kA), _table(B, kB)
    n = ta[2] + tb[2]
    G = np.zeros((n, n), dtype=np.float64)
    lib.oracle_join_gram(*ta, *tb, G)
    return G


def join_least_squares(A, kA, B, kB):
    """Least squares over the join with B's last column as the label (the
    paper's Section 1 names the closed-form solution of linear regression as
    an application of QR): J materialised, then min ||J_x beta - y||_2 by
    numpy's lstsq.  Returns (beta, residual norm)."""
    J = materialize(A, kA, B, kB)
    X, y = J[:, :-1], J[:, -1]
    beta = np.linalg.lstsq(X, y, rcond=None)[0]
    return beta, float(np.linalg.norm(X @ beta - y))


def qr_r(X, block_rows: int = 65536):
    """Householder R (sign-normalised) of a dense row-major matrix X."""
    lib = _load()
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    rows, n = X.shape
    R = np.zeros((n, n), dtype=np.float64)
    for s in range(0, rows, block_rows):
        blk = np.ascontiguousarray(X[s:s + block_rows])
        lib.oracle_qr_update(R, n, blk, blk.shape[0], n)
    lib.oracle_sign_normalise(R, n)
    return R


def jacobi_sigma(R, max_sweeps: int = 60):
    """Singular values (descending) of a square matrix by one-sided Jacobi."""
    lib = _load()
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    n = R.shape[0]
    if n == 0:
        return np.zeros(0)
    s = np.zeros(n, dtype=np.float64)
    sweeps = lib.oracle_jacobi_sigma(R, n, s, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    return s


def jacobi_svd(R, max_sweeps: int = 60):
    """(sigma, V) of a square matrix by one-sided Jacobi with the rotations
    accumulated: sigma descending, column j of V the unit right singular vector
    of sigma_j with its largest-magnitude component positive."""
    lib = _load()
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    n = R.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    s = np.zeros(n, dtype=np.float64)
    V = np.zeros((n, n), dtype=np.float64)
    sweeps = lib.oracle_jacobi_svd(R, n, s, V, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    return s, V


def qr_head(X):
    """H(X) of Section 1 for a dense matrix X (m x n)."""
    lib = _load()
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    m, n = X.shape
    rows = (ctypes.POINTER(ctypes.c_double) * max(m, 1))()
    for i in range(m):
        rows[i] = X[i].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = np.zeros(max(n, 1))
    lib.oracle_qr_head(rows, m, n, out)
    return out[:n]


def qr_tail(X):
    """T(X) of Section 1 for a dense matrix X (m x n): (m-1) x n."""
    lib = _load()
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    m, n = X.shape
    rows = (ctypes.POINTER(ctypes.c_double) * max(m, 1))()
    for i in range(m):
        rows[i] = X[i].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = np.zeros((max(m - 1, 1), max(n, 1)))
    lib.oracle_qr_tail(rows, m, n, out)
    return out[:max(m - 1, 0), :n]


def join_r_sigma(A, kA, B, kB, route: str = "reduced", block_rows: int = 65536):
    """(R, sigma) of the join through route 'materialized' (O1) or 'reduced' (O2)."""
    if route == "materialized":
        R = join_r_materialized(A, kA, B, kB, block_rows)
    elif route == "reduced":
        R = join_r_reduced(A, kA, B, kB, block_rows)
    else:
        raise ValueError(route)
    return R, jacobi_sigma(R)
