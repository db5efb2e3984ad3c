"""Python binding of libfigaro.so (include/figaro.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module turns
torch tensors (device memory, streams) or host arrays into the C structs and
raises :class:`FigaroError` on a non-OK status.  There is no CPU fallback:
importing works without a GPU, but every call needs the CUDA library and a
CUDA device.

Problem (arXiv 2503.23385, Section 1): for tables A (m1 x n1) and B (m2 x n2)
with int32 join keys, R of QR(J) and the singular values of J, where J is the
natural join of A and B, without forming J.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "FigaroError", "PATH_FP64", "PATH_MIXED", "GRAM_AUTO", "GRAM_SIMT", "GRAM_TCGEN05", "library",
    "workspace_size", "join_group", "join_head_tail", "join_qr_r", "join_singular_values", "join_qr_svd",
    "join_qr_svd_host", "batch_join", "get_status", "Solver", "STATUS_NAMES", "event_array", "kernel_launches",
    "host_workspace_size", "PHASES", "NUM_PHASE_EVENTS", "join_singular_values_fixed", "FIXED_SCRATCH_BYTES",
    "BatchSolver", "FLAG_AUTOTUNE", "join_least_squares", "LsqSolver", "join_svd", "get_info",
    "FLAG_ALLOW_RANK_DEFICIENT", "FLAG_SHIFTED_CHOLQR3", "FLAG_PRESORTED", "FLAG_SIGMA_DQDS",
    "triangular_singular_values",
]

PATH_FP64, PATH_MIXED = 0, 1
GRAM_AUTO, GRAM_SIMT, GRAM_TCGEN05 = 0, 1, 2
F32, F64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
FLAG_HOST_OUTPUT = 1
FLAG_AUTOTUNE = 1 << 2
FLAG_ALLOW_RANK_DEFICIENT = 1 << 3
FLAG_SHIFTED_CHOLQR3 = 1 << 4
FLAG_PRESORTED = 1 << 5
FLAG_SIGMA_DQDS = 1 << 6  # sigma by bidiagonalisation and dqds instead of one-sided Jacobi
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "WORKSPACE_TOO_SMALL", 3: "CUDA", 4: "NOT_SPD",
                5: "NO_CONVERGENCE", 6: "DEVICE_TIMEOUT", 7: "UNSUPPORTED", 8: "RANK_DEFICIENT"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libfigaro.so")
_lib = None
_lock = threading.Lock()


class FigaroError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        name = STATUS_NAMES.get(self.status, str(status))
        msg = _lib.figaro_status_string(self.status).decode() if _lib is not None else name
        super().__init__(f"{where}: FIGARO_ERR_{name} ({msg})" if where else f"FIGARO_ERR_{name} ({msg})")


class Table(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("key", ctypes.c_void_p), ("m", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("n", ctypes.c_int32), ("dtype", ctypes.c_int32), ("memory", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("gram_engine", ctypes.c_int32), ("max_jacobi_sweeps", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("spin_limit", ctypes.c_int64), ("rank_tol", ctypes.c_double),
                ("phase_events", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("num_runs_a", ctypes.c_int64), ("num_runs_b", ctypes.c_int64), ("num_groups", ctypes.c_int64),
                ("reduced_rows", ctypes.c_int64), ("jacobi_sweeps", ctypes.c_int32),
                ("dependent_columns", ctypes.c_int32)]


class Grouping(ctypes.Structure):
    _fields_ = [("perm", ctypes.c_void_p), ("sorted_key", ctypes.c_void_p), ("run_key", ctypes.c_void_p),
                ("run_offset", ctypes.c_void_p), ("other_count", ctypes.c_void_p), ("num_runs", ctypes.c_void_p)]


EXPORTS = ["figaro_default_options", "figaro_workspace_size", "figaro_join_group", "figaro_join_head_tail",
           "figaro_join_qr_r", "figaro_join_singular_values", "figaro_batch_workspace_size", "figaro_batch_join",
           "figaro_get_status", "figaro_get_info", "figaro_status_string", "figaro_version",
           "figaro_kernel_launches", "figaro_join_singular_values_fixed", "figaro_triangular_singular_values"]
FIXED_SCRATCH_BYTES = 32 << 20
NUM_PHASE_EVENTS = 9
PHASES = ["grouping", "ht_carry", "head_tail", "gram1", "chol1", "gram2", "chol2", "jacobi"]
FLAG_TEST_WITHHOLD = 1 << 8


def library(build_if_missing: bool = True) -> ctypes.CDLL:
    """The loaded CUDA library (built in-tree with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import _build
            _build.build()
        if not os.path.exists(_LIB_PATH):
            raise FigaroError(3, f"CUDA library missing at {_LIB_PATH}")
        lib = ctypes.CDLL(_LIB_PATH)
        P, I64, I32 = ctypes.POINTER, ctypes.c_int64, ctypes.c_int32
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        lib.figaro_default_options.argtypes = [P(Options)]
        lib.figaro_workspace_size.argtypes = [P(Table), P(Table), P(Options), P(sz)]
        lib.figaro_join_group.argtypes = [P(Table), P(Table), P(Options), P(Grouping), P(Grouping), vp, vp, sz, vp]
        lib.figaro_join_head_tail.argtypes = [P(Table), P(Table), P(Options), vp, vp, vp, vp, sz, vp]
        lib.figaro_join_qr_r.argtypes = [P(Table), P(Table), P(Options), vp, I64, vp, sz, vp]
        lib.figaro_join_singular_values.argtypes = [P(Table), P(Table), P(Options), vp, vp, I64, vp, sz, vp]
        lib.figaro_join_singular_values_fixed.argtypes = [P(Table), P(Table), P(Options), vp, vp, I64, P(vp), vp]
        lib.figaro_batch_workspace_size.argtypes = [I32, P(Table), P(Table), P(Options), P(sz)]
        lib.figaro_triangular_singular_values.argtypes = [vp, I64, I64, I32, I32, vp, vp, vp]
        lib.figaro_batch_join.argtypes = [I32, P(Table), P(Table), P(Options), P(vp), P(vp), vp, sz, vp]
        lib.figaro_get_status.argtypes = [vp, vp]
        lib.figaro_get_info.argtypes = [vp, vp, P(Info)]
        lib.figaro_status_string.argtypes = [ctypes.c_int]
        lib.figaro_status_string.restype = ctypes.c_char_p
        lib.figaro_version.restype = I32
        lib.figaro_kernel_launches.restype = I64
        for name in EXPORTS:
            if name not in ("figaro_status_string", "figaro_version", "figaro_kernel_launches"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != 0:
        raise FigaroError(status, where)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _device_table(x, key) -> Table:
    torch = _torch()
    if not (x.is_cuda and key.is_cuda):
        raise ValueError("device tables need CUDA tensors (use join_qr_svd_host for host buffers)")
    if x.dim() != 2 or key.dim() != 1 or key.shape[0] != x.shape[0]:
        raise ValueError("x must be (m, n) and key (m,)")
    if x.dtype not in (torch.float32, torch.float64) or key.dtype != torch.int32:
        raise ValueError("x must be float32/float64 and key int32")
    m, n = x.shape
    if m > 0 and n > 1 and x.stride(1) != 1:
        raise ValueError("x must be row-major (unit column stride)")
    ld = x.stride(0) if m > 1 else n
    return Table(x.data_ptr() if m else None, key.data_ptr() if m else None, m, max(ld, n), n,
                 F64 if x.dtype == torch.float64 else F32, MEM_DEVICE, 0)


def _host_table(x, key) -> Table:
    """Host table from a numpy array or a (pinned) CPU torch tensor; the
    caller keeps the buffers alive for the duration of the stream work."""
    import numpy as np
    if hasattr(x, "data_ptr"):
        m, n = x.shape
        ptr = x.data_ptr()
        dt = F64 if str(x.dtype) == "torch.float64" else F32
        kptr = key.data_ptr()
        ld = x.stride(0) if m > 1 else n
    else:
        x = np.asarray(x)
        key = np.asarray(key)
        if not x.flags.c_contiguous or not key.flags.c_contiguous or key.dtype != np.int32:
            raise ValueError("host arrays must be C-contiguous; keys int32")
        m, n = x.shape
        ptr, kptr = x.ctypes.data, key.ctypes.data
        dt = F64 if x.dtype == np.float64 else F32
        ld = n
    return Table(ptr if m else None, kptr if m else None, m, max(ld, n), n, dt, MEM_HOST, 0)


def _options(path=PATH_MIXED, gram_engine=GRAM_AUTO, max_jacobi_sweeps=0, flags=0, spin_limit=0, rank_tol=0.0,
             phase_events=None):
    """phase_events: None or a ctypes array of NUM_PHASE_EVENTS cudaEvent_t handles."""
    if isinstance(path, str):
        path = {"mixed": PATH_MIXED, "fp64": PATH_FP64}[path]
    ev = ctypes.cast(phase_events, ctypes.c_void_p) if phase_events is not None else None
    return Options(int(path), int(gram_engine), int(max_jacobi_sweeps), int(flags), int(spin_limit), float(rank_tol),
                   ev)


def event_array(events):
    """ctypes array of raw cudaEvent_t handles from torch.cuda.Event objects
    (torch creates the CUDA event at its first record, so each is recorded once)."""
    arr = (ctypes.c_void_p * len(events))()
    for i, e in enumerate(events):
        if not e.cuda_event:
            e.record()
        arr[i] = e.cuda_event
    _torch().cuda.synchronize()
    return arr


def kernel_launches() -> int:
    return int(library().figaro_kernel_launches())


def workspace_size(A, B, **opts) -> int:
    """Workspace bytes for tables A = (x, key), B = (x, key) (device tensors)."""
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    out = ctypes.c_size_t(0)
    _check(lib.figaro_workspace_size(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o), ctypes.byref(out)),
           "figaro_workspace_size")
    return int(out.value)


def _workspace(nbytes, device, workspace=None):
    torch = _torch()
    if workspace is not None and workspace.numel() >= nbytes:
        return workspace
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def join_group(A, B, stream=None, workspace=None, **opts):
    """Key grouping of both tables (stable sort, runs, partner run sizes)."""
    torch = _torch()
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    dev = A[0].device
    ws = _workspace(workspace_size(A, B, **opts), dev, workspace)
    res = []
    gs = []
    for t in (ta, tb):
        m = t.m
        d = {"perm": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
             "sorted_key": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
             "run_key": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
             "run_offset": torch.empty(m + 1, dtype=torch.int32, device=dev),
             "other_count": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
             "num_runs": torch.zeros(1, dtype=torch.int64, device=dev)}
        res.append(d)
        gs.append(Grouping(*(d[k].data_ptr() for k in ("perm", "sorted_key", "run_key", "run_offset",
                                                        "other_count", "num_runs"))))
    ng = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib.figaro_join_group(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o), ctypes.byref(gs[0]),
                                 ctypes.byref(gs[1]), ctypes.c_void_p(ng.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                 ws.numel(), _stream_handle(stream)), "figaro_join_group")
    out = []
    for d, t in zip(res, (ta, tb)):
        U = int(d["num_runs"].item())
        m = t.m
        out.append({"perm": d["perm"][:m], "sorted_key": d["sorted_key"][:m], "run_key": d["run_key"][:U],
                    "run_offset": d["run_offset"][:U + 1], "other_count": d["other_count"][:U], "num_runs": U})
    return out[0], out[1], int(ng.item())


def join_head_tail(A, B, stream=None, workspace=None, **opts):
    """The reduced matrix in per-row slots: (head [m1 x n], tail_a [m1 x n1], tail_b [m2 x n2])."""
    torch = _torch()
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    dev = A[0].device
    dt = torch.float64 if o.path == PATH_FP64 else torch.float32
    n1, n2 = ta.n, tb.n
    head = torch.zeros((max(ta.m, 1), n1 + n2), dtype=dt, device=dev)
    tail_a = torch.zeros((max(ta.m, 1), n1), dtype=dt, device=dev)
    tail_b = torch.zeros((max(tb.m, 1), n2), dtype=dt, device=dev)
    ws = _workspace(workspace_size(A, B, **opts), dev, workspace)
    _check(lib.figaro_join_head_tail(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                     ctypes.c_void_p(head.data_ptr()), ctypes.c_void_p(tail_a.data_ptr()),
                                     ctypes.c_void_p(tail_b.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                     _stream_handle(stream)), "figaro_join_head_tail")
    return head[:ta.m], tail_a[:ta.m], tail_b[:tb.m]


class Solver:
    """Reusable workspace + outputs for repeated calls with fixed shapes."""

    def __init__(self, A, B, **opts):
        torch = _torch()
        self.opts = opts
        self.lib = library()
        self.dev = A[0].device
        self.nbytes = workspace_size(A, B, **opts)
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=self.dev)
        n = A[0].shape[1] + B[0].shape[1]
        self.n = n
        self.R = torch.zeros((n, n), dtype=torch.float64, device=self.dev)
        self.sigma = torch.zeros(n, dtype=torch.float64, device=self.dev)

    def __call__(self, A, B, stream=None, want_r=True, want_sigma=True, record_phases=True):
        """record_phases=False leaves out the phase events given at construction."""
        ta, tb = _device_table(*A), _device_table(*B)
        opts = self.opts if record_phases else {k: v for k, v in self.opts.items() if k != "phase_events"}
        o = _options(**opts)
        s = _stream_handle(stream)
        ws = ctypes.c_void_p(self.ws.data_ptr())
        if want_sigma:
            rp = ctypes.c_void_p(self.R.data_ptr()) if want_r else None
            _check(self.lib.figaro_join_singular_values(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                                        ctypes.c_void_p(self.sigma.data_ptr()), rp, self.n, ws,
                                                        self.nbytes, s), "figaro_join_singular_values")
        else:
            _check(self.lib.figaro_join_qr_r(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                             ctypes.c_void_p(self.R.data_ptr()), self.n, ws, self.nbytes, s),
                   "figaro_join_qr_r")
        return self.R, self.sigma

    def status(self, stream=None) -> int:
        return get_status(self.ws, stream)

    def info(self, stream=None) -> dict:
        return get_info(self.ws, stream)


class LsqSolver(Solver):
    """Reusable workspace and outputs for repeated least-squares calls
    (figaro_join_least_squares: B's last column is the label)."""

    def __init__(self, A, B, **opts):
        super().__init__(A, B, **opts)
        torch = _torch()
        self.beta = torch.zeros(max(self.n - 1, 1), dtype=torch.float64, device=self.dev)
        self.residual = torch.zeros(1, dtype=torch.float64, device=self.dev)

    def __call__(self, A, B, stream=None, record_phases=True, **_):
        ta, tb = _device_table(*A), _device_table(*B)
        opts = self.opts if record_phases else {k: v for k, v in self.opts.items() if k != "phase_events"}
        o = _options(**opts)
        _check(self.lib.figaro_join_least_squares(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                                  ctypes.c_void_p(self.beta.data_ptr()),
                                                  ctypes.c_void_p(self.residual.data_ptr()),
                                                  ctypes.c_void_p(self.ws.data_ptr()), self.nbytes,
                                                  _stream_handle(stream)), "figaro_join_least_squares")
        return self.beta, self.residual


def join_qr_r(A, B, stream=None, **opts):
    """R of QR(J) as an (n x n) float64 device tensor."""
    s = Solver(A, B, **opts)
    R, _ = s(A, B, stream=stream, want_r=True, want_sigma=False)
    _check(s.status(stream), "figaro_join_qr_r (device status)")
    return R


def join_singular_values(A, B, stream=None, **opts):
    """Singular values of J (descending float64 device tensor)."""
    s = Solver(A, B, **opts)
    _, sigma = s(A, B, stream=stream, want_r=False, want_sigma=True)
    _check(s.status(stream), "figaro_join_singular_values (device status)")
    return sigma


def join_qr_svd(A, B, stream=None, check_status=True, **opts):
    """(R, sigma) of the join, both float64 device tensors."""
    s = Solver(A, B, **opts)
    R, sigma = s(A, B, stream=stream)
    if check_status:
        _check(s.status(stream), "figaro_join_singular_values (device status)")
    return R, sigma


def join_qr_svd_host(A, B, R_out, sigma_out, workspace, stream=None, **opts):
    """(R, sigma) from HOST tables through the C ABI: the library stages the
    inputs into the workspace (host-to-device copies on `stream`) and copies R
    and sigma back into the host buffers R_out (n x n float64) and sigma_out
    (n,).  Pinned host memory keeps the copies asynchronous.  Returns the
    status of the enqueue; synchronise the stream before reading outputs."""
    lib = library()
    ta, tb = _host_table(*A), _host_table(*B)
    flags = FLAG_HOST_OUTPUT | opts.pop("flags", 0)
    o = _options(flags=flags, **opts)
    n = ta.n + tb.n
    rptr = R_out.data_ptr() if hasattr(R_out, "data_ptr") else R_out.ctypes.data
    sptr = sigma_out.data_ptr() if hasattr(sigma_out, "data_ptr") else sigma_out.ctypes.data
    _check(lib.figaro_join_singular_values(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o), ctypes.c_void_p(sptr),
                                           ctypes.c_void_p(rptr), n, ctypes.c_void_p(workspace.data_ptr()),
                                           workspace.numel(), _stream_handle(stream)), "figaro_join_singular_values")


def triangular_singular_values(R, stream=None):
    """Singular values of upper-triangular FP64 device matrices by
    bidiagonalisation and dqds (figaro_triangular_singular_values).  R is
    (n, n) or (count, n, n), rows contiguous; only the upper triangle is read.
    Returns (sigma, info): sigma (count, n) descending (or (n,)), info the
    dqds transforms per matrix as an int32 device tensor (-1: stopped early)."""
    torch = _torch()
    lib = library()
    single = R.dim() == 2
    Rb = R.unsqueeze(0) if single else R
    if Rb.dtype != torch.float64 or not Rb.is_cuda or Rb.stride(-1) != 1 or Rb.shape[-2] != Rb.shape[-1]:
        raise FigaroError(1, "R must be a float64 CUDA tensor with contiguous rows")
    count, n = Rb.shape[0], Rb.shape[-1]
    sigma = torch.empty((count, n), dtype=torch.float64, device=Rb.device)
    info = torch.empty(count, dtype=torch.int32, device=Rb.device)
    _check(lib.figaro_triangular_singular_values(ctypes.c_void_p(Rb.data_ptr()), Rb.stride(1),
                                                 Rb.stride(0) if count > 1 else 0, n, count,
                                                 ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(info.data_ptr()),
                                                 _stream_handle(stream)), "figaro_triangular_singular_values")
    return (sigma[0], info) if single else (sigma, info)


def join_svd(A, B, stream=None, workspace=None, **opts):
    """(sigma, V, R) of the join as float64 device tensors: sigma descending,
    column j of V the unit right singular vector of sigma_j."""
    torch = _torch()
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    nbytes = workspace_size(A, B, **opts)
    dev = A[0].device
    ws = _workspace(nbytes, dev, workspace)
    n = ta.n + tb.n
    sigma = torch.zeros(n, dtype=torch.float64, device=dev)
    V = torch.zeros((n, n), dtype=torch.float64, device=dev)
    R = torch.zeros((n, n), dtype=torch.float64, device=dev)
    _check(lib.figaro_join_svd(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o), ctypes.c_void_p(sigma.data_ptr()),
                               ctypes.c_void_p(V.data_ptr()), n, ctypes.c_void_p(R.data_ptr()), n,
                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream)), "figaro_join_svd")
    _check(get_status(ws, stream), "figaro_join_svd (device status)")
    return sigma, V, R


def join_least_squares(A, B, stream=None, workspace=None, **opts):
    """Least squares over the join: the label is B's last column.  Returns
    (beta, residual) as float64 device tensors of n - 1 and 1 entries:
    beta minimises ||J_x beta - y||, residual = that minimum."""
    torch = _torch()
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    nbytes = workspace_size(A, B, **opts)
    dev = A[0].device
    ws = _workspace(nbytes, dev, workspace)
    n = ta.n + tb.n
    beta = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=dev)
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    _check(lib.figaro_join_least_squares(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                         ctypes.c_void_p(beta.data_ptr()), ctypes.c_void_p(res.data_ptr()),
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream)),
           "figaro_join_least_squares")
    _check(get_status(ws, stream), "figaro_join_least_squares (device status)")
    return beta, res


def join_singular_values_fixed(A, B, sigma, R=None, stream=None, **opts) -> int:
    """figaro_join_singular_values_fixed: sigma (and R when given) of the
    join into caller-owned float64 device tensors, with the library's own
    fixed scratch (FIXED_SCRATCH_BYTES per device).  Waits for the stream and
    raises FigaroError on a non-OK device status, like the other wrappers.
    Returns the scratch's device address, which the C calls
    figaro_get_status / figaro_get_info accept as their workspace argument."""
    lib = library()
    ta, tb = _device_table(*A), _device_table(*B)
    o = _options(**opts)
    n = ta.n + tb.n
    rp = ctypes.c_void_p(R.data_ptr()) if R is not None else None
    ldr = R.stride(0) if R is not None else n
    scratch = ctypes.c_void_p(0)
    _check(lib.figaro_join_singular_values_fixed(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o),
                                                 ctypes.c_void_p(sigma.data_ptr()), rp, ldr, ctypes.byref(scratch),
                                                 _stream_handle(stream)), "figaro_join_singular_values_fixed")
    _check(lib.figaro_get_status(scratch, _stream_handle(stream)), "figaro_join_singular_values_fixed (device status)")
    return int(scratch.value or 0)


def host_workspace_size(A, B, **opts) -> int:
    lib = library()
    ta, tb = _host_table(*A), _host_table(*B)
    o = _options(**opts)
    out = ctypes.c_size_t(0)
    _check(lib.figaro_workspace_size(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(o), ctypes.byref(out)),
           "figaro_workspace_size")
    return int(out.value)


def batch_join(pairs, stream=None, workspace=None, **opts):
    """Independent instances [(A, B), ...] -> [(R, sigma), ...] in one call."""
    torch = _torch()
    lib = library()
    count = len(pairs)
    TA = (Table * max(count, 1))(*[_device_table(*a) for a, _ in pairs])
    TB = (Table * max(count, 1))(*[_device_table(*b) for _, b in pairs])
    o = _options(**opts)
    need = ctypes.c_size_t(0)
    _check(lib.figaro_batch_workspace_size(count, TA, TB, ctypes.byref(o), ctypes.byref(need)),
           "figaro_batch_workspace_size")
    dev = pairs[0][0][0].device if count else torch.device("cuda")
    ws = _workspace(need.value, dev, workspace)
    outs = []
    Rp = (ctypes.c_void_p * max(count, 1))()
    Sp = (ctypes.c_void_p * max(count, 1))()
    for i, (a, b) in enumerate(pairs):
        n = a[0].shape[1] + b[0].shape[1]
        R = torch.zeros((n, n), dtype=torch.float64, device=dev)
        s = torch.zeros(n, dtype=torch.float64, device=dev)
        outs.append((R, s))
        Rp[i], Sp[i] = R.data_ptr(), s.data_ptr()
    _check(lib.figaro_batch_join(count, TA, TB, ctypes.byref(o), Rp, Sp, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 _stream_handle(stream)), "figaro_batch_join")
    return outs, ws


class BatchSolver:
    """Reusable workspace and outputs for repeated batched calls with fixed
    shapes (figaro_batch_join): nothing is allocated per call, so a call can
    be captured in a CUDA graph and replayed."""

    def __init__(self, pairs, **opts):
        torch = _torch()
        self.lib = library()
        self.opts = opts
        self.count = len(pairs)
        self.TA = (Table * max(self.count, 1))(*[_device_table(*a) for a, _ in pairs])
        self.TB = (Table * max(self.count, 1))(*[_device_table(*b) for _, b in pairs])
        o = _options(**opts)
        need = ctypes.c_size_t(0)
        _check(self.lib.figaro_batch_workspace_size(self.count, self.TA, self.TB, ctypes.byref(o), ctypes.byref(need)),
               "figaro_batch_workspace_size")
        dev = pairs[0][0][0].device if self.count else torch.device("cuda")
        self.ws = _workspace(need.value, dev)
        self.outs = []
        self.Rp = (ctypes.c_void_p * max(self.count, 1))()
        self.Sp = (ctypes.c_void_p * max(self.count, 1))()
        for i, (a, b) in enumerate(pairs):
            n = a[0].shape[1] + b[0].shape[1]
            R = torch.zeros((n, n), dtype=torch.float64, device=dev)
            sg = torch.zeros(n, dtype=torch.float64, device=dev)
            self.outs.append((R, sg))
            self.Rp[i], self.Sp[i] = R.data_ptr(), sg.data_ptr()

    def __call__(self, stream=None, phase_events=None):
        o = _options(phase_events=phase_events, **self.opts)
        _check(self.lib.figaro_batch_join(self.count, self.TA, self.TB, ctypes.byref(o), self.Rp, self.Sp,
                                          ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream_handle(stream)),
               "figaro_batch_join")
        return self.outs

    def schedule(self) -> dict:
        """The batch schedule in use (tuned by a FLAG_AUTOTUNE call, else the defaults)."""
        o = _options(**self.opts)
        rpc, hts = ctypes.c_int64(0), ctypes.c_int32(0)
        _check(self.lib.figaro_batch_schedule(self.count, self.TA, self.TB, ctypes.byref(o), ctypes.byref(rpc),
                                              ctypes.byref(hts)), "figaro_batch_schedule")
        return {"gram_rows_per_cta": int(rpc.value), "ht_ctas_per_sm": int(hts.value)}

    def status(self, stream=None) -> int:
        """Waits for the stream; the first non-OK device status among the instances."""
        o = _options(**self.opts)
        return int(self.lib.figaro_batch_get_status(self.count, self.TA, self.TB, ctypes.byref(o),
                                                    ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream)))


def get_info(workspace, stream=None) -> dict:
    """Key runs, key groups, reduced rows, Jacobi sweeps and dependent columns
    (zero rows of R) of the last call."""
    lib = library()
    out = Info()
    _check(lib.figaro_get_info(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream), ctypes.byref(out)),
           "figaro_get_info")
    return {f: int(getattr(out, f)) for f, _ in Info._fields_}


def get_status(workspace, stream=None) -> int:
    """Waits for the stream and returns the device-side status code."""
    lib = library()
    return int(lib.figaro_get_status(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream)))
