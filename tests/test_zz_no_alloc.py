"""figaro_join_singular_values_fixed (library-owned scratch, no allocation in
the call) against figaro_join_singular_values with a caller workspace, on two
calls in a row through the C ABI.  Collected last so that it also runs after
every other test has used the library on this device."""
import ctypes

import numpy as np
import pytest

from workloads import config, make_pair

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


def test_fixed_scratch_matches_workspace_entry_on_two_calls(fg, torch):
    cases = [
        (config("c0"), "fp64"),
        (make_pair(20_000, 8, 15_000, 8, 700, np.float32, "normal", 20250323), "mixed"),
    ]
    lib = fg.library()
    addrs = []
    got = []
    for (A, B), path in cases:  # two calls in a row on the library's scratch
        a, b = dev(torch, A), dev(torch, B)
        n = A.x.shape[1] + B.x.shape[1]
        R = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        addr = fg.join_singular_values_fixed(a, b, s, R=R, path=path)
        assert addr != 0 and addr % 256 == 0
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert lib.figaro_get_status(ctypes.c_void_p(addr), stream) == 0
        addrs.append(addr)
        got.append((R.cpu().numpy(), s.cpu().numpy()))
    assert addrs[0] == addrs[1]
    for ((A, B), path), (R, s) in zip(cases, got):
        Rw, sw = fg.join_qr_svd(dev(torch, A), dev(torch, B), path=path)
        torch.cuda.synchronize()
        Rw, sw = Rw.cpu().numpy(), sw.cpu().numpy()
        assert np.all(np.isfinite(R)) and np.all(np.isfinite(s))
        assert rel(R, Rw) <= TOL[path], path
        assert rel(s, sw) <= TOL[path], path


def test_fixed_scratch_rejects_inputs_beyond_its_size(fg, torch):
    A, B = make_pair(400_000, 16, 400_000, 16, 5_000, np.float32, "normal", 7)
    a, b = dev(torch, A), dev(torch, B)
    assert fg.workspace_size(a, b) > fg.FIXED_SCRATCH_BYTES
    s = torch.full((32,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FigaroError) as e:
        fg.join_singular_values_fixed(a, b, s)
    assert e.value.status == 2  # FIGARO_ERR_WORKSPACE_TOO_SMALL
    torch.cuda.synchronize()
    assert torch.all(s == -1.0)  # nothing was enqueued
