"""figaro_batch_join: many independent instances, one launch per phase.

The batched launches must give each instance the result its own call gives
(up to the order of the Gram partial sums, which follows the batch's
schedule: 1e-12 on the plain FP64 path, the mixed bar on the mixed path) and
stay within the usual bars of the FP64 oracle.  Instances the batched launches do not take (wide joins)
run one after another inside the same call.
"""
import ctypes

import numpy as np
import pytest

import oracle
from workloads import batch_instances, make_pair

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


@pytest.fixture(scope="module")
def c3_small():
    """40 instances shaped like the batching workload (m log-uniform, widths
    from {8, 16, 32, 64}, keys over min(m1, m2) / 10 ids), rows capped at
    5,000 so that the oracle stays quick."""
    return batch_instances(count=40, seed=0x250323385 + 3000, max_rows=5000)


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_batch_matches_oracle(fg, torch, c3_small, path):
    outs, _ = fg.batch_join([(dev(torch, a), dev(torch, b)) for a, b in c3_small], path=path)
    torch.cuda.synchronize()
    for (a, b), (R, s) in zip(c3_small, outs):
        Rref, sref = oracle.join_r_sigma(a.x, a.key, b.x, b.key, route="reduced")
        eR, es = rel(R.cpu().numpy(), Rref), rel(s.cpu().numpy(), sref)
        assert eR <= TOL[path] and es <= TOL[path], (a.x.shape, b.x.shape, eR, es)


def test_batch_fp64_matches_the_single_call(fg, torch, c3_small):
    """The same kernels as one call per instance; only the number of Gram
    partials (hence their summation order) differs."""
    pairs = [(dev(torch, a), dev(torch, b)) for a, b in c3_small[:16]]
    outs, _ = fg.batch_join(pairs, path="fp64")
    for (ta, tb), (R, s) in zip(pairs, outs):
        R1, s1 = fg.join_qr_svd(ta, tb, path="fp64", gram_engine=fg.GRAM_SIMT)
        assert rel(R.cpu().numpy(), R1.cpu().numpy()) <= 1e-12 and rel(s.cpu().numpy(), s1.cpu().numpy()) <= 1e-12


def test_batch_mixed_matches_single_calls(fg, torch, c3_small):
    pairs = [(dev(torch, a), dev(torch, b)) for a, b in c3_small[:16]]
    outs, _ = fg.batch_join(pairs, path="mixed")
    for (ta, tb), (R, s) in zip(pairs, outs):
        R1, s1 = fg.join_qr_svd(ta, tb, path="mixed", gram_engine=fg.GRAM_SIMT)
        assert rel(R.cpu().numpy(), R1.cpu().numpy()) <= 1e-6 and rel(s.cpu().numpy(), s1.cpu().numpy()) <= 1e-6


def test_batch_with_wide_empty_and_skipped_outputs(fg, torch):
    """A wide instance (run on its own inside the call), an instance whose
    table B is empty, one with only R requested and one with only sigma."""
    inst = [make_pair(3000, 100, 2000, 60, 40, np.float32, "normal", seed=701),   # wide: 160 columns
            make_pair(2500, 16, 0, 8, 30, np.float32, "normal", seed=702),        # empty B
            make_pair(1800, 8, 2200, 24, 50, np.float32, "normal", seed=703),
            make_pair(4000, 32, 3000, 32, 80, np.float32, "normal", seed=704)]
    lib = fg.library()
    tabs = [(dev(torch, a), dev(torch, b)) for a, b in inst]
    TA = (fg.Table * 4)(*[fg._device_table(*a) for a, _ in tabs])
    TB = (fg.Table * 4)(*[fg._device_table(*b) for _, b in tabs])
    o = fg._options(path=fg.PATH_MIXED)
    need = ctypes.c_size_t(0)
    assert lib.figaro_batch_workspace_size(4, TA, TB, ctypes.byref(o), ctypes.byref(need)) == 0
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    ns = [a.n + b.n for a, b in inst]
    Rs = [torch.full((n, n), -7.0, dtype=torch.float64, device="cuda") for n in ns]
    ss = [torch.full((n,), -7.0, dtype=torch.float64, device="cuda") for n in ns]
    Rp = (ctypes.c_void_p * 4)(Rs[0].data_ptr(), Rs[1].data_ptr(), Rs[2].data_ptr(), None)
    Sp = (ctypes.c_void_p * 4)(ss[0].data_ptr(), ss[1].data_ptr(), None, ss[3].data_ptr())
    assert lib.figaro_batch_join(4, TA, TB, ctypes.byref(o), Rp, Sp, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 None) == 0
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(inst):
        Rref, sref = oracle.join_r_sigma(a.x, a.key, b.x, b.key, route="reduced")
        if i != 3:
            assert rel(Rs[i].cpu().numpy(), Rref) <= 1e-6
        else:
            assert torch.all(Rs[i] == -7.0)  # not requested: untouched
        if i != 2:
            assert rel(ss[i].cpu().numpy(), sref) <= 1e-6
        else:
            assert torch.all(ss[i] == -7.0)
    assert torch.all(Rs[1] == 0) and torch.all(ss[1] == 0)  # empty join


def test_batch_replays_in_a_cuda_graph(fg, torch, c3_small):
    """The whole batched call captured once and replayed: the per-instance
    plans and job lists travel as kernel arguments inside the graph."""
    pairs = [(dev(torch, a), dev(torch, b)) for a, b in c3_small[:24]]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ref, ws = fg.batch_join(pairs, stream=s)
        s.synchronize()
        ref = [(R.clone(), sg.clone()) for R, sg in ref]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            outs, _ = fg.batch_join(pairs, stream=s, workspace=ws)
        for R, sg in outs:
            R.zero_()
            sg.zero_()
        g.replay()
        s.synchronize()
    for (R0, s0), (R, sg) in zip(ref, outs):
        assert torch.equal(R0, R) and torch.equal(s0, sg)


def test_autotuned_schedule_is_used_and_results_hold(fg, torch, c3_small):
    """A FLAG_AUTOTUNE call times the candidate schedules on the batch, keeps
    the fastest for its shape class, and the results stay within the bar."""
    pairs = [(dev(torch, a), dev(torch, b)) for a, b in c3_small[:20]]
    plain = fg.BatchSolver(pairs, path="mixed")
    assert plain.schedule() == {"gram_rows_per_cta": 4096, "ht_ctas_per_sm": 2}  # nothing tuned yet
    ref = [(R.clone(), s.clone()) for R, s in plain()]
    tuned = fg.BatchSolver(pairs, path="mixed", flags=fg.FLAG_AUTOTUNE)
    outs = tuned()
    assert tuned.status() == 0
    sched = tuned.schedule()
    assert sched["gram_rows_per_cta"] in (1024, 2048, 4096, 8192, 16384, 32768)
    assert sched["ht_ctas_per_sm"] in (1, 2, 4, 8)
    assert plain.schedule() == sched  # same shape class: the cache serves every solver
    for (R0, s0), (R, s) in zip(ref, outs):
        assert rel(R.cpu().numpy(), R0.cpu().numpy()) <= 1e-6 and rel(s.cpu().numpy(), s0.cpu().numpy()) <= 1e-6
