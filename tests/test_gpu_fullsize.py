"""The benchmark workloads at full size against the FP64 oracle, through the C
ABI and in the launch configuration the benchmark times.

* c1 (1e6 + 1e6 rows, 16 + 16 FP32 features, 1e4 uniform keys): grouping
  bit-exact against the oracle's stable sort; R and sigma of both paths
  against the reduced-matrix oracle O2, from a direct call and from the CUDA
  graph the benchmark replays.
* c2 (4e6 + 2e6 rows, 32 + 32 features, Zipf(1.2) keys over 1e5 ids: runs of
  up to 7.9e5 rows, most rows in runs that cross many head/tail chunks):
  grouping bit-exact, R and sigma of both paths against O2.
* c3 (the batching workload): 128 instances with their full row counts, every
  instance against O2, both paths.

Bars: bit-exact grouping; relative Frobenius error <= 1e-10 (FP64 path) and
<= 1e-6 (mixed path) for R and sigma.  These cases take from seconds (c1) to
about a minute (the oracle on c2's 6e6 reduced rows) each.
"""
import numpy as np
import pytest

import oracle
from workloads import batch_instances, config

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def check_grouping(fg, torch, A, B):
    ga, gb, G = fg.join_group(dev(torch, A), dev(torch, B))
    oa, ob = oracle.group(A.key), oracle.group(B.key)
    for g, o in ((ga, oa), (gb, ob)):
        assert np.array_equal(g["perm"].cpu().numpy(), o["perm"])
        assert np.array_equal(g["sorted_key"].cpu().numpy(), o["sorted_key"])
        assert np.array_equal(g["run_key"].cpu().numpy(), o["uniq"])
        assert np.array_equal(g["run_offset"].cpu().numpy(), o["offset"])
    assert G == oracle.match(oa, ob)["key"].size
    return oa, ob


def graph_call(fg, torch, a, b, path):
    """R and sigma from a replay of the CUDA graph of one call, as bench.py
    times it (a Solver with fixed buffers, captured once, replayed)."""
    solver = fg.Solver(a, b, path=path)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        solver(a, b, stream=s)  # warm-up outside the capture (first launches, attributes)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        solver(a, b, stream=s, record_phases=False)
    solver.R.zero_()
    solver.sigma.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert solver.status() == 0
    return solver.R.cpu().numpy(), solver.sigma.cpu().numpy()


def test_c1_full_size(fg, torch):
    A, B = config("c1")
    oa, ob = check_grouping(fg, torch, A, B)
    assert oa["uniq"].size > 9000
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    a, b = dev(torch, A), dev(torch, B)
    for path in ("fp64", "mixed"):
        R, s = fg.join_qr_svd(a, b, path=path)
        R, s = R.cpu().numpy(), s.cpu().numpy()
        assert rel(R, Rref) <= TOL[path] and rel(s, sref) <= TOL[path], (path, rel(R, Rref), rel(s, sref))
        Rg, sg = graph_call(fg, torch, a, b, path)
        assert np.array_equal(Rg, R) and np.array_equal(sg, s), path
        # sigma by bidiagonalisation and dqds on the same join
        _, sd = fg.join_qr_svd(a, b, path=path, flags=fg.FLAG_SIGMA_DQDS)
        assert rel(sd.cpu().numpy(), sref) <= TOL[path], (path, "dqds", rel(sd.cpu().numpy(), sref))


def test_c2_full_size_zipf(fg, torch):
    A, B = config("c2")
    oa, ob = check_grouping(fg, torch, A, B)
    assert oa["count"].max() > 500_000  # the hottest key's run crosses thousands of chunks
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    a, b = dev(torch, A), dev(torch, B)
    for path in ("fp64", "mixed"):
        R, s = fg.join_qr_svd(a, b, path=path)
        R, s = R.cpu().numpy(), s.cpu().numpy()
        assert rel(R, Rref) <= TOL[path] and rel(s, sref) <= TOL[path], (path, rel(R, Rref), rel(s, sref))
        _, sd = fg.join_qr_svd(a, b, path=path, flags=fg.FLAG_SIGMA_DQDS)
        assert rel(sd.cpu().numpy(), sref) <= TOL[path], (path, "dqds", rel(sd.cpu().numpy(), sref))


def test_c3_128_uncapped_instances(fg, torch):
    inst = batch_instances(count=128, seed=0x250323385 + 3000)
    assert max(max(a.m, b.m) for a, b in inst) > 50_000
    refs = [oracle.join_r_sigma(a.x, a.key, b.x, b.key, route="reduced") for a, b in inst]
    pairs = [(dev(torch, a), dev(torch, b)) for a, b in inst]
    for path in ("fp64", "mixed"):
        outs, ws = fg.batch_join(pairs, path=path)
        torch.cuda.synchronize()
        worst = 0.0
        for (Rref, sref), (R, s) in zip(refs, outs):
            eR, es = rel(R.cpu().numpy(), Rref), rel(s.cpu().numpy(), sref)
            worst = max(worst, eR, es)
        assert worst <= TOL[path], (path, worst)
        # the batch with sigma by bidiagonalisation and dqds
        outs, ws = fg.batch_join(pairs, path=path, flags=fg.FLAG_SIGMA_DQDS)
        torch.cuda.synchronize()
        worst = max(rel(s.cpu().numpy(), sref) for (_, sref), (_, s) in zip(refs, outs))
        assert worst <= TOL[path], (path, "dqds", worst)
