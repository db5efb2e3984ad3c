"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: key grouping bit-exact; R and sigma within relative Frobenius error
1e-10 on the plain FP64 path and 1e-6 on the mixed path (well-conditioned
inputs); head/tail rows within 1e-12 (FP64) / 2e-6 (FP32) of the row scale.
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


def gpu_r_sigma(fg, torch, A, B, path, **opts):
    R, s = fg.join_qr_svd(dev(torch, A), dev(torch, B), path=path, **opts)
    torch.cuda.synchronize()
    return R.cpu().numpy(), s.cpu().numpy()


def as_f32(T):
    return Table(T.x.astype(np.float32), T.key)


def oracle_ref(A, B, path, route="reduced"):
    """The oracle on the inputs the path computes with: the mixed path rounds
    FP64 features to FP32 on load, so its reference uses those FP32 values."""
    if path == "mixed" and A.x.dtype == np.float64:
        A, B = as_f32(A), as_f32(B)
    return oracle.join_r_sigma(A.x, A.key, B.x, B.key, route=route)


def check_against_oracle(fg, torch, A, B, paths=("fp64", "mixed"), route="reduced", tol=None):
    for path in paths:
        Rref, sref = oracle_ref(A, B, path, route)
        R, s = gpu_r_sigma(fg, torch, A, B, path)
        t = (tol or TOL)[path]
        eR, es = rel(R, Rref), rel(s, sref)
        assert eR <= t and es <= t, f"{path}: err_R={eR:.3e} err_sigma={es:.3e} (tol {t})"
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)


# ------------------------------------------------------------- grouping --

def grouping_cases():
    rng = np.random.default_rng(0)
    i32 = np.iinfo(np.int32)
    yield "c0", config("c0")
    adv = np.array([i32.min, i32.max, 0, -1, 1, i32.min, i32.max, -7] * 50, np.int32)
    yield "adversarial", (Table(np.ones((adv.size, 1), np.float32), adv),
                          Table(np.ones((9, 1), np.float32), np.array([0, i32.max, i32.min, 5, 5, -1, 3, 3, 3], np.int32)))
    yield "all_equal", (Table(np.ones((5000, 2), np.float32), np.full(5000, 42, np.int32)),
                        Table(np.ones((3, 2), np.float32), np.full(3, 42, np.int32)))
    yield "all_distinct", (Table(np.ones((9000, 2), np.float32), rng.permutation(9000).astype(np.int32) * 3 - 5000),
                           Table(np.ones((7000, 2), np.float32), rng.permutation(7000).astype(np.int32) * 2))
    yield "single_row", (Table(np.ones((1, 2), np.float32), np.array([3], np.int32)),
                         Table(np.ones((1, 2), np.float32), np.array([3], np.int32)))
    yield "empty_b", (Table(np.ones((100, 2), np.float32), rng.integers(0, 9, 100).astype(np.int32)),
                      Table(np.ones((0, 2), np.float32), np.zeros(0, np.int32)))
    yield "wide_range", (Table(np.ones((70000, 1), np.float32), rng.integers(i32.min, i32.max, 70000).astype(np.int32)),
                         Table(np.ones((50000, 1), np.float32), rng.integers(-1000, 1000, 50000).astype(np.int32)))
    yield "ragged_tiles", make_pair(4096 * 3 + 17, 2, 4095, 2, 300, np.float32, "normal", seed=3)


@pytest.mark.parametrize("name,tables", list(grouping_cases()), ids=[c[0] for c in grouping_cases()])
def test_grouping_bitexact(fg, torch, name, tables):
    A, B = tables
    ga, gb, G = fg.join_group(dev(torch, A), dev(torch, B))
    oa, ob = oracle.group(A.key), oracle.group(B.key)
    for g, o, other in ((ga, oa, ob), (gb, ob, oa)):
        assert np.array_equal(g["perm"].cpu().numpy(), o["perm"])
        assert np.array_equal(g["sorted_key"].cpu().numpy(), o["sorted_key"])
        assert g["num_runs"] == o["uniq"].size
        assert np.array_equal(g["run_key"].cpu().numpy(), o["uniq"])
        assert np.array_equal(g["run_offset"].cpu().numpy(), o["offset"])
        cnt = dict(zip(other["uniq"].tolist(), other["count"].tolist()))
        exp = np.array([cnt.get(k, 0) for k in o["uniq"].tolist()], np.int32)
        assert np.array_equal(g["other_count"].cpu().numpy(), exp)
    assert G == oracle.match(oa, ob)["key"].size


def test_grouping_is_deterministic(fg, torch):
    A, B = make_pair(200000, 2, 150000, 2, 5000, np.float32, "normal", seed=4)
    r1 = fg.join_group(dev(torch, A), dev(torch, B))
    r2 = fg.join_group(dev(torch, A), dev(torch, B))
    for a, b in zip(r1[:2], r2[:2]):
        assert all(torch.equal(a[k], b[k]) for k in ("perm", "sorted_key", "run_key", "run_offset", "other_count"))


# ------------------------------------------------------------ head/tail --

def gpu_head_tail_in_oracle_order(fg, torch, A, B, path):
    head, ta, tb = fg.join_head_tail(dev(torch, A), dev(torch, B), path=path)
    head, ta, tb = head.double().cpu().numpy(), ta.double().cpu().numpy(), tb.double().cpu().numpy()
    oa, ob = oracle.group(A.key), oracle.group(B.key)
    mt = oracle.match(oa, ob)
    runs_a = {k: u for u, k in enumerate(oa["uniq"].tolist())}
    Hd = np.array([head[runs_a[k]] for k in mt["key"].tolist()]).reshape(-1, A.n + B.n)
    TA = np.vstack([ta[o + 1:o + m] for o, m in zip(mt["offA"], mt["m1"])] or [np.zeros((0, A.n))])
    TB = np.vstack([tb[o + 1:o + m] for o, m in zip(mt["offB"], mt["m2"])] or [np.zeros((0, B.n))])
    # every other slot is zero
    mask_a = np.ones(A.m, bool)
    for o, m in zip(mt["offA"], mt["m1"]):
        mask_a[o + 1:o + m] = False
    assert np.all(ta[mask_a] == 0)
    unmatched = [u for u, k in enumerate(oa["uniq"].tolist()) if k not in set(mt["key"].tolist())]
    assert np.all(head[unmatched] == 0)
    return Hd, TA, TB


@pytest.mark.parametrize("path,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
@pytest.mark.parametrize("shape", [(1000, 4, 1000, 4, 100), (30000, 16, 20000, 16, 50), (5000, 3, 7000, 5, 400),
                                   (20000, 32, 300, 32, 3)])
def test_head_tail_rows(fg, torch, path, tol, shape):
    m1, n1, m2, n2, K = shape
    A, B = make_pair(m1, n1, m2, n2, K, np.float32, "uniform_pm1", seed=m1 + n2)
    ref = oracle.reduce(A.x, A.key, B.x, B.key)
    Hd, TA, TB = gpu_head_tail_in_oracle_order(fg, torch, A, B, path)
    for got, want in ((Hd, ref["Hd"]), (TA, ref["TA"]), (TB, ref["TB"])):
        assert got.shape == want.shape
        scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-300) if want.size else 1
        assert np.max(np.abs(got - want) / scale, initial=0) <= tol


# ------------------------------------------------------------- R, sigma --

def test_c0_matches_materialized_oracle(fg, torch):
    A, B = config("c0")
    check_against_oracle(fg, torch, A, B, route="materialized")


@pytest.mark.parametrize("seed", range(4))
def test_random_joins_with_unmatched_keys(fg, torch, seed):
    rng = np.random.default_rng(50 + seed)
    m1, m2 = rng.integers(200, 20000, 2)
    n1, n2 = rng.integers(1, 12, 2)
    A = Table(rng.standard_normal((m1, n1)), rng.integers(0, 300, m1).astype(np.int32))
    B = Table(rng.standard_normal((m2, n2)), rng.integers(100, 400, m2).astype(np.int32))
    check_against_oracle(fg, torch, A, B)
    A32 = Table(A.x.astype(np.float32), A.key)
    B32 = Table(B.x.astype(np.float32), B.key)
    check_against_oracle(fg, torch, A32, B32)


@pytest.mark.parametrize("m,n", [(100, 4), (400, 16), (1600, 32)])
def test_cartesian_paper_shape(fg, torch, m, n):
    """The paper's own experiment: one key, so J is the Cartesian product."""
    rng = np.random.default_rng(m)
    A = Table(rng.uniform(0, 1, (m, n)).astype(np.float32), np.zeros(m, np.int32))
    B = Table(rng.uniform(0, 1, (m, n)).astype(np.float32), np.zeros(m, np.int32))
    # U(0,1) columns share a large mean: well above 1 condition number; the
    # mixed bar is checked with the condition number in mind below
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key)
    R, s = gpu_r_sigma(fg, torch, A, B, "fp64")
    assert rel(R, Rref) <= 1e-10 and rel(s, sref) <= 1e-10
    R, s = gpu_r_sigma(fg, torch, A, B, "mixed")
    assert rel(R, Rref) <= 1e-6 and rel(s, sref) <= 1e-6


def test_groups_spanning_many_chunks(fg, torch):
    """Few keys, long runs: the segmented scan crosses many chunks."""
    A, B = make_pair(200000, 16, 150000, 16, 3, np.float32, "normal", seed=9)
    check_against_oracle(fg, torch, A, B)


def test_one_to_one_and_widths(fg, torch):
    rng = np.random.default_rng(77)
    m = 5000
    A = Table(rng.standard_normal((m, 7)).astype(np.float32), rng.permutation(m).astype(np.int32))
    B = Table(rng.standard_normal((m, 9)).astype(np.float32), rng.permutation(m).astype(np.int32))
    check_against_oracle(fg, torch, A, B)
    A, B = make_pair(3000, 64, 2500, 64, 30, np.float32, "normal", seed=78)
    check_against_oracle(fg, torch, A, B)
    A, B = make_pair(3000, 1, 2500, 1, 30, np.float64, "normal", seed=79)
    check_against_oracle(fg, torch, A, B)


def test_strided_rows(fg, torch):
    """Leading dimension larger than the width (views of wider tables)."""
    A, B = make_pair(4000, 12, 3000, 10, 50, np.float32, "normal", seed=80)
    Rref, sref = oracle.join_r_sigma(A.x[:, :9], A.key, B.x[:, :7], B.key)
    ta = (torch.from_numpy(A.x).cuda()[:, :9], torch.from_numpy(A.key).cuda())
    tb = (torch.from_numpy(B.x).cuda()[:, :7], torch.from_numpy(B.key).cuda())
    for path in ("fp64", "mixed"):
        R, s = fg.join_qr_svd(ta, tb, path=path)
        assert rel(R.cpu().numpy(), Rref) <= TOL[path] and rel(s.cpu().numpy(), sref) <= TOL[path]


def test_empty_and_short_joins(fg, torch):
    rng = np.random.default_rng(81)
    A = Table(rng.standard_normal((50, 3)), np.zeros(50, np.int32))
    B = Table(rng.standard_normal((40, 2)), np.ones(40, np.int32))
    for path in ("fp64", "mixed"):
        R, s = gpu_r_sigma(fg, torch, A, B, path)
        assert np.all(R == 0) and np.all(s == 0)
    # short join: 2 join rows, 5 columns -> R has 3 zero rows (accepted with
    # the flag; without it the call reports FIGARO_ERR_RANK_DEFICIENT, see
    # test_gpu_conditioning.py)
    A = Table(rng.standard_normal((5, 3)), np.array([0, 1, 2, 3, 4], np.int32))
    B = Table(rng.standard_normal((4, 2)), np.array([0, 9, 9, 1], np.int32))
    for path in ("fp64", "mixed"):
        Rref, sref = oracle_ref(A, B, path, route="materialized")
        R, s = gpu_r_sigma(fg, torch, A, B, path, flags=fg.FLAG_ALLOW_RANK_DEFICIENT)
        assert rel(R, Rref) <= TOL[path] and rel(s, sref) <= TOL[path]
        assert np.all(R[2:] == 0)
    # an empty table
    A0 = Table(np.zeros((0, 3)), np.zeros(0, np.int32))
    R, s = gpu_r_sigma(fg, torch, A0, B, "fp64")
    assert np.all(R == 0) and np.all(s == 0)


def test_results_are_deterministic(fg, torch):
    A, B = make_pair(100000, 16, 80000, 16, 1000, np.float32, "normal", seed=82)
    for path in ("fp64", "mixed"):
        R1, s1 = gpu_r_sigma(fg, torch, A, B, path)
        R2, s2 = gpu_r_sigma(fg, torch, A, B, path)
        assert np.array_equal(R1, R2) and np.array_equal(s1, s2)


def test_host_buffers_match_device_call(fg, torch):
    A, B = make_pair(20000, 8, 15000, 8, 500, np.float32, "normal", seed=83)
    Rd, sd = gpu_r_sigma(fg, torch, A, B, "mixed")
    n = 16
    nbytes = fg.host_workspace_size((A.x, A.key), (B.x, B.key))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    R = torch.zeros((n, n), dtype=torch.float64).pin_memory()
    s = torch.zeros(n, dtype=torch.float64).pin_memory()
    fg.join_qr_svd_host((A.x, A.key), (B.x, B.key), R, s, ws)
    torch.cuda.synchronize()
    assert np.array_equal(R.numpy(), Rd) and np.array_equal(s.numpy(), sd)


@pytest.mark.parametrize("shape", [(50000, 16, 40000, 16, 500), (30000, 32, 20000, 32, 300), (20000, 4, 30000, 8, 100),
                                   (9000, 12, 7000, 20, 50)])
def test_gram_engines_agree_with_oracle(fg, torch, shape):
    """The tensor-core (tcgen05, 3xTF32) and CUDA-core Gram engines both meet
    the mixed-path bar, and agree with each other."""
    m1, n1, m2, n2, K = shape
    A, B = make_pair(m1, n1, m2, n2, K, np.float32, "normal", seed=m1 + n1)
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key)
    out = {}
    for eng in (fg.GRAM_SIMT, fg.GRAM_TCGEN05):
        R, s = fg.join_qr_svd(dev(torch, A), dev(torch, B), path="mixed", gram_engine=eng)
        R, s = R.cpu().numpy(), s.cpu().numpy()
        assert rel(R, Rref) <= 1e-6 and rel(s, sref) <= 1e-6, (eng, rel(R, Rref), rel(s, sref))
        out[eng] = R
    assert rel(out[fg.GRAM_SIMT], out[fg.GRAM_TCGEN05]) <= 1e-6


@pytest.mark.parametrize("shape", [(20000, 64, 15000, 64, 300), (9001, 32, 12345, 64, 77), (5000, 64, 6000, 8, 40)],
                         ids=["128", "96-ragged", "72"])
def test_wide_q_tail_block_on_tensor_cores(fg, torch, shape):
    """Joins of 65 to 128 columns: the Gram blocks with n output columns, more
    than the narrow tensor-core engines take (the head rows in both passes,
    pass 2 of the A tails after the tensor-core formation Q = X W), run the
    tile Gram.  Both engine settings meet the mixed-path bar and agree; a batch
    holding the same join (table launches of the same kernels) does too."""
    m1, n1, m2, n2, K = shape
    A, B = make_pair(m1, n1, m2, n2, K, np.float32, "normal", seed=m1 + n2)
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key)
    out = {}
    for eng in (fg.GRAM_SIMT, fg.GRAM_AUTO):
        R, s = fg.join_qr_svd(dev(torch, A), dev(torch, B), path="mixed", gram_engine=eng)
        R, s = R.cpu().numpy(), s.cpu().numpy()
        assert rel(R, Rref) <= 1e-6 and rel(s, sref) <= 1e-6, (eng, rel(R, Rref), rel(s, sref))
        out[eng] = R
    assert rel(out[fg.GRAM_SIMT], out[fg.GRAM_AUTO]) <= 1e-6
    small = make_pair(3000, 8, 2000, 16, 30, np.float32, "normal", seed=7)
    outs, ws = fg.batch_join([(dev(torch, A), dev(torch, B)), (dev(torch, small[0]), dev(torch, small[1]))])
    torch.cuda.synchronize()
    Rb, sb = outs[0]
    assert rel(Rb.cpu().numpy(), Rref) <= 1e-6 and rel(sb.cpu().numpy(), sref) <= 1e-6
    R2, s2 = oracle.join_r_sigma(small[0].x, small[0].key, small[1].x, small[1].key)
    assert rel(outs[1][0].cpu().numpy(), R2) <= 1e-6 and rel(outs[1][1].cpu().numpy(), s2) <= 1e-6


@pytest.mark.parametrize("shape", [(20000, 16, 15000, 8, 300), (257, 8, 1000, 16, 20), (9001, 16, 123, 16, 40),
                                   (3000, 8, 4000, 32, 50)],
                         ids=["16+8", "ragged-tile", "short-B", "8+32-one-table"])
def test_tail_gram_inside_head_tail_stream(fg, torch, shape):
    """Mixed path, FP32 tables of 8 or 16 columns, automatic engine: the
    head/tail stream also accumulates the pass-1 Gram of those tables' tails
    (3xTF32 warp MMAs on each tile), so pass 1 launches the Gram only for the
    head rows and the other tables.  The result meets the mixed-path bar and
    agrees with the tensor-core engine setting, whose pass 1 reads the tails;
    the automatic call makes fewer launches."""
    m1, n1, m2, n2, K = shape
    A, B = make_pair(m1, n1, m2, n2, K, np.float32, "normal", seed=m1 + 3 * n2)
    Rref, sref = oracle.join_r_sigma(A.x, A.key, B.x, B.key)
    out, launches = {}, {}
    for eng in (fg.GRAM_TCGEN05, fg.GRAM_AUTO):
        before = fg.kernel_launches()
        R, s = fg.join_qr_svd(dev(torch, A), dev(torch, B), path="mixed", gram_engine=eng)
        torch.cuda.synchronize()
        launches[eng] = fg.kernel_launches() - before
        R, s = R.cpu().numpy(), s.cpu().numpy()
        assert rel(R, Rref) <= 1e-6 and rel(s, sref) <= 1e-6, (eng, rel(R, Rref), rel(s, sref))
        out[eng] = R
    assert rel(out[fg.GRAM_TCGEN05], out[fg.GRAM_AUTO]) <= 1e-6
    assert launches[fg.GRAM_AUTO] < launches[fg.GRAM_TCGEN05], launches


# ---------------------------------------------------------- status codes --

def test_status_codes(fg, torch):
    A, B = make_pair(1000, 4, 1000, 4, 10, np.float32, "normal", seed=84)
    ta, tb = dev(torch, A), dev(torch, B)
    with pytest.raises(fg.FigaroError) as e:
        fg.join_qr_svd((ta[0], ta[1]), (tb[0].double(), tb[1]))
    assert e.value.status == 1
    with pytest.raises(fg.FigaroError) as e:
        big = torch.zeros((10, 300), device="cuda")  # 300 + 300 columns: above the 512-column limit
        fg.join_qr_svd((big, torch.zeros(10, dtype=torch.int32, device="cuda")),
                       (big, torch.zeros(10, dtype=torch.int32, device="cuda")))
    assert e.value.status == 7
    solver = fg.Solver(ta, tb)
    solver.nbytes -= 1024
    with pytest.raises(fg.FigaroError) as e:
        solver(ta, tb)
    assert e.value.status == 2
    bad = A.x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(fg.FigaroError) as e:
        fg.join_qr_svd((torch.from_numpy(bad).cuda(), ta[1]), tb)
    assert e.value.status == 4


def test_batch_matches_single_calls(fg, torch):
    pairs = [make_pair(2000 + 500 * i, 4 + 4 * (i % 3), 1500 + 300 * i, 8, 100 + i, np.float32, "normal", seed=90 + i)
             for i in range(5)]
    outs, ws = fg.batch_join([(dev(torch, a), dev(torch, b)) for a, b in pairs])
    torch.cuda.synchronize()
    for (a, b), (R, s) in zip(pairs, outs):
        Rref, sref = oracle.join_r_sigma(a.x, a.key, b.x, b.key)
        assert rel(R.cpu().numpy(), Rref) <= 1e-6 and rel(s.cpu().numpy(), sref) <= 1e-6


def test_withheld_lookback_word_times_out_and_context_survives(fg, torch):
    """Fault injection on the host's request: the first tile of table A never
    publishes its run count, so the next tile's bounded wait gives up; the call
    reports FIGARO_ERR_DEVICE_TIMEOUT and the next normal call is correct."""
    A, B = make_pair(10000, 4, 3000, 4, 50, np.float32, "normal", seed=91)
    with pytest.raises(fg.FigaroError) as e:
        fg.join_qr_svd(dev(torch, A), dev(torch, B), flags=fg.FLAG_TEST_WITHHOLD, spin_limit=2000)
    assert e.value.status == 6
    check_against_oracle(fg, torch, A, B, paths=("mixed",))


def test_narrow_graded_columns(fg, torch):
    """B's columns scaled by 10^(-6 j / 15) (condition number ~1e6): the
    column-scaled error of R and the relative error of every singular value
    stay at the working precision, as the one-sided Jacobi on a graded R allows."""
    A, B = make_pair(20000, 16, 15000, 16, 200, np.float64, "normal", seed=95)
    d = 10.0 ** (-6.0 * np.arange(16) / 15.0)
    B = Table(np.ascontiguousarray(B.x * d), B.key)
    dd = np.concatenate([np.ones(16), d])
    # per-sigma bars: the FP64 path reaches ~1e-14, the mixed path ~6e-7 here
    for path, tol, tol_sv in (("fp64", 1e-10, 1e-9), ("mixed", 1e-6, 5e-6)):
        Rref, sref = oracle_ref(A, B, path)
        R, s = gpu_r_sigma(fg, torch, A, B, path)
        assert rel(R, Rref) <= tol and rel(s, sref) <= tol
        assert rel(R / dd, Rref / dd) <= 100 * tol
        assert np.max(np.abs(s - sref) / sref) <= tol_sv, np.max(np.abs(s - sref) / sref)


@pytest.mark.parametrize("n1,n2", [(15, 16), (16, 16), (17, 16)], ids=["31", "32", "33"])
def test_widths_around_the_register_kernels(fg, torch, n1, n2):
    """n = 31 and 32 take the register-resident factorisations and Jacobi
    (one column per lane), n = 33 the shared-memory forms: both against the
    oracle, including an odd n (a zero column pads the Jacobi pairing)."""
    A, B = make_pair(6000, n1, 5000, n2, 60, np.float32, "normal", seed=500 + n1)
    check_against_oracle(fg, torch, A, B)


@pytest.mark.parametrize("n1,n2,dup", [(16, 16, (3, 11)), (12, 11, (20, 14)), (4, 3, (1, 0))],
                         ids=["32", "23-odd", "7"])
def test_narrow_rank_deficient(fg, torch, n1, n2, dup):
    """A column that repeats another (in A, or in B across the tables' block
    boundary): the semi-definite factorisations mark it dependent, its row of
    R is zero, R^T R matches the oracle's J^T J, sigma matches the oracle's and
    the smallest singular value is at rounding level."""
    A, B = make_pair(4000, n1, 3500, n2, 40, np.float64, "normal", seed=510 + n1 + n2)
    xa, xb = A.x.copy(), B.x.copy()
    i, j = dup  # column i of J repeats column j (indices in J = [A | B])
    src = xa[:, j] if j < n1 else None
    if i < n1:
        xa[:, i] = src
    else:
        assert j >= n1
        xb[:, i - n1] = xb[:, j - n1]
    A, B = Table(xa, A.key), Table(xb, B.key)
    for path, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        Ar, Br = (A, B) if path == "fp64" else (as_f32(A), as_f32(B))
        G = oracle.join_gram(Ar.x, Ar.key, Br.x, Br.key)
        _, sref = oracle.join_r_sigma(Ar.x, Ar.key, Br.x, Br.key, route="reduced")
        R, s = gpu_r_sigma(fg, torch, A, B, path, flags=fg.FLAG_ALLOW_RANK_DEFICIENT)
        assert np.all(R[max(i, j)] == 0), path
        assert s[-1] <= 10 * tol * s[0], (path, s[-1] / s[0])
        assert rel(s, sref) <= tol, (path, rel(s, sref))
        assert rel(R.T @ R, G) <= tol, (path, rel(R.T @ R, G))


def test_presorted_tables_skip_the_sort(fg, torch):
    """FIGARO_FLAG_PRESORTED (Section 2's setting: inputs sorted by the join
    attribute): on tables already in key order the call skips the radix sort
    and gives bitwise the results of the sorting path (a stable sort of
    sorted keys is the identity); the grouping is the oracle's; a table that
    is not in order is reported as an invalid argument."""
    A, B = make_pair(30000, 8, 20000, 8, 700, np.float32, "normal", seed=97)
    pa, pb = np.argsort(A.key, kind="stable"), np.argsort(B.key, kind="stable")
    As, Bs = Table(np.ascontiguousarray(A.x[pa]), A.key[pa]), Table(np.ascontiguousarray(B.x[pb]), B.key[pb])
    for path in ("fp64", "mixed"):
        R0, s0 = gpu_r_sigma(fg, torch, As, Bs, path)
        R1, s1 = gpu_r_sigma(fg, torch, As, Bs, path, flags=fg.FLAG_PRESORTED)
        assert np.array_equal(R0, R1) and np.array_equal(s0, s1), path
    ga, gb, G = fg.join_group(dev(torch, As), dev(torch, Bs), flags=fg.FLAG_PRESORTED)
    oa, ob = oracle.group(As.key), oracle.group(Bs.key)
    for g, o in ((ga, oa), (gb, ob)):
        assert np.array_equal(g["perm"].cpu().numpy(), np.arange(o["perm"].size))
        assert np.array_equal(g["perm"].cpu().numpy(), o["perm"])
        assert np.array_equal(g["run_key"].cpu().numpy(), o["uniq"])
        assert np.array_equal(g["run_offset"].cpu().numpy(), o["offset"])
    assert G == oracle.match(oa, ob)["key"].size
    with pytest.raises(fg.FigaroError) as e:
        fg.join_qr_svd(dev(torch, A), dev(torch, Bs), flags=fg.FLAG_PRESORTED)
    assert e.value.status == 1
