"""Throughput benchmark: input rows/s to R + sigma of a two-table natural join.

Default workload (N=1): 1,000,000 + 1,000,000 rows, 16 + 16 FP32 features
N(0,1), int32 keys uniform over 10,000 ids (join of about 1e8 rows x 32
columns), mixed-precision path.  One step = the whole hot path on one
instance: key grouping, head/tail of both tables, CholeskyQR2 (two Gram
passes, two FP64 Cholesky), one-sided Jacobi.  Inputs are resident in HBM
before the timed region; a 256 MB buffer is rewritten between steps (outside
the timed events) so that no step starts with a warm L2.

Multi-GPU (torchrun): every rank runs its own independently seeded instance
(the instances share nothing, so there is no data-path collective); value =
all ranks' input rows / max-over-ranks time (weak scaling).

--impl reference: the FP64 CPU oracle (materialised join, Householder QR,
one-sided Jacobi) on bounded samples of the same workload, on host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input rows/s to R+σ on 1 GB300, mixed vs plain FP64 at rel err ≤1e-6; % roofline"
WORKLOADS = {
    "c1": "1e6+1e6 rows x 16+16 FP32 N(0,1), int32 keys uniform over 1e4 ids (join ~1e8 x 32)",
    "c2": "4e6+2e6 rows x 32+32 FP32 U[-1,1], Zipf(1.2) keys over 1e5 ids",
    "c0": "1000+1000 rows x 4+4 FP64 U[-1,1], 100 keys",
    "c4": "2e5+2e5 rows x 256+256 FP32, B column-scaled to condition 1e8, int32 keys uniform over 100 ids "
          "(join ~4e8 x 512)",
    "c3": "512 independent instances, m1, m2 log-uniform in [1e3, 1e5], n1, n2 from {8, 16, 32, 64}, FP32 N(0,1), "
          "int32 keys uniform over max(1, min(m1, m2) / 10) ids; one batched call replayed as a CUDA graph",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c1", choices=sorted(WORKLOADS))
    ap.add_argument("--path", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--gram-engine", default="auto", choices=["auto", "simt", "tcgen05"])
    ap.add_argument("--task", default="qr_svd", choices=["qr_svd", "lstsq"],
                    help="lstsq: least squares over the join with B's last column as the label")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-materialized", action="store_true")
    ap.add_argument("--sigma", default="jacobi", choices=["jacobi", "dqds"],
                    help="singular values of R by one-sided Jacobi or by bidiagonalisation and dqds (n <= 128)")
    ap.add_argument("--cpu-sample-keys", type=int, default=0)
    return ap.parse_args()


# FP64 FMA issue on this GPU, measured by a clock64 microbenchmark on one SM
# (1.9 FMA per SM per clock): 152 SMs x 1.9 x 2 flops x 2,070 MHz
FP64_PEAK_TFLOPS = 152 * 1.9 * 2 * 2070e6 / 1e12


def host_cpu():
    """Host cores and CPU model (for the oracle's timing rows)."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    model = line.split(":", 1)[1].strip()
                    if low.startswith("model name"):
                        break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def gram_pass_flops(A, B, heads, pass2):
    """Algorithmic flops (2 per FMA) of one CholeskyQR Gram pass over the
    reduced matrix: the symmetric Gram (k (k + 1) / 2 FMA per row of a block of
    width k) and, in pass 2, the formation Q = X W (k x kout FMA per row)."""
    n = A.n + B.n
    blocks = [(heads, n, n), (A.m, A.n, n), (B.m, B.n, B.n)]
    f = 0.0
    for rows, k, kout in blocks:
        w = kout if pass2 else k
        f += rows * (w * (w + 1) / 2 + (k * kout if pass2 else 0))
    return 2.0 * f


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def tf32_peak():
    """Dense TF32 tensor rate for a kernel timed inside a long step: the measured
    sustained BF16 GEMM rate times the nominal TF32 / BF16 ratio (1.1 / 2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]) * 1.1 / 2.25, "measured bf16 sustained x 1.1 / 2.25"
    except Exception:
        return 1700.0 * 1.1 / 2.25, "fallback bf16 sustained x 1.1 / 2.25"


def max_over_ranks(total_ms, world, device):
    """The slowest rank's time (every rank runs its own instance; the job
    ends when the slowest one does)."""
    if world <= 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(rows_per_rank, world, ms_per_step):
    """Input rows of all ranks per second (weak scaling: each rank has its own rows)."""
    return world * rows_per_rank / (ms_per_step / 1e3)


def measured_traffic(kernel, cfg):
    """DRAM bytes (read + write) per launch from the committed ncu capture, or
    None when the capture is for another workload or the kernel's source has
    changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[kernel]
        src = os.path.join(ROOT, "paper_2503_23385_gb300", "csrc", rec.get("source", "headtail.cu"))
        with open(src, "rb") as f:
            same = hashlib.sha256(f.read()).hexdigest() == rec["source_sha256"]
        return float(rec["traffic_bytes"]) if same and rec["workload"] == cfg else None
    except Exception:
        return None


# ------------------------------------------------------------ clocks ------

class NvmlClocks:
    """The SM clock and the clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise OSError("nvmlDeviceGetHandleByIndex")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        if self.reasons_fn is None:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None

    def sample(self):
        clk, rs = self.ct.c_uint(0), self.ct.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(clk)) != 0:
            return None
        names = []
        if self.reasons_fn(self.h, self.ct.byref(rs)) == 0:
            names = [n for bit, n in self.REASONS.items() if rs.value & bit]
        return float(clk.value), names


class ClockSampler:
    """SM clocks and throttle reasons during the timed region: NVML read about
    every millisecond on a thread, or nvidia-smi every 10 ms where NVML cannot
    be loaded."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.nvml = None
        self.thread = None
        self.samples = []

    def _loop(self):
        while not self.stop.is_set():
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)
            time.sleep(0.001)

    def __enter__(self):
        import threading
        try:
            self.nvml = NvmlClocks(self.dev)
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if self.nvml is not None and self.samples:
            sm = [c for c, _ in self.samples]
            reasons = sorted({n for _, ns in self.samples for n in ns})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.nvml.max_mhz or max(sm), "reasons": reasons,
                    "samples": len(sm), "source": "nvml"}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


# -------------------------------------------------------------- oracle ----

def key_sample(A, B, num_keys):
    """The rows of both tables whose key is among the first num_keys ids."""
    keys = np.unique(np.concatenate([A.key, B.key]))[:num_keys]
    ma, mb = np.isin(A.key, keys), np.isin(B.key, keys)
    return (A.x[ma], A.key[ma]), (B.x[mb], B.key[mb])


def oracle_rows_per_s(A, B, sample_keys):
    import oracle
    (ax, ak), (bx, bk) = key_sample(A, B, sample_keys)
    t0 = time.perf_counter()
    R = oracle.join_r_materialized(ax, ak, bx, bk)
    oracle.jacobi_sigma(R)
    dt = time.perf_counter() - t0
    rows = ax.shape[0] + bx.shape[0]
    return rows / dt, dt, rows, oracle.join_rows(ak, bk)


def oracle_batch_rows_per_s(instances, budget_s):
    """The oracle (O1) on whole instances of a batch, in order, until about
    budget_s seconds have passed."""
    import oracle
    t0 = time.perf_counter()
    rows, used, jrows = 0, 0, 0
    for A, B in instances:
        R = oracle.join_r_materialized(A.x, A.key, B.x, B.key)
        oracle.jacobi_sigma(R)
        rows += A.m + B.m
        jrows += oracle.join_rows(A.key, B.key)
        used += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return rows / dt, dt, rows, used, jrows


def default_sample_keys(cfg, reference_arm=False):
    """Key ids in the oracle's sample: about 15 s of single-core work for the
    cpu_baseline leg, about 4 s per step for the reference arm."""
    if reference_arm:
        return {"c0": 100, "c1": 500, "c2": 40}.get(cfg, 100)
    return {"c0": 100, "c1": 2000, "c2": 150}.get(cfg, 100)


def run_reference(args, rank, world):
    """The oracle timed on host cores (rank 0 only)."""
    if rank != 0:
        return
    from workloads import config
    # each step is a bounded sample, sized so that the whole run stays near a minute
    per_step_s = 60.0 / max(1, args.steps + args.warmup)
    if args.config == "c3":
        inst = config("c3")
        for _ in range(args.warmup):
            oracle_batch_rows_per_s(inst[:1], 0.0)
        times, rows, used = [], 0, 0
        for _ in range(args.steps):
            rps, dt, rows, used, jrows = oracle_batch_rows_per_s(inst, min(4.0, per_step_s))
            times.append(dt)
        ms = 1e3 * sum(times) / len(times)
        value = rows / (ms / 1e3)
        sample = f"the first {used} of the 512 instances ({rows} input rows, {jrows} join rows) per step"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config], "path": "oracle O1 per instance"},
                "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle", "sample": sample,
                                 **host_cpu()},
                "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    A, B = config(args.config)
    # the default sample takes about 3 s per step on one core; the oracle's time grows with the sampled keys
    keys = args.cpu_sample_keys or max(5, int(default_sample_keys(args.config, reference_arm=True) *
                                              min(1.0, per_step_s / 3.2)))
    for _ in range(args.warmup):
        oracle_rows_per_s(A, B, max(1, keys // 10))
    times, rows = [], 0
    for _ in range(args.steps):
        rps, dt, rows, jrows = oracle_rows_per_s(A, B, keys)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = rows / (ms / 1e3)
    sample = f"rows with one of the first {keys} key ids ({rows} input rows, {jrows} join rows) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "path": "oracle O1 (materialised join, Householder QR, "
                       "one-sided Jacobi)"},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle", "sample": sample,
                                 **host_cpu()},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- GPU arm ------

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_2503_23385_gb300 as fg
    from workloads import config

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.config == "c3":
        run_batch(args, rank, world, torch, dist, fg, dev, local)
        if world > 1:
            dist.destroy_process_group()
        return

    A, B = config(args.config, rank=rank)
    rows = A.m + B.m
    tA = (torch.from_numpy(A.x).to(dev), torch.from_numpy(A.key).to(dev))
    tB = (torch.from_numpy(B.x).to(dev), torch.from_numpy(B.key).to(dev))
    n = A.n + B.n

    evs = [torch.cuda.Event(enable_timing=True) for _ in range(fg.NUM_PHASE_EVENTS)]
    ev_arr = fg.event_array(evs)
    engine = {"auto": fg.GRAM_AUTO, "simt": fg.GRAM_SIMT, "tcgen05": fg.GRAM_TCGEN05}[args.gram_engine]
    solver_cls = fg.LsqSolver if args.task == "lstsq" else fg.Solver
    sig_flags = fg.FLAG_SIGMA_DQDS if (args.sigma == "dqds" and args.task == "qr_svd") else 0
    solver = solver_cls(tA, tB, path=args.path, phase_events=ev_arr, gram_engine=engine, flags=sig_flags)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            solver(tA, tB, stream=stream)
        stream.synchronize()
    status = solver.status(stream)
    if status != 0:
        raise fg.FigaroError(status, "warm-up")

    # The timed graph holds the call without phase events (an event between two
    # kernels would stop the next one from starting early); a second graph with
    # the events gives the per-phase breakdown from separate replays.
    graph = graph_ph = None
    launches_before = fg.kernel_launches()
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
            solver(tA, tB, stream=stream, record_phases=False)
        launches_per_step = fg.kernel_launches() - launches_before
        graph_ph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_ph, stream=stream, capture_error_mode="relaxed"):
            solver(tA, tB, stream=stream)
        for _ in range(2):
            graph.replay()
            graph_ph.replay()
        torch.cuda.synchronize()
    else:
        solver(tA, tB, stream=stream)
        stream.synchronize()
        launches_per_step = fg.kernel_launches() - launches_before

    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, phase_ms = [], [[] for _ in range(fg.NUM_PHASE_EVENTS - 1)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.fill_(1)
                s0.record(stream)
                if graph is not None:
                    graph.replay()
                else:
                    solver(tA, tB, stream=stream)
                s1.record(stream)
                s1.synchronize()
                step_ms.append(s0.elapsed_time(s1))
                if graph is None:
                    for i in range(fg.NUM_PHASE_EVENTS - 1):
                        phase_ms[i].append(evs[i].elapsed_time(evs[i + 1]))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    if graph_ph is not None:  # the phase breakdown, outside the timed region
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.fill_(1)
                graph_ph.replay()
                evs[-1].synchronize()
                for i in range(fg.NUM_PHASE_EVENTS - 1):
                    phase_ms[i].append(evs[i].elapsed_time(evs[i + 1]))
        torch.cuda.synchronize()
    info = solver.info(stream)
    status = solver.status(stream)
    if status != 0:
        raise fg.FigaroError(status, "timed steps")

    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(rows, world, ms_per_step)
    phases = {name: statistics.mean(v) for name, v in zip(fg.PHASES, phase_ms)}

    # ---- roofline of the dominant kernel: the Gram passes ----------------
    # (the tensor-core Gram of the reduced matrix, HBM-bound at these widths:
    # a tail row of n_t FP32 values is read once per CholeskyQR pass, a head
    # row of n values likewise; per pass: three Gram launches and a reduce)
    hbm, peak_kind = measured_peaks()
    s = 4 if args.path == "mixed" else 8
    ein = A.x.itemsize
    heads = info.get("num_runs_a", 0) if isinstance(info, dict) else 0
    gram_bytes = sum(T.m * T.n * s for T in (A, B)) + heads * n * s
    # mixed path, FP32 tables of 8 or 16 columns, automatic engine: the head/tail stream also
    # accumulates the pass-1 Gram of that table's tails (no extra HBM bytes)
    fused = [args.path == "mixed" and ein == 4 and args.gram_engine == "auto" and T.n in (8, 16) for T in (A, B)]
    roofline_avg = None
    roofline_avg_key = "roofline_gram_avg"
    if n <= 128:
        # the dominant launch group is the second pass (formation Q = X W and the Gram of Q); the
        # average of the two passes is reported beside it
        g2 = gram_bytes / (phases["gram2"] / 1e3) / 1e9
        roofline = {"kernel": "gram_pack_kernel: CholeskyQR pass 2 (head rows with the A tails in one launch, B tails, reduce)",
                    "bound": "hbm", "achieved": g2, "peak": hbm, "unit": "GB/s", "frac": g2 / hbm,
                    "traffic": measured_traffic("gram_pass", args.config), "bytes_per_launch": gram_bytes,
                    "peak_source": peak_kind}
        if any(fused):
            # pass 1 then reads only the head rows (and the tails of a table the stream does not cover)
            g1_bytes = heads * n * s + sum(T.m * T.n * s for T, f in zip((A, B), fused) if not f)
            g1 = g1_bytes / (phases["gram1"] / 1e3) / 1e9
            roofline_avg_key = "roofline_gram_pass1"
            roofline_avg = {"kernel": "CholeskyQR pass 1 outside the head/tail stream (head-row launch + reduce)",
                            "bound": "hbm", "achieved": g1, "peak": hbm, "unit": "GB/s", "frac": g1 / hbm,
                            "bytes_per_launch": g1_bytes, "peak_source": peak_kind,
                            "note": "the pass-1 Gram of the 8- and 16-column FP32 tails runs inside ht_stream_kernel"}
        else:
            gram_ms = (phases["gram1"] + phases["gram2"]) / 2
            g_avg = gram_bytes / (gram_ms / 1e3) / 1e9
            roofline_avg = {"kernel": "gram_pack_kernel: one CholeskyQR Gram pass, average of the two passes",
                            "bound": "hbm", "achieved": g_avg, "peak": hbm, "unit": "GB/s", "frac": g_avg / hbm,
                            "bytes_per_launch": gram_bytes, "peak_source": peak_kind}
    elif args.path == "mixed":
        # wide joins, mixed path: pass 1's tail blocks run the tensor-core tile Gram (128 x 128 upper
        # tiles, 3 x TF32: three tensor products per FP32 product); tensor flops of the tiles it computes
        # over the pass's time (the head block's CUDA-core tiles and the reduce included)
        tiles = lambda k: ((k + 127) // 128) * ((k + 127) // 128 + 1) // 2
        flops = 3 * 2.0 * 128 * 128 * (A.m * tiles(A.n) + B.m * tiles(B.n))
        tpeak, tsrc = tf32_peak()
        achieved_tf = flops / (phases["gram1"] / 1e3) / 1e12
        roofline = {"kernel": "wide_gram_tc_kernel, Gram pass 1 (tcgen05 kind::tf32, 3 x TF32)", "bound": "tensor",
                    "achieved": achieved_tf, "peak": tpeak, "unit": "TFLOP/s", "frac": achieved_tf / tpeak,
                    "traffic": None, "flops_per_launch": flops, "peak_source": tsrc}
    else:
        # wide joins, FP64 path: pass 1 of the CUDA-core tile Gram (64 x 64 upper tiles), bound by FP64 FMA
        # issue is reported in fp64_path; here the FP32-ALU form of the same line
        tiles = lambda k: ((k + 63) // 64) * ((k + 63) // 64 + 1) // 2
        flops = 2.0 * 64 * 64 * (A.m * tiles(A.n) + B.m * tiles(B.n) + heads * tiles(n))
        alu_peak = 152 * 128 * 2 * 2070e6 / 1e12
        achieved_tf = flops / (phases["gram1"] / 1e3) / 1e12
        roofline = {"kernel": "wide_gram_kernel, Gram pass 1 (CUDA cores, FP32 products)", "bound": "alu",
                    "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tf / alu_peak,
                    "traffic": None, "flops_per_launch": flops,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"}
    # the head/tail kernel (one launch covers both tables)
    # per input row: perm + run index (4 + 4 B), the gathered features, the tail row written
    ht_bytes = sum(T.m * (4 + 4 + T.n * ein + T.n * s) for T in (A, B))
    ht_ms = phases["head_tail"]
    achieved = ht_bytes / (ht_ms / 1e3) / 1e9
    ht_name = "ht_stream_kernel (both tables" + ("; pass-1 Gram of the tails inside)" if any(fused) else ")")
    roofline_ht = {"kernel": ht_name, "bound": "hbm", "achieved": achieved, "peak": hbm,
                   "unit": "GB/s", "frac": achieved / hbm, "traffic": measured_traffic("ht_stream_kernel", args.config),
                   "bytes_per_launch": ht_bytes, "peak_source": peak_kind}

    # ---- end to end through the C ABI with host buffers -----------------
    e2e = None
    try:
        if args.task != "qr_svd":
            raise RuntimeError("the end-to-end leg times the qr_svd task")
        hA = (torch.from_numpy(A.x).pin_memory(), torch.from_numpy(A.key).pin_memory())
        hB = (torch.from_numpy(B.x).pin_memory(), torch.from_numpy(B.key).pin_memory())
        Rh = torch.zeros((n, n), dtype=torch.float64).pin_memory()
        sh = torch.zeros(n, dtype=torch.float64).pin_memory()
        wsh = torch.empty(fg.host_workspace_size(hA, hB, path=args.path), dtype=torch.uint8, device=dev)
        for _ in range(2):
            fg.join_qr_svd_host(hA, hB, Rh, sh, wsh, stream=stream, path=args.path, flags=sig_flags)
        stream.synchronize()
        e_ms = []
        for _ in range(max(3, min(args.steps, 10))):
            s0.record(stream)
            fg.join_qr_svd_host(hA, hB, Rh, sh, wsh, stream=stream, path=args.path, flags=sig_flags)
            s1.record(stream)
            s1.synchronize()
            e_ms.append(s0.elapsed_time(s1))
        st = fg.get_status(wsh, stream)
        if st != 0:
            raise fg.FigaroError(st, "e2e")
        em = statistics.mean(e_ms)
        h2d = A.x.nbytes + A.key.nbytes + B.x.nbytes + B.key.nbytes
        e2e = {"value": world * rows / (em / 1e3), "unit": "rows/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": n * n * 8 + n * 8, "ms_per_step": em}
        del wsh
    except Exception as exc:  # reported, not hidden
        e2e = {"error": repr(exc)}

    # ---- the plain FP64 path on the same instance ------------------------
    fp64 = None
    if args.path == "mixed" and args.fp64_steps > 0 and args.task == "qr_svd":
        try:
            s64 = fg.Solver(tA, tB, path="fp64")
            s64(tA, tB, stream=stream)
            stream.synchronize()
            f_ms = []
            for _ in range(args.fp64_steps):
                flush.fill_(1)
                s0.record(stream)
                s64(tA, tB, stream=stream)
                s1.record(stream)
                s1.synchronize()
                f_ms.append(s0.elapsed_time(s1))
            fm = statistics.mean(f_ms)
            d = np.linalg.norm((solver.R - s64.R).cpu().numpy()) / np.linalg.norm(s64.R.cpu().numpy())
            ds = np.linalg.norm((solver.sigma - s64.sigma).cpu().numpy()) / np.linalg.norm(s64.sigma.cpu().numpy())
            # phase times of the FP64 path (one call with the phase events)
            s64p = fg.Solver(tA, tB, path="fp64", phase_events=ev_arr)
            flush.fill_(1)
            s64p(tA, tB, stream=stream)
            evs[-1].synchronize()
            ph64 = {name: evs[i].elapsed_time(evs[i + 1]) for i, name in enumerate(fg.PHASES)}
            # its dominant kernel: the second Gram pass on CUDA cores, bound by FP64 FMA issue
            f2 = gram_pass_flops(A, B, heads, True)
            tf = f2 / (ph64["gram2"] / 1e3) / 1e12
            fp64 = {"value": world * rows / (fm / 1e3), "unit": "rows/s", "ms_per_step": fm,
                    "mixed_vs_fp64_rel_err_R": float(d), "mixed_vs_fp64_rel_err_sigma": float(ds),
                    "phases_ms": ph64,
                    "roofline": {"kernel": "gram_kernel<double>: CholeskyQR pass 2 (CUDA cores, FP64)", "bound": "alu",
                                 "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": tf / FP64_PEAK_TFLOPS, "flops_per_launch": f2,
                                 "peak_source": "measured FP64 FMA issue: 1.9 per SM per clock x 152 SMs x 2 x "
                                                "2070 MHz"}}
            del s64p
            del s64
        except Exception as exc:
            fp64 = {"error": repr(exc)}

    # ---- pre-sorted tables (G13: the paper times inputs already in key order) --
    presorted = None
    if args.task == "qr_svd" and args.config in ("c1", "c2", "c0"):
        try:
            pa, pb = np.argsort(A.key, kind="stable"), np.argsort(B.key, kind="stable")
            sA = (torch.from_numpy(np.ascontiguousarray(A.x[pa])).to(dev), torch.from_numpy(A.key[pa]).to(dev))
            sB = (torch.from_numpy(np.ascontiguousarray(B.x[pb])).to(dev), torch.from_numpy(B.key[pb]).to(dev))
            sp = fg.Solver(sA, sB, path=args.path, flags=fg.FLAG_PRESORTED | sig_flags)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    sp(sA, sB, stream=stream)
            stream.synchronize()
            gp = None
            if graph is not None:
                gp = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gp, stream=stream, capture_error_mode="relaxed"):
                    sp(sA, sB, stream=stream)
            p_ms = []
            with torch.cuda.stream(stream):
                for _ in range(max(3, min(args.steps, 50))):
                    flush.fill_(1)
                    s0.record(stream)
                    if gp is not None:
                        gp.replay()
                    else:
                        sp(sA, sB, stream=stream)
                    s1.record(stream)
                    s1.synchronize()
                    p_ms.append(s0.elapsed_time(s1))
            st = sp.status(stream)
            if st != 0:
                raise fg.FigaroError(st, "presorted")
            pm = statistics.mean(p_ms)
            presorted = {"value": world * rows / (pm / 1e3), "unit": "rows/s", "ms_per_step": pm,
                         "what": "tables in key order (host-sorted once, outside the timing), FIGARO_FLAG_PRESORTED: "
                                 "the grouping without the radix sort"}
            del sp, gp, sA, sB
        except Exception as exc:
            presorted = {"error": repr(exc)}

    # ---- the other singular-value method on the same resident inputs ---------
    sigma_alt = None
    if args.task == "qr_svd" and args.config in ("c1", "c2", "c0"):
        alt = "dqds" if args.sigma == "jacobi" else "jacobi"
        try:
            sa = fg.Solver(tA, tB, path=args.path, flags=fg.FLAG_SIGMA_DQDS if alt == "dqds" else 0)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    sa(tA, tB, stream=stream)
            stream.synchronize()
            ga = None
            if graph is not None:
                ga = torch.cuda.CUDAGraph()
                with torch.cuda.graph(ga, stream=stream, capture_error_mode="relaxed"):
                    sa(tA, tB, stream=stream)
            a_ms = []
            with torch.cuda.stream(stream):
                for _ in range(max(3, min(args.steps, 50))):
                    flush.fill_(1)
                    s0.record(stream)
                    if ga is not None:
                        ga.replay()
                    else:
                        sa(tA, tB, stream=stream)
                    s1.record(stream)
                    s1.synchronize()
                    a_ms.append(s0.elapsed_time(s1))
            st = sa.status(stream)
            if st != 0:
                raise fg.FigaroError(st, "sigma_alt")
            am = statistics.mean(a_ms)
            sigma_alt = {"sigma": alt, "value": world * rows / (am / 1e3), "unit": "rows/s", "ms_per_step": am,
                         "transforms_or_sweeps": sa.info(stream)["jacobi_sweeps"],
                         "what": "the whole step with sigma by " + ("bidiagonalisation and dqds (FIGARO_FLAG_SIGMA_DQDS)"
                                                                   if alt == "dqds" else "one-sided Jacobi")}
            del sa, ga
        except Exception as exc:
            sigma_alt = {"error": repr(exc)}

    # ---- materialised-join QR baseline (torch / cuSOLVER on J) ----------
    mat = None
    if not args.no_materialized and rank == 0:
        mat = materialized_baseline(torch, A, B, dev, stream)

    # ---- oracle on host cores ------------------------------------------
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        keys = args.cpu_sample_keys or default_sample_keys(args.config)
        rps, dt, srows, jrows = oracle_rows_per_s(A, B, keys)
        cpu = {"value": rps, "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": f"rows with one of the first {keys} key ids: {srows} input rows, {jrows} join rows, "
                         f"{dt:.1f} s (O1: materialised join, Householder QR, one-sided Jacobi)", **host_cpu()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.path == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config], "path": args.path, "rows_per_gpu": rows,
                           "graph": graph is not None, "gram_engine": args.gram_engine, "task": args.task,
                           "sigma": args.sigma,
                           "l2": "inputs 136 MB + ~300 MB workspace exceed L2; 256 MB flush between steps"},
                "roofline": roofline, roofline_avg_key: roofline_avg, "roofline_head_tail": roofline_ht,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "phases_ms": phases, "instance": info,
                "fp64_path": fp64, "presorted": presorted, "sigma_alt": sigma_alt,
                "materialized_baseline": mat}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args, rank, world, torch, dist, fg, dev, local):
    """The batching workload: 512 independent instances in one
    figaro_batch_join call (one launch per phase for all of them), captured
    once in a CUDA graph and replayed every step.  The instances' tables are
    views of two flat device buffers, so that the end-to-end leg moves them
    with one host-to-device copy each and reads all outputs back with one
    device-to-host copy."""
    from workloads import config
    inst = config("c3", rank=rank)
    rows = sum(A.m + B.m for A, B in inst)
    xs = np.concatenate([T.x.reshape(-1) for AB in inst for T in AB])
    ks = np.concatenate([T.key for AB in inst for T in AB])
    x_dev = torch.from_numpy(xs).to(dev)
    k_dev = torch.from_numpy(ks).to(dev)
    pairs, xo, ko = [], 0, 0
    for A, B in inst:
        pr = []
        for T in (A, B):
            pr.append((x_dev[xo:xo + T.m * T.n].view(T.m, T.n), k_dev[ko:ko + T.m]))
            xo += T.m * T.n
            ko += T.m
        pairs.append(tuple(pr))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(fg.NUM_PHASE_EVENTS)]
    ev_arr = fg.event_array(evs)
    # the first call tunes the schedule on this batch (outside the capture)
    sig_flags = fg.FLAG_SIGMA_DQDS if args.sigma == "dqds" else 0
    solver = fg.BatchSolver(pairs, path=args.path, flags=fg.FLAG_AUTOTUNE | sig_flags)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            solver(stream=stream, phase_events=ev_arr)
    st = solver.status(stream)
    if st != 0:
        raise fg.FigaroError(st, "warm-up")
    launches_before = fg.kernel_launches()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        solver(stream=stream)
    launches_per_step = fg.kernel_launches() - launches_before
    graph_ph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_ph, stream=stream, capture_error_mode="relaxed"):
        solver(stream=stream, phase_events=ev_arr)
    for _ in range(2):
        graph.replay()
        graph_ph.replay()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, phase_ms = [], [[] for _ in range(fg.NUM_PHASE_EVENTS - 1)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.fill_(1)
                s0.record(stream)
                graph.replay()
                s1.record(stream)
                s1.synchronize()
                step_ms.append(s0.elapsed_time(s1))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    with torch.cuda.stream(stream):  # the phase breakdown, outside the timed region
        for _ in range(args.steps):
            flush.fill_(1)
            graph_ph.replay()
            evs[-1].synchronize()
            for i in range(fg.NUM_PHASE_EVENTS - 1):
                phase_ms[i].append(evs[i].elapsed_time(evs[i + 1]))
    torch.cuda.synchronize()
    st = solver.status(stream)
    if st != 0:
        raise fg.FigaroError(st, "timed steps")
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(rows, world, ms_per_step)
    phases = {name: statistics.mean(v) for name, v in zip(fg.PHASES, phase_ms)}
    hbm, peak_kind = measured_peaks()
    s_c = 4 if args.path == "mixed" else 8
    # head/tail (both tables of every instance, carry pre-pass included)
    ht_bytes = sum(T.m * (4 + 4 + T.n * T.x.itemsize + T.n * s_c) for AB in inst for T in AB)
    ht_ms = phases["head_tail"]
    achieved = ht_bytes / (ht_ms / 1e3) / 1e9
    roofline = {"kernel": "ht_plan/ht_scan/ht_stream_batched (all instances)", "bound": "hbm", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None, "bytes_per_launch": ht_bytes,
                "peak_source": peak_kind}
    # ---- end to end: inputs from pinned host memory, every R and sigma back
    e2e = None
    try:
        hx = torch.from_numpy(xs).pin_memory()
        hk = torch.from_numpy(ks).pin_memory()
        out_elems = sum(R.numel() + sg.numel() for R, sg in solver.outs)
        hout = torch.empty(out_elems, dtype=torch.float64).pin_memory()
        e_ms = []
        with torch.cuda.stream(stream):
            for it in range(max(3, min(args.steps, 10)) + 1):
                s0.record(stream)
                x_dev.copy_(hx, non_blocking=True)
                k_dev.copy_(hk, non_blocking=True)
                graph.replay()
                flat = torch.cat([t.reshape(-1) for R, sg in solver.outs for t in (R, sg)])
                hout.copy_(flat, non_blocking=True)
                s1.record(stream)
                s1.synchronize()
                if it > 0:
                    e_ms.append(s0.elapsed_time(s1))
        em = statistics.mean(e_ms)
        e2e = {"value": world * rows / (em / 1e3), "unit": "rows/s", "h2d_bytes_per_step": xs.nbytes + ks.nbytes,
               "d2h_bytes_per_step": out_elems * 8, "ms_per_step": em}
    except Exception as exc:
        e2e = {"error": repr(exc)}
    # ---- the plain FP64 path, mixed-vs-FP64 error over all instances
    fp64 = None
    if args.path == "mixed" and args.fp64_steps > 0:
        try:
            s64 = fg.BatchSolver(pairs, path="fp64")
            with torch.cuda.stream(stream):
                s64(stream=stream)
                stream.synchronize()
                f_ms = []
                for _ in range(args.fp64_steps):
                    flush.fill_(1)
                    s0.record(stream)
                    s64(stream=stream)
                    s1.record(stream)
                    s1.synchronize()
                    f_ms.append(s0.elapsed_time(s1))
            fm = statistics.mean(f_ms)
            eR = max(float(torch.linalg.norm(R - R64) / torch.linalg.norm(R64))
                     for (R, _), (R64, _) in zip(solver.outs, s64.outs))
            es = max(float(torch.linalg.norm(sg - s6) / torch.linalg.norm(s6))
                     for (_, sg), (_, s6) in zip(solver.outs, s64.outs))
            fp64 = {"value": world * rows / (fm / 1e3), "unit": "rows/s", "ms_per_step": fm,
                    "mixed_vs_fp64_max_rel_err_R": eR, "mixed_vs_fp64_max_rel_err_sigma": es,
                    "timing": "direct call (host plan building included), not a graph replay"}
            del s64
        except Exception as exc:
            fp64 = {"error": repr(exc)}
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        rps, dt, srows, used, jrows = oracle_batch_rows_per_s(inst, 12.0)
        cpu = {"value": rps, "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {used} of the 512 instances: {srows} input rows, {jrows} join rows, {dt:.1f} s "
                         f"(O1: materialised join, Householder QR, one-sided Jacobi, per instance)", **host_cpu()}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.path == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS["c3"], "path": args.path, "rows_per_gpu": rows, "graph": True,
                           "sigma": args.sigma,
                           "instances": len(inst), "schedule (autotuned)": solver.schedule(),
                           "l2": f"inputs {(xs.nbytes + ks.nbytes) / 1e9:.1f} GB exceed L2; 256 MB flush between steps"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks, "phases_ms": phases, "fp64_path": fp64}
        print(json.dumps(line), flush=True)


def materialized_baseline(torch, A, B, dev, stream):
    """Builds J on the device with torch ops and times torch.linalg.qr (R only)
    on it: the paper's comparison (Householder QR of the materialised join).
    Not the product path; reported where J fits in memory."""
    try:
        ka, kb = torch.from_numpy(A.key).to(dev).long(), torch.from_numpy(B.key).to(dev).long()
        pa, pb = torch.argsort(ka, stable=True), torch.argsort(kb, stable=True)
        ua, ca = torch.unique_consecutive(ka[pa], return_counts=True)
        ub, cb = torch.unique_consecutive(kb[pb], return_counts=True)
        common, ia, ib = np.intersect1d(ua.cpu().numpy(), ub.cpu().numpy(), return_indices=True)
        ca, cb = ca.cpu().numpy()[ia], cb.cpu().numpy()[ib]
        join_rows = int(np.sum(ca.astype(np.int64) * cb))
        n = A.n + B.n
        bytes_needed = join_rows * n * 4
        free, _ = torch.cuda.mem_get_info(dev)
        if bytes_needed * 2.5 > free:
            return {"skipped": f"J needs {bytes_needed / 1e9:.1f} GB (FP32); {free / 1e9:.1f} GB free"}
        xa, xb = torch.from_numpy(A.x).to(dev).float()[pa], torch.from_numpy(B.x).to(dev).float()[pb]
        offa = np.concatenate([[0], np.cumsum(ca)])
        offb = np.concatenate([[0], np.cumsum(cb)])
        J = torch.empty((join_rows, n), dtype=torch.float32, device=dev)
        r = 0
        for g in range(len(common)):
            a = xa[offa[g]:offa[g + 1]]
            b = xb[offb[g]:offb[g + 1]]
            k = a.shape[0] * b.shape[0]
            J[r:r + k, :A.n] = a.repeat_interleave(b.shape[0], dim=0)
            J[r:r + k, A.n:] = b.repeat(a.shape[0], 1)
            r += k
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)

        def timed(Jm):
            torch.linalg.qr(Jm[:4096], mode="r")
            t0.record()
            R = torch.linalg.qr(Jm, mode="r")[1]
            torch.linalg.svdvals(R)
            t1.record()
            t1.synchronize()
            return t0.elapsed_time(t1)

        ms = timed(J)
        out = {"value": (A.m + B.m) / (ms / 1e3), "unit": "rows/s", "ms": ms, "join_rows": join_rows,
               "dtype": "f32", "what": "torch.linalg.qr(J, mode='r') + svdvals(R) on the materialised join"}
        free, _ = torch.cuda.mem_get_info(dev)
        if 2 * bytes_needed * 2.5 < free:  # J in FP64 beside J in FP32, and the QR's work space
            J64 = J.double()
            del J
            ms64 = timed(J64)
            del J64
            out["fp64"] = {"value": (A.m + B.m) / (ms64 / 1e3), "unit": "rows/s", "ms": ms64, "dtype": "f64"}
        else:
            del J
            out["fp64"] = {"skipped": f"J in FP64 needs {2 * bytes_needed / 1e9:.1f} GB"}
        return out
    except Exception as exc:
        return {"error": repr(exc)}


if __name__ == "__main__":
    main()
