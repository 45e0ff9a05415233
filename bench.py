#!/usr/bin/env python
"""Benchmark: semiring contraction of the independent-set tensor network.

Workload (one "step"): random 3-regular graphs n = 100 and n = 140 (seeds
1, 2, 3 each; configuration model), each contracted along its greedy order in
three element types -- tropical int32 (MIS size), counting tropical (MIS
size and count) and ordinary (+,*) modulo three 31-bit primes (the count of
all independent sets, recombined by CRT).  Orders and plans are built on the
host before timing (reported separately as plan_ms).

Metric: semiring-contraction Gop/s = sum over contractions of tc (Sec. 4.1:
2^{|LA u LB|} multiply-adds per pairwise step; once per prime for mod p)
divided by device time.  L2 is flushed (a 256 MiB write) before every timed
step, outside the timed events.

--impl reference times the CPU oracle (plain C loops, all host cores) on the
same six graphs with the same orders (one whole headline step per step), and
once on a single thread over a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402

PRIMES3 = (2147483647, 2147483629, 2147483587)
GRAPHS = [("reg3", 100, s) for s in (1, 2, 3)] + [("reg3", 140, s) for s in (1, 2, 3)]
SEMIRINGS = [("tropical_i32", None), ("counting", None), ("modp", PRIMES3)]
METRIC = "semiring-contraction Gop/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["tn", "reference"], default="tn")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the host cost model's tile choices")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the largest-contraction and tensor-core ablation sections")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# The int32 roofline of every executor instantiation: the instruction-issue
# bound of the 152-SM GB300 for int32 ALU instructions (64 per clock per SM;
# one (max,+) multiply-add is one __viaddmax_s32) at the maximum SM clock,
# or the register-only __viaddmax_s32 microbenchmark (tn_alu_peak), whichever
# is higher.  The microbenchmark spends 1 of 17 instructions on varying its
# operand and reached 17.9 Tops/s at 2.07 GHz, below the 20.1 Tops/s bound.
SMS = 152
INT32_PER_CLK_SM = 64

# DRAM bytes (read + write) per executor launch over the bench workload:
# one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum for every
# launch of the small bench command (profiles/launches_bench_reg3_n100_n140.md),
# averaged per instantiation.  Null once a kernel changes after the capture.
DRAM_BYTES_PER_LAUNCH = {
    "tropical_i32": 0.31e6, "counting": 55.84e6, "modp": 27.33e6,
    "profile": "profiles/launches_bench_reg3_n100_n140.md",
}

# Thread instructions per semiring multiply-add of each executor (warp
# instructions executed x 32 / (tc x primes)), from the ncu captures kept
# under profiles/ (one launch on random 3-regular n = 140).
INSTR_PER_OP = {
    "tropical_i32": {"value": 47.72e6 * 32 / 4.423e8, "profile": "profiles/k_exec_tropical_i32_reg3_n140.md"},
    "counting": {"value": 187.49e6 * 32 / 4.423e8, "profile": "profiles/k_exec_counting_reg3_n140_s3.md"},
    "modp": {"value": 215.00e6 * 32 / (3 * 4.423e8), "profile": "profiles/k_exec_modp_reg3_n140.md"},
}


def headline_orders():
    """The headline graphs with the contraction orders the GPU arm uses (the
    library's greedy order, nrepeat 10, seed 1; host code only, no GPU)."""
    from paper_2501_00227_gb300 import tn
    out = []
    for kind, n, seed in GRAPHS:
        nn, e = graphgen.random_regular3(n, seed)
        out.append((f"reg3:{n}:{seed}", nn, e, tn.tn_order_greedy(nn, e, 0.0, 10, 1)))
    return out


def cpu_reference(graphs, threads: int):
    """Times the CPU oracle over (name, n, edges, order) graphs in the three
    element types of the headline (tropical, counting, 3 primes): returns
    (semiring multiply-adds, seconds, threads used)."""
    import oracle
    oracle.build()
    used = oracle.set_threads(threads)
    ops, secs = 0, 0.0
    for _, nn, e, order in graphs:
        tc = oracle.complexity(nn, e, order)[0]
        t = time.perf_counter()
        oracle.mis_size(nn, e, order)
        oracle.mis_count(nn, e, order)
        oracle.count_modp(nn, e, order, PRIMES3)
        secs += time.perf_counter() - t
        ops += tc * (2 + len(PRIMES3))
    return ops, secs, used


def cpu_single_thread_sample(graphs):
    """The oracle on one thread over a bounded sample of the headline: the
    three n = 100 graphs and the n = 140 seed 1 graph (same orders)."""
    sample = [g for g in graphs if g[0].startswith("reg3:100:")] + [g for g in graphs if g[0] == "reg3:140:1"]
    ops, secs, used = cpu_reference(sample, 1)
    return {"value": ops / secs / 1e9, "unit": "Gop/s", "cores": used, "seconds": secs,
            "sample": "reg3 n=100 seeds 1-3 and n=140 seed 1, the GPU arm's orders, tropical + counting + 3 "
                      "primes"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    graphs = headline_orders()
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_reference(graphs, threads)
    ops = secs = 0.0
    used = threads
    for _ in range(args.steps):
        o, s, used = cpu_reference(graphs, threads)
        ops += o
        secs += s
    val = ops / secs / 1e9
    single = cpu_single_thread_sample(graphs)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "random 3-regular n=100 and n=140, seeds 1-3, greedy order (nrepeat 10)",
                       "semirings": ["tropical", "counting", "mod 3 primes"],
                       "order": "the GPU arm's orders (library greedy, nrepeat 10, seed 1), computed before timing"},
            "cpu_baseline": {"value": val, "unit": "Gop/s", "cores": used, "kind": "oracle",
                             "sample": "the whole headline step (six graphs x tropical + counting + 3 primes) on "
                                       "all cores, every step",
                             "single_thread": single},
            "e2e": {"value": val, "unit": "Gop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


_TUNE_ROWS = []


def _current_rows(rows=None):
    """The launch-shape rows installed so far in this process (set with rows)."""
    global _TUNE_ROWS
    if rows is not None:
        _TUNE_ROWS = list(rows)
    return list(_TUNE_ROWS)


def batching_bench(tn, torch, count: int = 4096):
    """Grouped persistent launch of `count` random 3-regular graphs with n
    uniform over the even numbers in [30, 60] (seed 0), MIS size and MIS count
    per instance, replayed from a CUDA graph; compared with one executor
    launch per instance (timed on the first 512 instances)."""
    rng = np.random.default_rng(0)
    ns = rng.integers(15, 31, size=count) * 2
    t0 = time.perf_counter()
    plans = [tn.Plan(*graphgen.random_regular3(int(n), 10000 + i), nrepeat=2, seed=1) for i, n in enumerate(ns)]
    plan_s = time.perf_counter() - t0
    out = {"workload": f"{count} random 3-regular graphs, n uniform even in [30,60], seed 0",
           "plan_s": plan_s}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    from paper_2501_00227_gb300 import tune
    sample = sorted(plans, key=lambda p: -p.info("tropical_i32", 1)["tc"])[:32]
    for sr in ("tropical_i32", "counting"):
        ops = sum(p.info(sr, 1)["tc"] for p in plans)
        # measured tile shapes for the largest instances' GEMM steps (kept
        # only if they beat the cost model on those instances)
        tr = tune.autotune(sample, sr, None, min_ops_bits=16, keep=_current_rows())
        _current_rows(tr["rows"])
        b = tn.Batch(plans, sr)
        res = b.run(graph=True)
        for _ in range(3):
            b.launch(graph=True)
        torch.cuda.synchronize()
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            b.launch(graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if b.results() != res:
            raise RuntimeError("batched results changed between launches")
        S = min(count, 512)
        ws = torch.empty(max(p.workspace_bytes(sr) for p in plans[:S]), dtype=torch.uint8, device="cuda")
        raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
        for p in plans[:16]:
            tn.tn_contract_async(p.handle, sr, None, ws.data_ptr(), ws.numel(), stream.cuda_stream, raw.data_ptr())
        torch.cuda.synchronize()
        e0.record(stream)
        for p in plans[:S]:
            tn.tn_contract_async(p.handle, sr, None, ws.data_ptr(), ws.numel(), stream.cuda_stream, raw.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        per_ms = e0.elapsed_time(e1) / S
        out[sr] = {"autotune": {k: tr[k] for k in ("baseline_ms", "tuned_ms", "kept", "shapes")},
                   "ms_per_batch": ms, "inst_per_s": count / ms * 1e3, "gops": ops / ms / 1e6,
                   "per_instance_launch_inst_per_s": 1e3 / per_ms,
                   "speedup_vs_per_instance": (count / ms) / (1.0 / per_ms), "tasks": b.info["tasks"]}
        b.close()
    for p in plans:
        p.close()
    return out


def largest_bench(tn, torch, peak_tops: float, autotune: bool = True):
    """The largest tropical contractions of the configs: King's subgraph 20 x 20
    at filling 0.8 (seeds 1-3, ~320 vertices, tc ~ 2^31), tropical int32, one
    executor launch each, L2 flushed before each launch; Tops/s and fraction of
    the int32 (max,+) issue peak."""
    out = {"workload": "King's subgraph 20x20 p=0.8 seeds 1-3, tropical int32, greedy (nrepeat 10)"}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    rows = []
    for seed in (1, 2, 3):
        p = tn.Plan(*graphgen.kings_subgraph(20, 0.8, seed), nrepeat=10, seed=1)
        tuned = None
        if autotune:  # measured tile shapes for this instance's steps, before timing
            from paper_2501_00227_gb300 import tune
            r = tune.autotune([p], "tropical_i32", None, keep=_current_rows())
            _current_rows(r["rows"])
            tuned = r["kept"]
        ws = torch.empty(p.workspace_bytes("tropical_i32"), dtype=torch.uint8, device="cuda")
        raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
        for _ in range(2):
            tn.tn_contract_async(p.handle, "tropical_i32", None, ws.data_ptr(), ws.numel(), stream.cuda_stream,
                                 raw.data_ptr())
        ms = []
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tn.tn_contract_async(p.handle, "tropical_i32", None, ws.data_ptr(), ws.numel(), stream.cuda_stream,
                                 raw.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        tc = p.info("tropical_i32")["tc"]
        tops = tc / (statistics.median(ms) * 1e-3) / 1e12
        rows.append({"seed": seed, "log2_tc": float(np.log2(tc)), "ms": statistics.median(ms), "tops": tops,
                     "frac": tops / peak_tops, "autotuned": tuned})
        p.close()
    out["instances"] = rows
    out["best_frac"] = max(r["frac"] for r in rows)
    return out


def umma_contraction_bench(tn, torch):
    """The tensor-core ablation inside a whole contraction (config 4): the
    King's subgraph 20x20 seed 1, count mod 4 primes, timed three ways on one
    plan -- the executor (CUDA cores, one launch), one launch per step on the
    CUDA cores (TN_EXEC=0), and one launch per step with every GEMM-shaped
    step (M % 128, N % 64, K % 64 == 0) on the tcgen05 limb GEMM (TN_UMMA=1:
    gather to row-major operands, tn_modp_gemm_umma, scatter of the result)."""
    import graphgen
    primes = tuple(tn.PRIMES31[:4])
    n, e = graphgen.by_name("ksg:20:0.8:1")
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    si = tn.tn_plan_step_info(p.handle, "modp", 4)
    ops = 2.0 ** (si[:, 6] + si[:, 7] + si[:, 8] + si[:, 9])
    fit = (si[:, 7] >= 7) & (si[:, 8] >= 6) & (si[:, 9] >= 6)
    ws = torch.empty(p.workspace_bytes("modp", 4), dtype=torch.uint8, device="cuda")
    raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    total_ops = float(ops.sum()) * 4
    out = {"workload": "King's subgraph 20x20 p=0.8 seed 1, count mod 4 primes, greedy (nrepeat 10)",
           "log2_tc": float(np.log2(ops.sum())), "tensor_core_steps": int(fit.sum()),
           "tensor_core_share_of_tc": float(ops[fit].sum() / ops.sum())}
    saved = {k: os.environ.get(k) for k in ("TN_EXEC", "TN_UMMA")}
    try:
        for name, env in (("executor_cuda_cores", {}), ("per_step_cuda_cores", {"TN_EXEC": "0"}),
                          ("per_step_tcgen05", {"TN_EXEC": "0", "TN_UMMA": "1"})):
            for k in ("TN_EXEC", "TN_UMMA"):
                os.environ.pop(k, None)
            os.environ.update(env)
            res = p.contract("modp", primes, workspace=ws)["residues"]
            times = []
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                tn.tn_contract_async(p.handle, "modp", primes, ws.data_ptr(), ws.numel(), st, raw.data_ptr())
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            out[name] = {"ms": ms, "tops": total_ops / (ms * 1e-3) / 1e12, "residues": res}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        p.close()
    out["equal"] = (out["executor_cuda_cores"]["residues"] == out["per_step_cuda_cores"]["residues"]
                    == out["per_step_tcgen05"]["residues"])
    return out


def limb_ablation_bench(tn, torch):
    """Tensor-core ablation of the mod-p GEMM (config 4): the largest King's
    subgraph 20x20 step shape, (batch, M, N, K) = (2, 1024, 512, 1024), 4
    primes, on 8-bit limbs with integer MMAs vs the CUDA-core tile path
    (tn_contract_pair) on the same buffers."""
    primes = tuple(tn.PRIMES31[:4])
    batch, m, n, k = 2, 1024, 512, 1024
    g = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randint(0, 2 ** 31 - 1, (4 * batch * m * k,), dtype=torch.int64, device="cuda", generator=g)
    b = torch.randint(0, 2 ** 31 - 1, (4 * batch * n * k,), dtype=torch.int64, device="cuda", generator=g)
    pr = torch.tensor(primes, dtype=torch.int64, device="cuda")
    a = (a.view(4, -1) % pr[:, None]).to(torch.int32).reshape(-1)
    b = (b.view(4, -1) % pr[:, None]).to(torch.int32).reshape(-1)
    c1 = torch.zeros(4 * batch * m * n, dtype=torch.int32, device="cuda")
    c2 = torch.zeros_like(c1)
    st = torch.cuda.current_stream().cuda_stream
    lk, lm, ln, lb = list(range(0, 10)), list(range(20, 30)), list(range(40, 49)), [60]

    c3 = torch.zeros_like(c1)

    def limb():
        tn.tn_modp_gemm_limb(primes, a.data_ptr(), b.data_ptr(), c1.data_ptr(), batch, m, n, k, st)

    def umma():
        tn.tn_modp_gemm_umma(primes, a.data_ptr(), b.data_ptr(), c3.data_ptr(), batch, m, n, k, st)

    def core():
        tn.tn_contract_pair("modp", primes, a.data_ptr(), lk + lm + lb, b.data_ptr(), lk + ln + lb, ln + lm + lb,
                            c2.data_ptr(), st)

    out = {"shape": {"batch": batch, "M": m, "N": n, "K": k, "primes": 4}}
    ops = 4.0 * batch * m * n * k
    for name, fn in (("tcgen05_bf16_limbs", umma), ("mma_sync_u8_limbs", limb), ("cuda_core_tile", core)):
        for _ in range(2):
            fn()
        times = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        out[name] = {"ms": ms, "tops": ops / (ms * 1e-3) / 1e12}
    out["equal"] = bool(torch.equal(c1, c2)) and bool(torch.equal(c3, c2))
    # tensor work of the tcgen05 path: 16 limb products, 2 flops per multiply-add
    out["tcgen05_bf16_tflops"] = 16 * 2 * ops / (out["tcgen05_bf16_limbs"]["ms"] * 1e-3) / 1e12
    out["note"] = ("tcgen05.mma kind::i8 is rejected by ptxas for sm_103a: the tcgen05 path uses kind::f16 on "
                   "bf16 limbs (exact integers) with fp32 accumulators; mma.sync u8 is the integer tensor path")
    return out


def polynomial_bench(tn, torch, plans, cpu: bool = True):
    """Independence polynomial (Eq. 13, finite-field method) of the headline
    graphs: degree = alpha from a tropical contraction, the fewest 31-bit
    primes whose product exceeds 2^n, (alpha + 1) x nprimes weighted mod-p
    evaluations in launches of 16 slots, Newton interpolation and CRT on the
    host.  Timed end to end (the call is synchronous).  The oracle computes
    the same polynomial of the first n=100 graph beside it."""
    out = {"workload": "random 3-regular n=100 and n=140 seeds 1-3 (the headline plans), degree alpha, "
                       "x = 1..alpha+1 per prime", "instances": []}
    st = torch.cuda.current_stream()
    for (kind, n, seed), p in zip(GRAPHS, plans):
        alpha = p.contract("tropical_i32")["max"]
        k, prod = 0, 1
        while prod <= (1 << n):
            k += 1
            prod *= tn.primes31(k)[-1]
        primes = tn.primes31(k)
        slots = (alpha + 1) * k
        ws = torch.empty(p.workspace_bytes("modp", min(tn.TN_MAX_PRIMES, slots)), dtype=torch.uint8, device="cuda")
        tn.tn_independence_polynomial(p.handle, primes, alpha, ws.data_ptr(), ws.numel(), st.cuda_stream)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            coeffs, _ = tn.tn_independence_polynomial(p.handle, primes, alpha, ws.data_ptr(), ws.numel(),
                                                      st.cuda_stream)
            times.append(time.perf_counter() - t)
        sec = statistics.median(times)
        tc = p.info("modp", 1)["tc"]
        out["instances"].append({"n": n, "seed": seed, "alpha": alpha, "primes": k, "evaluations": slots,
                                 "launches": -(-slots // tn.TN_MAX_PRIMES), "ms": sec * 1e3,
                                 "evals_per_s": slots / sec, "gops": tc * slots / sec / 1e9,
                                 "coeff_sum_bits": int(sum(coeffs)).bit_length()})
        del ws
    if cpu:
        import oracle
        oracle.build()
        cores = oracle.set_threads(os.cpu_count() or 1)
        kind, n, seed = GRAPHS[0]
        nn, e = graphgen.random_regular3(n, seed)
        first = out["instances"][0]
        t = time.perf_counter()
        oracle.independence_polynomial(nn, e, plans[0].order, tn.primes31(first["primes"]), degree=first["alpha"])
        sec = time.perf_counter() - t
        out["cpu_baseline"] = {"value": sec * 1e3, "unit": "ms per polynomial", "cores": cores, "kind": "oracle",
                               "sample": f"the n={n} seed {seed} polynomial, same order, primes and degree"}
    return out


def kbest_bench(tn, torch, plans, poly=None):
    """SizeMax(k) and CountingMax(k) (Sec. 5.3, Table 1) of the headline graphs
    in one contraction with the k-best element types (tn_contract_kbest,
    synchronous, timed end to end), next to the polynomial route (the same
    numbers read off the exact independence polynomial, from
    independence_polynomial)."""
    st = torch.cuda.current_stream().cuda_stream
    out = {"workload": "random 3-regular n=100 and n=140 seeds 1-3 (the headline plans), unit weights",
           "instances": []}
    poly_ms = {(r["n"], r["seed"]): r["ms"] for r in (poly or {}).get("instances", [])}
    for (kind, n, seed), p in zip(GRAPHS, plans):
        row = {"n": n, "seed": seed}
        for name in ("size_max", "counting_max"):
            for k in (2, 4):
                ws = torch.empty(tn.tn_kbest_workspace_bytes(p.handle, name, k), dtype=torch.uint8, device="cuda")
                f = lambda: tn.tn_contract_kbest(p.handle, name, k, ws.data_ptr(), ws.numel(), st)
                r = f()
                ts = []
                for _ in range(5):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    f()
                    ts.append(time.perf_counter() - t)
                row[f"{name}_{k}_ms"] = statistics.median(ts) * 1e3
                row[f"{name}_{k}"] = r.get("values") or [r["max"], r["counts"]]
                del ws
        if (n, seed) in poly_ms:
            row["polynomial_route_ms"] = poly_ms[(n, seed)]
        out["instances"].append(row)
    return out


def weighted_bench(tn, torch, plans, cpu: bool = True):
    """Weighted networks on the headline plans: the spin glass of Eq. 1 with
    seeded +-1 couplings (tropical and counting, stored leaves generated on
    the GPU), next to the unit-weight IS contraction of the same plans; and
    the Buckyball's exact energy histogram (ln Z at any temperature), with the
    oracle computing the same histogram beside it."""
    from paper_2501_00227_gb300 import properties as props

    def med_ms(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t)
        return statistics.median(ts) * 1e3

    out = {"workload": "random 3-regular n=100 and n=140 seeds 1-3 (the headline plans), spin glass with "
                       "couplings J uniform in {-1, +1} (seed = graph seed), h = 0; Buckyball C60, J = 1",
           "spin_glass": []}
    for (kind, n, seed), p in zip(GRAPHS, plans):
        J = graphgen.random_weights(len(p.edges), seed)
        row = {"n": n, "seed": seed}
        for sr in ("tropical_i32", "counting"):
            need = tn.tn_weighted_workspace_bytes(p.handle, sr, 1)
            ws = torch.empty(max(need, p.workspace_bytes(sr)), dtype=torch.uint8, device="cuda")
            st = torch.cuda.current_stream().cuda_stream
            row[sr + "_ms"] = med_ms(lambda: tn.tn_contract_weighted(p.handle, sr, "spin", J, None, None, None,
                                                                     ws.data_ptr(), ws.numel(), st))
            row[sr + "_unit_is_ms"] = med_ms(lambda: tn.tn_contract(p.handle, sr, None, ws.data_ptr(), ws.numel(),
                                                                    st))
            del ws
        r = p.contract_weighted("counting", "spin", J)
        row["ground_energy"], row["degeneracy"] = -r["max"], r["count"]
        out["spin_glass"].append(row)
    n, e = graphgen.fullerene()
    pb = tn.Plan(n, e, nrepeat=10, seed=1)
    hist = props.energy_histogram(pb)
    t_hist = med_ms(lambda: props.energy_histogram(pb), reps=3)
    out["buckyball"] = {"histogram_ms": t_hist, "evaluations": 2 * (2 * hist[0] + 1), "primes": 2,
                        "ground_state": props.spin_glass_ground_state(pb),
                        "log_z_per_site_beta1": props.log_partition_function(pb, 1.0, histogram=hist) / n}
    if cpu:
        import oracle
        oracle.build()
        cores = oracle.set_threads(os.cpu_count() or 1)
        t = time.perf_counter()
        oracle.weighted_polynomial("spin", n, e, pb.order, tn.primes31(2), 2 * hist[0])
        out["buckyball"]["cpu_baseline"] = {"value": (time.perf_counter() - t) * 1e3, "unit": "ms per histogram",
                                            "cores": cores, "kind": "oracle",
                                            "sample": "the Buckyball energy histogram, same order and primes"}
    pb.close()
    return out


def single_config_bench(tn, torch, plans):
    """SingleConfigMax on the headline plans: the (max,+) contraction with
    every intermediate kept plus the GPU backward pass, timed end to end
    (synchronous call), next to the plain tropical contraction; the returned
    configuration is checked for independence and size."""
    out = {"workload": "random 3-regular n=100 and n=140 seeds 1-3 (the headline plans), unit weights",
           "instances": []}
    st = torch.cuda.current_stream().cuda_stream
    for (kind, n, seed), p in zip(GRAPHS, plans):
        ws = torch.empty(tn.tn_single_config_workspace_bytes(p.handle), dtype=torch.uint8, device="cuda")

        def run():
            return tn.tn_single_config_max(p.handle, "is", None, None, p.n, ws.data_ptr(), ws.numel(), st)

        def plain():
            return tn.tn_contract(p.handle, "tropical_i32", None, ws.data_ptr(), ws.numel(), st)

        res = {}
        for name, fn in (("single_config", run), ("tropical", plain)):
            fn()
            ts = []
            for _ in range(5):
                torch.cuda.synchronize()
                t = time.perf_counter()
                r = fn()
                ts.append(time.perf_counter() - t)
            res[name] = (statistics.median(ts) * 1e3, r)
        val, cfg = res["single_config"][1]
        e = p.edges
        valid = not bool(np.any(cfg[e[:, 0]].astype(bool) & cfg[e[:, 1]].astype(bool))) and int(cfg.sum()) == val
        out["instances"].append({"n": n, "seed": seed, "mis": val, "valid": valid,
                                 "single_config_ms": res["single_config"][0], "tropical_ms": res["tropical"][0],
                                 "keep_workspace_mb": ws.numel() / 2 ** 20})
        del ws
    return out


def treesa_bench(tn, torch):
    """Contraction order quality (Sec. 4.2): the headline 3-regular graphs and
    the 20x20 King's subgraphs with the greedy order (nrepeat 10) and with a
    TreeSA order (8 trials, the default schedule), each contracted in the
    three element types on the GPU (device time, CUDA events)."""
    st = torch.cuda.current_stream()
    raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")

    def dev_ms(p, sr, primes):
        k = len(primes) if primes else 1
        ws = torch.empty(p.workspace_bytes(sr, k), dtype=torch.uint8, device="cuda")
        f = lambda: tn.tn_contract_async(p.handle, sr, primes, ws.data_ptr(), ws.numel(), st.cuda_stream,
                                         raw.data_ptr())
        f()
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            f()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"workload": "random 3-regular n=100, 140 seeds 1-3 and King's subgraphs 20x20 p=0.8 seeds 1-3; "
                       "tropical_i32 + counting + modp x3 per graph", "graphs": []}
    specs = [(f"reg3:{n}:{s}", graphgen.random_regular3(n, s)) for _, n, s in GRAPHS]
    specs += [(f"ksg:20:0.8:{s}", graphgen.kings_subgraph(20, 0.8, s)) for s in (1, 2, 3)]
    for name, (n, e) in specs:
        row = {"graph": name}
        for opt in ("greedy", "treesa"):
            t = time.perf_counter()
            p = tn.Plan(n, e, nrepeat=10, seed=1, optimizer=opt, treesa={"ntrials": 8})
            opt_s = time.perf_counter() - t
            info = p.info("tropical_i32")
            ms = sum(dev_ms(p, sr, pr) for sr, pr in SEMIRINGS)
            row[opt] = {"log2_tc": info["log2_tc"], "log2_sc": info["log2_sc"], "optimize_s": opt_s,
                        "gpu_ms_3_semirings": ms}
            p.close()
        row["speedup"] = row["greedy"]["gpu_ms_3_semirings"] / row["treesa"]["gpu_ms_3_semirings"]
        out["graphs"].append(row)
    return out


def slicing_bench(tn, torch):
    """Slicing (Sec. 4.2.2) on the 20x20 King's subgraph (seed 1, greedy
    order): s labels picked by tn_slice_labels, all 2^s slices contracted
    (counting element type, stored leaves written per slice) and added, one
    slice per launch and all slices in one merged launch; workspace and time
    against s."""
    n, e = graphgen.kings_subgraph(20, 0.8, 1)
    order = tn.tn_order_greedy(n, e, 0.0, 10, 1)
    out = {"workload": "King's subgraph 20x20 p=0.8 seed 1, greedy order (nrepeat 10), counting", "rows": []}
    ref = None
    st = torch.cuda.current_stream().cuda_stream
    for s in (0, 2, 4, 6):
        p = tn.Plan(n, e, order, sliced=s)
        info = p.info("counting")
        row = {"slices": 1 << s, "log2_sc_per_slice": info["log2_sc"], "log2_tc_all_slices": info["log2_tc"] + s}
        for name, batch in (("one_per_launch", 1), ("batched", 1 << s)):
            need = tn.tn_sliced_workspace_bytes(p.handle, "counting", 1, batch)
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            run = lambda: tn.tn_contract_sliced(p.handle, "counting", "is", None, None, None, None, 0, 1 << s,
                                                ws.data_ptr(), ws.numel(), st)
            r = run()
            ref = ref or r
            ts = []
            for _ in range(3):
                torch.cuda.synchronize()
                t = time.perf_counter()
                run()
                ts.append(time.perf_counter() - t)
            row[name] = {"workspace_mb": need / 2 ** 20, "ms": statistics.median(ts) * 1e3, "same_result": r == ref}
            del ws
        out["rows"].append(row)
        p.close()
    return out


def serving_bench(tn, torch, nreq: int = 600, budget_gb: int = 120, optimizer: str = "greedy",
                  sweep_rates: bool = True):
    """Poisson request stream mixing random 3-regular graphs (n even in
    [40,160]) and King's subgraphs (L in [8,16], filling 0.8), each asking the
    MIS size, the MIS count or the count of all independent sets mod 4 primes,
    served with continuous batching under a 120 GB budget.  Plain baseline:
    the same requests one at a time (synchronous tn_contract).  optimizer:
    the contraction orders of the pool ("greedy": the paper's default,
    Sec. 4.2.1; "treesa": a light TreeSA run, Sec. 4.2.2), the same for both
    arms."""
    rng = np.random.default_rng(5)
    pool = []
    t_opt = time.perf_counter()
    for i in range(96):
        if i % 2 == 0:
            n, e = graphgen.random_regular3(int(rng.integers(20, 81)) * 2, 20000 + i)
        else:
            n, e = graphgen.kings_subgraph(int(rng.integers(8, 17)), 0.8, 30000 + i)
        pool.append(tn.Plan(n, e, nrepeat=10, seed=1, optimizer=optimizer,
                            treesa={"ntrials": 2, "niters": 10}))
    t_opt = time.perf_counter() - t_opt
    kinds = [("tropical_i32", None), ("counting", None), ("modp", tuple(tn.PRIMES31[:4]))]
    reqs = [(pool[int(rng.integers(0, len(pool)))], *kinds[int(rng.integers(0, 3))]) for _ in range(nreq)]
    need = max(p.workspace_bytes(sr, len(pr) if pr else 1) for p, sr, pr in reqs)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # plain: one request at a time
    for p, sr, pr in reqs[:20]:
        tn.tn_contract(p.handle, sr, pr, ws.data_ptr(), need, st)
    lat = []
    t0 = time.perf_counter()
    ref = []
    for p, sr, pr in reqs:
        t = time.perf_counter()
        ref.append(tn.tn_contract(p.handle, sr, pr, ws.data_ptr(), need, st))
        lat.append(time.perf_counter() - t)
    plain_s = time.perf_counter() - t0
    plain = {"inst_per_s": nreq / plain_s, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
             "p99_ms": 1e3 * float(np.percentile(lat, 99))}
    # device time of every request alone (CUDA events around its launch, run
    # back to back): what the GPU must spend on the stream if requests do not
    # overlap, and its five largest requests' share
    raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in reqs]
    torch.cuda.synchronize()
    for (p, sr, pr), (e0, e1) in zip(reqs, evs):
        e0.record()
        tn.tn_contract_async(p.handle, sr, pr, ws.data_ptr(), need, st, raw.data_ptr())
        e1.record()
    torch.cuda.synchronize()
    dev_ms = sorted((e0.elapsed_time(e1) for e0, e1 in evs), reverse=True)
    device = {"sum_ms": float(sum(dev_ms)), "largest5_ms": float(sum(dev_ms[:5])),
              "plain_s_over_device_sum": plain_s / (sum(dev_ms) * 1e-3)}

    def serve(rate):
        server = tn.tn_server_create(budget_gb << 30, 4)
        try:
            arrive = np.cumsum(rng.exponential(1.0 / rate, size=nreq)) if rate else np.zeros(nreq)
            tickets, done, meta = [], {}, {}
            t_start = time.perf_counter()
            i = 0
            while len(done) < nreq:
                now = time.perf_counter() - t_start
                while i < nreq and arrive[i] <= now:
                    p, sr, pr = reqs[i]
                    tk = (tn.tn_submit(server, p.handle, sr, pr), sr, arrive[i])
                    tickets.append(tk)
                    meta[tk[0]] = (sr, arrive[i])
                    i += 1
                fin = tn.tn_server_completed(server)
                if fin:
                    now = time.perf_counter() - t_start
                    for t in fin:
                        sr, a = meta[t]
                        done[t] = (tn.tn_poll(server, t, sr), now - a)
            total = time.perf_counter() - t_start
        finally:
            tn.tn_server_destroy(server)
        res = [done[t][0] for t, _, _ in tickets]
        if res != ref:
            raise RuntimeError("served results differ from the same requests run alone")
        lats = [done[t][1] for t, _, _ in tickets]
        return {"offered_per_s": rate or None, "inst_per_s": nreq / total,
                "p50_ms": 1e3 * float(np.percentile(lats, 50)), "p99_ms": 1e3 * float(np.percentile(lats, 99))}

    sat = serve(0)  # every request offered at once
    # Poisson rates from a quarter to four times the plain path's capacity
    sweep = [dict(serve(f * plain["inst_per_s"]), of_plain_capacity=f) for f in (0.25, 0.5, 1.0, 2.0, 4.0)] \
        if sweep_rates else None
    pool_tc = sum(2.0 ** p.info("tropical_i32")["log2_tc"] for p in pool)
    for p in pool:
        p.close()
    return {"workload": f"{nreq} requests, Poisson arrivals (seed 5), 50/50 3-regular n in [40,160] / "
                        "King's subgraph L in [8,16] p=0.8, MIS size | MIS count | count mod 4 primes, "
                        f"{budget_gb} GB budget, 4 launch slots",
            "orders": optimizer, "order_s": t_opt, "log2_pool_tc": float(np.log2(pool_tc)),
            "plain_one_at_a_time": plain, "served_saturated": sat, "served_rate_sweep": sweep,
            "device_time_alone": device,
            "served_s_over_device_sum": (nreq / sat["inst_per_s"]) / (device["sum_ms"] * 1e-3),
            "speedup_inst_per_s": sat["inst_per_s"] / plain["inst_per_s"]}


def run_tn(args):
    import torch
    import torch.distributed as dist

    from paper_2501_00227_gb300 import build as B
    from paper_2501_00227_gb300 import shard
    from paper_2501_00227_gb300 import tn

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()

    # ---- plans (host; not timed in the metric)
    t0 = time.perf_counter()
    plans = []
    for kind, n, seed in GRAPHS:
        nn, e = graphgen.random_regular3(n, seed)
        plans.append(tn.Plan(nn, e, nrepeat=10, seed=1))
    plan_ms = 1e3 * (time.perf_counter() - t0)
    jobs = []          # (plan, semiring, primes, ops)
    for p in plans:
        info = p.info(tn.TN_COUNT_MODP, len(PRIMES3))
        for sr, pr in SEMIRINGS:
            jobs.append((p, sr, pr, info["tc"] * (len(pr) if pr else 1), info["nsteps"]))
    ops_per_step = sum(j[3] for j in jobs)
    # measured tile / split-K shapes for the GEMM steps of these plans (before
    # timing, like the plans themselves)
    tune_report = {}
    if not args.no_autotune:
        from paper_2501_00227_gb300 import tune
        t0 = time.perf_counter()
        rows = []
        for sr, pr in SEMIRINGS:
            r = tune.autotune(plans, sr, pr, keep=rows)
            rows = r["rows"]
            tune_report[sr] = {k: r[k] for k in ("baseline_ms", "tuned_ms", "kept", "shapes", "candidates")}
        tune_report["tune_s"] = time.perf_counter() - t0
        tune_report["table_rows"] = len(rows)
        _current_rows(rows)
    # register-only rates of the kernels' inner steps (the ALU roofline
    # denominators), measured on this GPU before the timed region
    alu = {"maxplus": tn.tn_alu_peak("maxplus"), "maxplus16x2": tn.tn_alu_peak("maxplus16x2"),
           "modp": tn.tn_alu_peak("modp")}
    ws_bytes = max(p.workspace_bytes(sr, len(pr) if pr else 1) for p, sr, pr, _, _ in jobs)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    raw = torch.zeros(len(jobs) * tn.TN_RAW_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    def one_step():
        for i, (p, sr, pr, _, _) in enumerate(jobs):
            tn.tn_contract_async(p.handle, sr, pr, ws.data_ptr(), ws_bytes, sptr,
                                 raw.data_ptr() + i * tn.TN_RAW_BYTES)

    def check(raw_host, ref=None):
        out = []
        for i, (p, sr, pr, _, _) in enumerate(jobs):
            r = tn.tn_result_decode(sr, pr, bytes(raw_host[i * tn.TN_RAW_BYTES:(i + 1) * tn.TN_RAW_BYTES]))
            out.append(json.dumps(r, sort_keys=True))
        if ref is not None and out != ref:
            raise RuntimeError("results changed between steps")
        return out

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize()
    ref = check(raw.cpu().numpy())

    # ---- timed region: K steps; device time between events, L2 flushed before each
    #      (events also bracket every contraction: its executor launch is the kernel timed)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    jev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in jobs]
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            for i, (p, sr, pr, _, _) in enumerate(jobs):
                jev[k][i][0].record(stream)
                tn.tn_contract_async(p.handle, sr, pr, ws.data_ptr(), ws_bytes, sptr,
                                     raw.data_ptr() + i * tn.TN_RAW_BYTES)
                jev[k][i][1].record(stream)
            ends[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    check(raw.cpu().numpy(), ref)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # every rank contracts the same per-GPU workload (independent networks, no
    # data-path collective); the job's time is the slowest rank's
    total_ms = shard.max_over_ranks(sum(step_ms), dist if world > 1 else None, dev)
    value = world * ops_per_step * args.steps / (total_ms * 1e-3) / 1e9

    # ---- per-kernel attribution: one executor launch per contraction
    per = {}
    for k in range(args.steps):
        for i, (p, sr, pr, ops, _) in enumerate(jobs):
            a = per.setdefault(sr, [0.0, 0, 0])
            a[0] += jev[k][i][0].elapsed_time(jev[k][i][1])
            a[1] += ops
            a[2] += 1
    dom_sr, (dom_ms, dom_ops, dom_n) = max(per.items(), key=lambda kv: kv[1][0])

    # ---- end to end through the public API: for every graph, build the plan
    # from the host edge list + order, contract it in the three element types
    # (each contraction uploads its step / task tables on first use and reads
    # its result back to the host), destroy the plan
    e2e_steps = max(1, min(args.steps, 3))
    # bytes each contraction uploads (its tables), from the same plans,
    # counted before the timed region
    table_bytes = {(id(p), sr): p.info(sr, len(pr) if pr else 1)["exec_table_bytes"] for p, sr, pr, _, _ in jobs}
    torch.cuda.synchronize()
    h2d = 0
    t = time.perf_counter()
    for _ in range(e2e_steps):
        for p in plans:
            h = tn.tn_plan(p.n, p.edges, p.order)
            for sr, pr in SEMIRINGS:
                tn.tn_contract(h, sr, pr, ws.data_ptr(), ws_bytes, sptr)
                h2d += table_bytes[(id(p), sr)]
            tn.tn_plan_destroy(h)
    e2e_s = time.perf_counter() - t
    e2e_val = ops_per_step * e2e_steps / e2e_s / 1e9

    csum = clk.summary()
    clock_mhz = csum["sm_max_mhz"] or 2070.0
    issue_peak = SMS * INT32_PER_CLK_SM * clock_mhz * 1e6 / 1e12   # Tops/s, int32 issue bound
    peak = max(issue_peak, alu["maxplus"])
    achieved = dom_ops / (dom_ms * 1e-3) / 1e12
    per_tops = {k: v[1] / (v[0] * 1e-3) / 1e12 for k, v in per.items()}
    # algorithmic bytes of one launch of the dominant kernel: every operand and
    # output entry of every step once (rwc entries, Sec. 4.1) x entry bytes,
    # averaged over its launches
    ebytes = {"tropical_i32": 4, "counting": 12, "modp": 4 * len(PRIMES3)}[dom_sr]
    alg_bytes = statistics.mean(p.info(sr, len(pr) if pr else 1)["rwc"] * ebytes
                                for p, sr, pr, _, _ in jobs if sr == dom_sr)
    roofline = {"bound": "alu", "kernel": f"k_exec<{dom_sr}>", "achieved": achieved, "peak": peak,
                "unit": "Tops/s", "frac": achieved / peak, "traffic": DRAM_BYTES_PER_LAUNCH[dom_sr],
                "traffic_basis": "DRAM bytes read + written per launch of this kernel, mean over the bench "
                                 "workload's launches, one ncu capture (" + DRAM_BYTES_PER_LAUNCH["profile"] + ")",
                "algorithmic_bytes_per_launch": alg_bytes,
                "peak_basis": f"int32 issue bound: {SMS} SMs x {INT32_PER_CLK_SM} int32 instr/clk/SM x "
                              f"{clock_mhz:.0f} MHz (max SM clock) = {issue_peak:.2f} Tops/s, or the "
                              f"register-only __viaddmax_s32 rate {alu['maxplus']:.2f} Tops/s measured in this "
                              "run, whichever is higher; one semiring multiply-add per op (tc)",
                "time_share": dom_ms / sum(v[0] for v in per.values()), "launches": dom_n,
                "per_semiring_tops": per_tops,
                "per_semiring_frac": {k: per_tops[k] / peak for k in per_tops},
                "instr_per_op": INSTR_PER_OP,
                "inner_step_rates": {"unit": "Tops/s", "maxplus": alu["maxplus"],
                                     "maxplus16x2": alu["maxplus16x2"], "modp_fold4": alu["modp"],
                                     "note": "register-only rates of each kernel's inner step (tn_alu_peak): "
                                             "int32 add-max, the packed tile's two int16 add-maxes per "
                                             "instruction, and the mod-p 64-bit multiply-add folded every "
                                             "fourth term; context, not the denominator"}}

    line = {"metric": METRIC, "value": value, "unit": "Gop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32/uint64", "data": "synthetic",
            "config": {"workload": "random 3-regular n=100 and n=140, seeds 1-3, greedy order (nrepeat 10)",
                       "semirings": ["tropical_i32", "counting(int32,uint64)", "modp x3 (31-bit) + CRT"],
                       "ops_per_step": ops_per_step, "contractions_per_step": len(jobs),
                       "l2": "flushed (256 MiB write) before each timed step", "plan_ms": plan_ms,
                       "autotune": tune_report or "off"},
            "e2e": {"value": e2e_val, "unit": "Gop/s", "h2d_bytes_per_step": h2d // e2e_steps,
                    "d2h_bytes_per_step": tn.TN_RAW_BYTES * len(jobs)},
            "gpu_launches": None, "roofline": roofline, "clocks": csum}
    # one executor launch per contraction
    line["gpu_launches"] = args.steps * len(jobs)
    if rank == 0 and not args.no_extras:
        line["largest_tropical"] = largest_bench(tn, torch, peak, autotune=not args.no_autotune)
        line["modp_tensor_core_ablation"] = limb_ablation_bench(tn, torch)
        line["modp_tensor_core_contraction"] = umma_contraction_bench(tn, torch)
        line["independence_polynomial"] = polynomial_bench(tn, torch, plans, cpu=not args.no_cpu_baseline)
        line["kbest"] = kbest_bench(tn, torch, plans, line["independence_polynomial"])
        line["weighted"] = weighted_bench(tn, torch, plans, cpu=not args.no_cpu_baseline)
        line["single_config"] = single_config_bench(tn, torch, plans)
        line["treesa"] = treesa_bench(tn, torch)
        line["slicing"] = slicing_bench(tn, torch)
    if rank == 0 and not args.no_batching:
        line["batching"] = batching_bench(tn, torch)
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(tn, torch)
        line["serving_treesa_orders"] = serving_bench(tn, torch, optimizer="treesa")
    if rank == 0 and not args.no_cpu_baseline:
        graphs = [(f"reg3:{n}:{seed}", p.n, p.edges, p.order) for (kind, n, seed), p in zip(GRAPHS, plans)]
        ops, secs, used = cpu_reference(graphs, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": ops / secs / 1e9, "unit": "Gop/s", "cores": used, "kind": "oracle",
                                "sample": "the whole headline step on all cores: the six graphs with the GPU "
                                          f"arm's orders, tropical + counting + 3 primes each, {secs:.1f} s",
                                "single_thread": cpu_single_thread_sample(graphs)}
    if rank == 0:
        print(json.dumps(line))
    for p in plans:
        p.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_tn(args)


if __name__ == "__main__":
    sys.exit(main())
