"""Autotuner for the executor's GEMM-tile launch shapes.

The host picks a tile shape and a split-K factor for every GEMM-shaped
pairwise step from a cost model (kernels_tiled.cu).  This module measures
the alternatives instead: for the step shapes (nb, nm, nn, nk) of a set of
plans it runs traced contractions (tn_contract_trace) with every candidate
(tile, split) installed for all shapes at once, reads each step's span on
the device (first task ready to last task published), keeps the fastest
candidate per shape, and installs the winners with tn_tune_set.  The table
is kept only if the plans' whole contractions get faster with it (CUDA-event
timing); otherwise the cost model stays in charge.

Everything runs through the C ABI; PyTorch only provides device buffers.
"""
from __future__ import annotations

import statistics

import numpy as np

from . import tn

TILES_BK = {0: 8, 1: 16, 2: 32, 3: 32, 4: 32, 5: 16}   # k rows per staged chunk of each tile shape
SPLITS = (1, 2, 3, 4, 6, 8, 12, 16)


def _candidates(semiring: str, nk: int):
    tropical = semiring.startswith("tropical")
    out = []
    for t, bk in TILES_BK.items():
        if t == 0 and not tropical:
            continue
        nch = max(1, (1 << nk) // bk)
        out += [(t, s) for s in SPLITS if s <= nch]
    return out


def _trace(torch, plan, semiring, primes, stream):
    k = len(primes) if primes else 1
    info = plan.info(semiring, k)
    ws = torch.empty(plan.workspace_bytes(semiring, k), dtype=torch.uint8, device="cuda")
    tr = torch.zeros(8 * info["exec_tasks"], dtype=torch.int64, device="cuda")
    tn.tn_contract_async(plan.handle, semiring, primes, ws.data_ptr(), ws.numel(), stream,
                         torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda").data_ptr())
    _, ts, _, _ = tn.tn_contract_trace(plan.handle, semiring, primes, ws.data_ptr(), ws.numel(), stream,
                                       tr.data_ptr(), info["exec_tasks"], info["nsteps"])
    T = tr.cpu().numpy().reshape(-1, 8).astype(np.int64)
    spans = {}
    for x in np.unique(ts):
        m = ts == x
        spans[int(x)] = float(T[m, 4].max() - T[m, 2].min()) * 1e-3   # us
    return spans


def _time_ms(torch, plans, semiring, primes, stream, reps: int = 5):
    k = len(primes) if primes else 1
    ws = torch.empty(max(p.workspace_bytes(semiring, k) for p in plans), dtype=torch.uint8, device="cuda")
    raw = torch.zeros(tn.TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    for p in plans:
        tn.tn_contract_async(p.handle, semiring, primes, ws.data_ptr(), ws.numel(), stream, raw.data_ptr())
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for p in plans:
            tn.tn_contract_async(p.handle, semiring, primes, ws.data_ptr(), ws.numel(), stream, raw.data_ptr())
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune(plans, semiring: str, primes=None, *, min_ops_bits: int = 18, keep=()):
    """Measure and install launch shapes for the GEMM-tile steps of `plans`
    (tn.Plan objects) in `semiring`.  `keep`: table rows of other semirings
    to install alongside.  Returns {"rows", "baseline_ms", "tuned_ms",
    "kept", "shapes", "candidates"}."""
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    k = len(primes) if primes else 1
    sr_id = tn.SEMIRINGS[semiring]
    keep = [list(r) for r in keep]
    tn.tn_tune_set(keep)
    # shapes of the steps the cost model runs as tiles, and where they are
    shapes = {}
    for i, p in enumerate(plans):
        info = tn.tn_plan_step_info(p.handle, semiring, k)
        for row in info:
            x, _, kernel, _, _, _, nb, nm, nn, nk = (int(v) for v in row)
            if kernel == 1 and nb + nm + nn + nk >= min_ops_bits:
                shapes.setdefault((nb, nm, nn, nk), []).append((i, x))
    if not shapes:
        return {"rows": keep, "baseline_ms": None, "tuned_ms": None, "kept": False, "shapes": 0, "candidates": 0}
    baseline = _time_ms(torch, plans, semiring, primes, stream)
    cand = sorted({c for (nb, nm, nn, nk) in shapes for c in _candidates(semiring, nk)})
    cost = {sh: {} for sh in shapes}
    for c in cand:
        rows = keep + [[sr_id, *sh, *c] for sh in shapes if c in _candidates(semiring, sh[3])]
        tn.tn_tune_set(rows)
        for i, p in enumerate(plans):
            spans = _trace(torch, p, semiring, primes, stream)
            for sh, where in shapes.items():
                if c in _candidates(semiring, sh[3]):
                    t = sum(spans.get(x, 0.0) for j, x in where if j == i)
                    cost[sh][c] = cost[sh].get(c, 0.0) + t
    best = [[sr_id, *sh, *min(cs, key=cs.get)] for sh, cs in cost.items() if cs]
    tn.tn_tune_set(keep + best)
    tuned = _time_ms(torch, plans, semiring, primes, stream)
    kept = tuned < baseline
    if not kept:
        tn.tn_tune_set(keep)
    return {"rows": keep + (best if kept else []), "baseline_ms": baseline, "tuned_ms": tuned, "kept": kept,
            "shapes": len(shapes), "candidates": len(cand)}
