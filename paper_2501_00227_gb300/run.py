"""Command-line contraction of one synthetic graph on the GPU.

    python -m paper_2501_00227_gb300.run --graph reg3:140:1 --semiring tropical_i32 --repeat 3

Builds the greedy order and plan on the host, contracts the network
`--repeat` times through the C ABI (the persistent executor) and prints the
result and the device time of the last contraction.  Graph specs are those of
graphgen.by_name (reg3:n:seed, ksg:L:p:seed, square:L, petersen, ...).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--graph", default="reg3:140:1")
    ap.add_argument("--semiring", default="tropical_i32", choices=["tropical_f32", "tropical_i32", "counting", "modp"])
    ap.add_argument("--primes", type=int, default=3, help="number of 31-bit primes for modp")
    ap.add_argument("--nrepeat", type=int, default=10, help="greedy order restarts")
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    import graphgen
    from paper_2501_00227_gb300 import build
    from paper_2501_00227_gb300 import tn

    build.build()
    n, e = graphgen.by_name(args.graph)
    plan = tn.Plan(n, e, nrepeat=args.nrepeat, seed=1)
    primes = tn.PRIMES31[: args.primes] if args.semiring == "modp" else None
    ws = torch.empty(plan.workspace_bytes(args.semiring, args.primes), dtype=torch.uint8, device="cuda")
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = None
    for _ in range(args.repeat):
        start.record()
        res = plan.contract(args.semiring, primes, workspace=ws)
        end.record()
    torch.cuda.synchronize()
    info = plan.info(args.semiring, args.primes)
    print(json.dumps({"graph": args.graph, "semiring": args.semiring, "result": res,
                      "log2_tc": info["log2_tc"], "log2_sc": info["log2_sc"],
                      "last_ms": start.elapsed_time(end)}))
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
