"""Command-line contraction of one synthetic graph on the GPU, or one
standalone mod-p step GEMM (the tensor-core ablations).

    python -m paper_2501_00227_gb300.run --graph reg3:140:1 --semiring tropical_i32 --repeat 3
    python -m paper_2501_00227_gb300.run --gemm umma --shape 2,1024,512,1024 --primes 4

Builds the order (greedy, or TreeSA with --order treesa) and plan on the host, contracts the network
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
    ap.add_argument("--order", default="greedy", choices=["greedy", "treesa"],
                    help="contraction order: greedy (Sec. 4.2.1) or TreeSA (Sec. 4.2.2, 8 trials)")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--gemm", choices=["umma", "limb", "core"],
                    help="run one mod-p step GEMM instead: tcgen05 limbs, mma.sync limbs or the CUDA-core tile")
    ap.add_argument("--shape", default="2,1024,512,1024", help="batch,M,N,K of --gemm")
    args = ap.parse_args(argv)
    if args.gemm:
        return gemm(args)

    import torch

    import graphgen
    from paper_2501_00227_gb300 import build
    from paper_2501_00227_gb300 import tn

    build.build()
    n, e = graphgen.by_name(args.graph)
    plan = tn.Plan(n, e, nrepeat=args.nrepeat, seed=1, optimizer=args.order, treesa={"ntrials": 8})
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


def gemm(args) -> int:
    """C[q,b] = A[q,b] B[q,b]^T mod p on random residues, `--repeat` times;
    prints the device time of the last call."""
    import torch

    from paper_2501_00227_gb300 import build
    from paper_2501_00227_gb300 import tn

    build.build()
    batch, m, n, k = (int(v) for v in args.shape.split(","))
    primes = tuple(tn.PRIMES31[: args.primes])
    g = torch.Generator(device="cuda").manual_seed(7)
    pr = torch.tensor(primes, dtype=torch.int64, device="cuda")[:, None]
    a = (torch.randint(0, 2 ** 31 - 1, (len(primes), batch * m * k), dtype=torch.int64, device="cuda", generator=g)
         % pr).to(torch.int32)
    b = (torch.randint(0, 2 ** 31 - 1, (len(primes), batch * n * k), dtype=torch.int64, device="cuda", generator=g)
         % pr).to(torch.int32)
    c = torch.zeros(len(primes) * batch * m * n, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    lk = list(range(int(k).bit_length() - 1))
    lm = [32 + i for i in range(int(m).bit_length() - 1)]
    ln = [64 + i for i in range(int(n).bit_length() - 1)]
    lb = [96 + i for i in range(int(batch).bit_length() - 1)]
    for _ in range(args.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.gemm == "umma":
            tn.tn_modp_gemm_umma(primes, a.data_ptr(), b.data_ptr(), c.data_ptr(), batch, m, n, k, st)
        elif args.gemm == "limb":
            tn.tn_modp_gemm_limb(primes, a.data_ptr(), b.data_ptr(), c.data_ptr(), batch, m, n, k, st)
        else:
            tn.tn_contract_pair("modp", primes, a.data_ptr(), lk + lm + lb, b.data_ptr(), lk + ln + lb,
                                ln + lm + lb, c.data_ptr(), st)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"gemm": args.gemm, "shape": [batch, m, n, k], "primes": len(primes), "last_ms": ms,
                      "modp_tops": len(primes) * batch * m * n * k / (ms * 1e-3) / 1e12}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
