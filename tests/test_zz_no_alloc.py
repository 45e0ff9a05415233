"""tn_contract_static: the contraction entry point that allocates no device
memory (its workspace is a fixed 64 MiB device array inside libtn), for
callers that cannot call cudaMalloc, e.g. when another component owns device
memory through its own pool or a latency-critical loop must avoid the
synchronisation an allocation can cause.

Checked through the C ABI against tn_contract (the entry point that takes a
caller workspace) on two calls in a row, so that the second call runs on the
array the first one left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import graphgen as g
from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import build as B
    B.build()


def _with_workspace(plan, semiring, primes):
    nprimes = len(primes) if primes else 1
    need = plan.workspace_bytes(semiring, nprimes)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    return tn.tn_contract(plan.handle, semiring, primes, ws.data_ptr(), need,
                          torch.cuda.current_stream().cuda_stream)


CASES = [("petersen", "tropical_i32", None), ("petersen", "counting", None),
         ("reg3:100:1", "tropical_f32", None), ("reg3:100:1", "counting", None),
         ("reg3:100:1", "modp", tn.PRIMES31[:3]), ("reg3:100:2", "tropical_i32", None),
         ("ksg:10:0.8:3", "modp", tn.PRIMES31[:2]), ("empty:5", "counting", None)]


def _static_need(plan, semiring, nprimes):
    info = plan.info(semiring, nprimes)
    ws = info["peak_bytes"][tn.SEMIRINGS[semiring] - 1]
    return (ws + 255) // 256 * 256 + (info["exec_table_bytes"] + 255) // 256 * 256


@pytest.mark.parametrize("spec,semiring,primes", CASES)
def test_static_matches_workspace_entry_point_twice(spec, semiring, primes):
    n, e = g.by_name(spec)
    plan = tn.Plan(n, e, nrepeat=4, seed=1)
    try:
        assert _static_need(plan, semiring, len(primes) if primes else 1) <= tn.TN_STATIC_WORKSPACE_BYTES
        ref = _with_workspace(plan, semiring, primes)
        stream = torch.cuda.current_stream().cuda_stream
        first = tn.tn_contract_static(plan.handle, semiring, primes, stream)
        second = tn.tn_contract_static(plan.handle, semiring, primes, stream)
        assert first == ref
        assert second == ref
    finally:
        plan.close()


def test_static_alternating_plans_keep_results():
    """The array keeps the previous call's contents: alternating two plans
    must still give each plan its own result."""
    stream = torch.cuda.current_stream().cuda_stream
    pa = tn.Plan(*g.random_regular3(100, 3), nrepeat=2, seed=1)
    pb = tn.Plan(*g.kings_subgraph(8, 0.8, 2), nrepeat=2, seed=1)
    try:
        ra = _with_workspace(pa, "counting", None)
        rb = _with_workspace(pb, "counting", None)
        for _ in range(2):
            assert tn.tn_contract_static(pa.handle, "counting", None, stream) == ra
            assert tn.tn_contract_static(pb.handle, "counting", None, stream) == rb
    finally:
        pa.close()
        pb.close()


def test_static_call_allocates_no_device_memory():
    """The defining property: once a first round of calls has looked up the
    array's address and loaded the kernels, further calls change the
    device's free memory by nothing (torch's caching allocator stays idle)."""
    stream = torch.cuda.current_stream().cuda_stream
    plan = tn.Plan(*g.random_regular3(100, 1), nrepeat=2, seed=1)
    kinds = (("counting", None), ("modp", tn.PRIMES31[:3]), ("tropical_i32", None))
    try:
        ref = [tn.tn_contract_static(plan.handle, sr, pr, stream) for sr, pr in kinds]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        again = [tn.tn_contract_static(plan.handle, sr, pr, stream) for sr, pr in kinds]
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert again == ref
    finally:
        plan.close()


def test_static_accepts_exactly_the_plans_the_documented_rule_admits():
    """Plans on both sides of the 64 MiB limit: a call succeeds exactly when
    peak_bytes + exec_table_bytes (each rounded up to 256 bytes) fits."""
    stream = torch.cuda.current_stream().cuda_stream
    seen = set()
    for L in range(10, 19):
        plan = tn.Plan(*g.kings_subgraph(L, 0.8, 1), nrepeat=1, seed=1)
        try:
            fits = _static_need(plan, "counting", 1) <= tn.TN_STATIC_WORKSPACE_BYTES
            if fits:
                assert tn.tn_contract_static(plan.handle, "counting", None, stream) == \
                    _with_workspace(plan, "counting", None)
            else:
                with pytest.raises(tn.TNError) as ei:
                    tn.tn_contract_static(plan.handle, "counting", None, stream)
                assert ei.value.code == tn.TN_ENOMEM
            seen.add(fits)
        finally:
            plan.close()
    assert seen == {True, False}


def test_static_rejects_plans_beyond_the_array():
    n, e = g.kings_subgraph(20, 0.8, 1)
    plan = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        info = plan.info("counting", 1)
        assert info["peak_bytes"][tn.TN_COUNTING_TROPICAL - 1] > tn.TN_STATIC_WORKSPACE_BYTES
        with pytest.raises(tn.TNError) as ei:
            tn.tn_contract_static(plan.handle, "counting", None, torch.cuda.current_stream().cuda_stream)
        assert ei.value.code == tn.TN_ENOMEM
    finally:
        plan.close()
