"""Serving: requests of different sizes and semirings submitted while others
run, admitted against an HBM budget and grouped into launches; every result
equals the same request contracted alone."""
import time

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


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    kinds = [("tropical_i32", None), ("counting", None), ("modp", tn.PRIMES31[:4])]
    for i in range(count):
        if rng.random() < 0.5:
            n, e = g.random_regular3(int(rng.integers(20, 51)) * 2, 500 + i)
        else:
            n, e = g.kings_subgraph(int(rng.integers(5, 11)), 0.8, 700 + i)
        reqs.append((tn.Plan(n, e, nrepeat=2, seed=1), *kinds[int(rng.integers(0, 3))]))
    return reqs


def _poll_all(server, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < timeout:
        for t, sr in tickets:
            if t not in out:
                r = tn.tn_poll(server, t, sr)
                if r is not None:
                    out[t] = r
        time.sleep(0.0005)
    return out


@pytest.mark.parametrize("budget_mb,inflight", [(4096, 4), (64, 2), (8, 1)])
def test_served_results_equal_alone(budget_mb, inflight):
    reqs = _requests(40, budget_mb)
    alone = [p.contract(sr, pr) for p, sr, pr in reqs]
    server = tn.tn_server_create(budget_mb << 20, inflight)
    try:
        tickets = []
        for i, (p, sr, pr) in enumerate(reqs):
            tickets.append((tn.tn_submit(server, p.handle, sr, pr), sr))
            if i % 7 == 3:
                time.sleep(0.002)            # arrivals while earlier requests run
        got = _poll_all(server, tickets)
        assert len(got) == len(tickets)
        for (t, _), ref in zip(tickets, alone):
            assert got[t] == ref
        # a ticket is handed out once; afterwards it is unknown
        with pytest.raises(tn.TNError):
            tn.tn_poll(server, tickets[0][0], tickets[0][1])
    finally:
        tn.tn_server_destroy(server)
        for p, _, _ in reqs:
            p.close()


def test_request_larger_than_budget_rejected():
    p = tn.Plan(*g.random_regular3(60, 1), nrepeat=1)
    server = tn.tn_server_create(1024, 1)
    try:
        with pytest.raises(tn.TNError) as ei:
            tn.tn_submit(server, p.handle, "counting")
        assert ei.value.code == tn.TN_ENOMEM
    finally:
        tn.tn_server_destroy(server)
        p.close()


def test_completed_tickets_are_reported_once_in_order_of_completion():
    reqs = _requests(30, 11)
    alone = [p.contract(sr, pr) for p, sr, pr in reqs]
    server = tn.tn_server_create(4096 << 20, 3)
    try:
        tickets = {tn.tn_submit(server, p.handle, sr, pr): (i, sr) for i, (p, sr, pr) in enumerate(reqs)}
        seen, t0 = [], time.time()
        while len(seen) < len(tickets) and time.time() - t0 < 60:
            seen += tn.tn_server_completed(server, 7)
            time.sleep(0.0005)
        assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
        assert tn.tn_server_completed(server) == []
        for t in seen:
            i, sr = tickets[t]
            assert tn.tn_poll(server, t, sr) == alone[i]
    finally:
        tn.tn_server_destroy(server)
        for p, _, _ in reqs:
            p.close()
