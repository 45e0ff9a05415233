"""Failure detection on the GPU without a fault.  With the executor's wait
limit cut to 1 ns, a contraction whose tasks must wait for earlier steps
gives up instead of waiting: its CTAs stop claiming tasks and return, and
tn_contract reports TN_ETIMEOUT.  The next contraction, with the default
limit, is exact: the context stays usable.  (Named to run after the other
GPU tests; the limit is restored whatever happens.)"""
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_2501_00227_gb300 import build as B
    B.build()


@pytest.mark.gpu
def test_wait_limit_expires_and_the_context_stays_usable():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, e = g.random_regular3(140, 1)
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o)
    try:
        # ~5000 tasks over 14 dependency levels: tasks are claimed while the
        # steps they read are still in flight, so some wait must run out
        assert p.info("counting")["exec_levels"] > 10
        tn.tn_set_wait_timeout_ns(1)
        try:
            with pytest.raises(tn.TNError) as ei:
                p.contract("counting")
        finally:
            tn.tn_set_wait_timeout_ns(0)
        assert ei.value.code == tn.TN_ETIMEOUT
        r = p.contract("counting")
        assert r["status"] == tn.TN_OK and (r["max"], r["count"]) == O.mis_count(n, e, o)
    finally:
        p.close()


@pytest.mark.gpu
def test_static_entry_point_reports_an_expired_wait():
    """tn_contract_static maps an expired dependency wait to TN_ETIMEOUT like
    tn_contract, and its next call (default limit) is exact again."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, e = g.random_regular3(100, 1)
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        info = p.info("counting")
        assert info["exec_levels"] > 10
        assert info["peak_bytes"][tn.TN_COUNTING_TROPICAL - 1] + info["exec_table_bytes"] < tn.TN_STATIC_WORKSPACE_BYTES
        tn.tn_contract_static(p.handle, "counting", None, stream)   # address set-up, default limit
        tn.tn_set_wait_timeout_ns(1)
        try:
            with pytest.raises(tn.TNError) as ei:
                tn.tn_contract_static(p.handle, "counting", None, stream)
        finally:
            tn.tn_set_wait_timeout_ns(0)
        assert ei.value.code == tn.TN_ETIMEOUT
        r = tn.tn_contract_static(p.handle, "counting", None, stream)
        assert r["status"] == tn.TN_OK and (r["max"], r["count"]) == O.mis_count(n, e, o)
    finally:
        p.close()
