"""Slicing (Sec. 4.2.2): sliced plans, the label picker, slice ranges and the
element-type addition that combines them.  Host logic runs on the CPU (two
gloo ranks combine slice ranges); the GPU tests compare sliced contractions
with the oracle's unsliced ones, and single slices with the oracle on the
graph the slice fixes."""
import math
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

U64 = 2 ** 64 - 1


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_2501_00227_gb300 import build as B
    B.build()
    O.set_threads(os.cpu_count() or 1)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _fixed_graph(n, e, sliced, k):
    """The graph a slice k of an IS network leaves: vertices fixed to 0 are
    removed, vertices fixed to 1 are removed with their neighbours and add 1
    to the size.  None if two vertices fixed to 1 are adjacent."""
    ones = {int(v) for j, v in enumerate(sliced) if (k >> j) & 1}
    gone = {int(v) for v in sliced}
    for u, v in e:
        if int(u) in ones and int(v) in ones:
            return None
        if int(u) in ones:
            gone.add(int(v))
        if int(v) in ones:
            gone.add(int(u))
    keep = [v for v in range(n) if v not in gone]
    idx = {v: i for i, v in enumerate(keep)}
    e2 = [(idx[int(u)], idx[int(v)]) for u, v in e if int(u) in idx and int(v) in idx]
    return len(keep), np.array(e2, dtype=np.int32).reshape(-1, 2), len(ones)


# ------------------------------------------------------------------ host (no GPU)

def test_slice_labels_shrink_the_largest_intermediate():
    n, e = g.random_regular3(60, 4)
    o = tn.tn_order_greedy(n, e, 0.0, 4, 1)
    base = math.log2(O.complexity(n, e, o)[1])
    last = base
    for s in (1, 2, 4, 6):
        labels, (lw, lsc) = tn.tn_slice_labels(n, e, o, s)
        assert len(set(labels.tolist())) == s and all(0 <= v < n for v in labels)
        p = tn.Plan(n, e, o, sliced=labels)
        try:
            info = p.info("tropical_i32")
            assert info["log2_sc"] == pytest.approx(lsc)
            assert lsc <= last and lsc >= base - s
            assert lw == pytest.approx(info["log2_tc"] + s, abs=1e-9)
        finally:
            p.close()
        last = lsc


@pytest.mark.parametrize("sliced", [[0, 0], [-1], [99], list(range(63))])
def test_plan_sliced_rejects_bad_labels(sliced):
    n, e = g.random_regular3(70, 1)
    o = tn.tn_order_greedy(n, e, 0.0, 1, 1)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_plan_sliced(n, e, o, sliced)
    assert ei.value.code == tn.TN_EINVAL


def test_sliced_plans_refuse_generated_leaves():
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=1, seed=1, sliced=[3])
    try:
        with pytest.raises(tn.TNError) as ei:
            tn.tn_contract_async(p.handle, "tropical_i32", None, 256, 1 << 30, 0, 256)
        assert ei.value.code == tn.TN_EINVAL
        with pytest.raises(tn.TNError):
            tn.tn_single_config_max(p.handle, "is", None, None, n, 256, 1 << 30, 0)
    finally:
        p.close()


def test_result_combine_is_the_element_type_addition():
    c = tn.tn_result_combine
    assert c("tropical_i32", {"max": 3}, {"max": 5}) == {"status": 0, "max": 5}
    assert c("tropical_i32", {"max": None}, {"max": 2})["max"] == 2
    assert c("counting", {"max": 4, "count": 7}, {"max": 4, "count": 5})["count"] == 12
    assert c("counting", {"max": 4, "count": 7}, {"max": 5, "count": 1}) == {"status": 0, "max": 5, "count": 1}
    sat = c("counting", {"max": 1, "count": U64 - 1}, {"max": 1, "count": 9})
    assert sat["count"] == U64 and sat["status"] == tn.TN_EOVERFLOW
    p = tn.PRIMES31[0]
    a = {"primes": [p, 7], "residues": [p - 1, 6]}
    b = {"primes": [p, 7], "residues": [5, 3]}
    assert c("modp", a, b)["residues"] == [4, 2]
    with pytest.raises(tn.TNError):
        c("modp", a, {"primes": [p, 11], "residues": [0, 0]})


def _rank_main(rank, world, port, n, e, sliced, out):
    """One gloo rank: brute-force results of its slice range, combined across
    ranks with tn_result_combine."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from paper_2501_00227_gb300 import tn as T
    from paper_2501_00227_gb300 import shard
    nsl = 1 << len(sliced)
    b, en = shard.slice_range(nsl, rank, world)
    acc = {"max": None, "count": 0}
    for k in range(b, en):
        fg = _fixed_graph(n, e, sliced, k)
        if fg is None:
            continue
        n2, e2, ones = fg
        poly = O.bruteforce_poly(n2, e2) if n2 else [1]
        a = max(i for i, c in enumerate(poly) if c)
        acc = T.tn_result_combine("counting", acc, {"max": a + ones, "count": poly[a]})
    parts = [None] * world
    dist.all_gather_object(parts, acc)
    tot = parts[0]
    for x in parts[1:]:
        tot = T.tn_result_combine("counting", tot, x)
    out.put((rank, tot["max"], tot["count"]))
    dist.destroy_process_group()


def test_two_ranks_combine_slice_ranges():
    import multiprocessing as mp
    import socket
    n, e = g.erdos_renyi(14, 0.3, 12)
    sliced = [2, 5, 9]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, e, sliced, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    o = O.greedy_order(n, e, nrepeat=1, seed=1)
    want = O.mis_count(n, e, o)
    assert all((mx, cnt) == want for _, mx, cnt in res)


# ------------------------------------------------------------------ GPU

@pytest.mark.gpu
@pytest.mark.parametrize("spec,s", [("petersen", 2), ("reg3:40:1", 3), ("ksg:8:0.8:2", 4), ("reg3:100:2", 3),
                                    ("er:16:0.2:1", 5)])
def test_sliced_contraction_equals_unsliced(spec, s):
    _cuda()
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o, sliced=s)
    try:
        assert len(p.sliced) == s
        assert p.contract_sliced("tropical_i32")["max"] == O.mis_size(n, e, o)
        r = p.contract_sliced("counting")
        assert (r["max"], r["count"]) == O.mis_count(n, e, o)
        pr = list(tn.PRIMES31[:3])
        assert p.contract_sliced("modp", primes=pr, xs=[1, 1, 1])["residues"] == O.count_modp(n, e, o, pr)
        J = g.random_weights(len(e), s)
        r = p.contract_sliced("counting", "spin", J)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "spin", n, e, o, J)
        w = g.random_weights(n, s, (0, 1, 2, 3))
        assert p.contract_sliced("tropical_f32", "is", vertex_w=w)["max"] == \
            O.weighted_contract("tropical", "is", n, e, o, vertex_w=w)
        half = (1 << s) // 2
        a = p.contract_sliced("counting", slices=(0, half))
        b = p.contract_sliced("counting", slices=(half, 1 << s))
        both = tn.tn_result_combine("counting", a, b)
        assert (both["max"], both["count"]) == O.mis_count(n, e, o)
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,s,fixed", [("reg3:60:2", 3, ()), ("ksg:8:0.8:2", 2, (5,))])
def test_annealed_sliced_plans_equal_the_oracle(spec, s, fixed):
    """Orders and slices from the annealing with slicing (TreeSA, Sec.
    4.2.2) contract to the oracle's unsliced values."""
    _cuda()
    n, e = g.by_name(spec)
    p = tn.Plan(n, e, optimizer="treesa", seed=4,
                treesa={"ntrials": 2, "niters": 5, "nslices": s, "fixed_slices": fixed, "sc_target": 4.0})
    try:
        assert len(p.sliced) == s + len(fixed)
        ref = O.greedy_order(n, e, nrepeat=2, seed=1)
        r = p.contract_sliced("counting")
        assert (r["max"], r["count"]) == O.mis_count(n, e, ref)
        pr = list(tn.PRIMES31[:2])
        assert p.contract_sliced("modp", primes=pr, xs=[1, 1])["residues"] == O.count_modp(n, e, ref, pr)
    finally:
        p.close()


@pytest.mark.gpu
def test_single_slices_match_the_fixed_graphs():
    _cuda()
    n, e = g.erdos_renyi(18, 0.2, 3)
    o = O.greedy_order(n, e, nrepeat=2, seed=1)
    sliced = [1, 4, 7]
    p = tn.Plan(n, e, o, sliced=sliced)
    try:
        for k in range(8):
            r = p.contract_sliced("counting", slices=(k, k + 1))
            fg = _fixed_graph(n, e, sliced, k)
            if fg is None:
                assert r["max"] is None and r["count"] == 0
                continue
            n2, e2, ones = fg
            poly = O.bruteforce_poly(n2, e2) if n2 else [1]
            a = max(i for i, c in enumerate(poly) if c)
            assert (r["max"], r["count"]) == (a + ones, poly[a])
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,s,batch", [("reg3:40:1", 4, 16), ("ksg:8:0.8:2", 5, 8), ("reg3:100:3", 3, 8),
                                          ("er:16:0.2:1", 6, 64)])
def test_batched_slices_equal_one_at_a_time(spec, s, batch):
    """Several slices per executor launch (one merged plan) give the results
    of one launch per slice and of the oracle."""
    _cuda()
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o, sliced=s)
    try:
        for sr, pr in (("tropical_i32", None), ("counting", None), ("modp", list(tn.PRIMES31[:2]))):
            xs = [1] * len(pr) if pr else None
            one = p.contract_sliced(sr, primes=pr, xs=xs, batch=1)
            many = p.contract_sliced(sr, primes=pr, xs=xs, batch=batch)
            assert one == many
        r = p.contract_sliced("counting", batch=batch, slices=(1, (1 << s) - 1))
        ref = p.contract_sliced("counting", batch=1, slices=(1, (1 << s) - 1))
        assert r == ref
        full = p.contract_sliced("counting", batch=batch)
        assert (full["max"], full["count"]) == O.mis_count(n, e, o)
        J = g.random_weights(len(e), s)
        r = p.contract_sliced("counting", "spin", J, batch=batch)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "spin", n, e, o, J)
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,sliced", [("path:3", [0, 1, 2]), ("empty:4", [1, 3]), ("complete:5", [0, 4]),
                                         ("path:1", [0]), ("cycle:6", [0, 1, 2, 3, 4, 5])])
def test_edge_case_slicings(spec, sliced):
    """Every label sliced (all leaves rank 0), isolated vertices, a single
    vertex: the slices still add up to the oracle's counts."""
    _cuda()
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=1, seed=1) if n + len(e) > 1 else np.zeros((0, 2), dtype=np.int32)
    p = tn.Plan(n, e, o, sliced=sliced)
    try:
        r = p.contract_sliced("counting", batch=1)
        poly = O.bruteforce_poly(n, e)
        a = max(k for k, c in enumerate(poly) if c)
        assert (r["max"], r["count"]) == (a, poly[a])
        r = p.contract_sliced("modp", primes=[tn.PRIMES31[0]], xs=[3], batch=1 << len(sliced))
        assert r["residues"] == [sum(c * 3 ** k for k, c in enumerate(poly)) % tn.PRIMES31[0]]
    finally:
        p.close()


def test_result_combine_is_commutative_and_associative():
    """Slice ranges may be combined in any grouping and order."""
    rng = np.random.default_rng(17)
    c = tn.tn_result_combine
    for _ in range(200):
        xs = [{"max": int(rng.integers(0, 4)) if rng.random() < 0.9 else None,
               "count": int(rng.integers(0, 1 << 62))} for _ in range(3)]
        for x in xs:
            if x["max"] is None:
                x["count"] = 0
        a, b, d = xs
        assert c("counting", a, b) == c("counting", b, a)
        assert c("counting", c("counting", a, b), d) == c("counting", a, c("counting", b, d))
        p = [tn.PRIMES31[0], 1000003]
        ra, rb, rd = ({"primes": p, "residues": [int(rng.integers(0, q)) for q in p]} for _ in range(3))
        assert c("modp", ra, rb) == c("modp", rb, ra)
        assert c("modp", c("modp", ra, rb), rd) == c("modp", ra, c("modp", rb, rd))
