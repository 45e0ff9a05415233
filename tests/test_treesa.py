"""The TreeSA order optimiser (Sec. 4.2.2): host code, tested on the CPU.
Its orders must be valid SSA orders, contract to the same results, carry the
complexities the oracle computes for them, never be worse (Eq. 10) than the
greedy tree the first trial starts from, and reach the optimum the paper
prints for the 4-cycle of Sec. 4.1."""
import json
import math
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_2501_00227_gb300 import build as B
    B.build()


def _cost(lg, sc_target=20.0, ws=1.0, wrw=0.2):
    return lg[0] + ws * max(0.0, lg[1] - sc_target) + wrw * lg[2]


def _log2c(n, e, o):
    return tuple(math.log2(x) for x in O.complexity(n, e, o))


def test_c4_reaches_the_printed_optimum():
    """Sec. 4.1: the largest tensor of the 4-cycle network has rank >= 2 in
    any order; TreeSA prints tc = 2^5.087 (34), sc = 2^2, rwc = 2^6.109 (69)."""
    gd = json.load(open(os.path.join(GOLD, "c4_tree.json")))
    edges = [(u - 1, v - 1) for u, v in gd["edges_1based"]]
    o, lg = tn.tn_order_treesa(4, edges, seed=3, ntrials=2)
    assert O.check_order(4, edges, o)
    assert lg[1] == 2.0 and lg[0] <= gd["tree_log2"][0] + 1e-12
    assert lg == pytest.approx(_log2c(4, edges, o), abs=1e-12)


@pytest.mark.parametrize("spec", ["petersen", "reg3:40:1", "er:20:0.2:3", "ksg:6:0.8:2", "square:6", "path:30",
                                  "cycle:25", "empty:5", "complete:6"])
def test_orders_are_valid_and_contract_to_the_same_values(spec):
    n, e = g.by_name(spec)
    o, lg = tn.tn_order_treesa(n, e, seed=2, ntrials=3, nthreads=2)
    assert O.check_order(n, e, o)
    assert lg == pytest.approx(_log2c(n, e, o), abs=1e-9)
    ref = O.greedy_order(n, e, nrepeat=2, seed=1)
    assert O.mis_count(n, e, o) == O.mis_count(n, e, ref)
    assert O.count_modp(n, e, o) == O.count_modp(n, e, ref)


@pytest.mark.parametrize("spec", ["reg3:100:1", "ksg:12:0.8:1", "square:9"])
def test_never_worse_than_its_greedy_start(spec):
    n, e = g.by_name(spec)
    seed = 11
    o, lg = tn.tn_order_treesa(n, e, seed=seed, ntrials=2, niters=10)
    start = tn.tn_order_greedy(n, e, 0.0, 1, seed)      # the first trial's starting tree
    assert _cost(lg) <= _cost(_log2c(n, e, start)) + 1e-9


def test_improves_on_greedy_for_a_3_regular_graph():
    """On a 100-vertex random 3-regular graph the annealed order needs fewer
    multiply-adds than the best of 10 greedy runs."""
    n, e = g.random_regular3(100, 1)
    o, lg = tn.tn_order_treesa(n, e, seed=1, ntrials=4)
    greedy = _log2c(n, e, tn.tn_order_greedy(n, e, 0.0, 10, 1))
    assert lg[0] < greedy[0] - 1.0


def test_trees_and_grids_get_small_intermediates():
    """A path needs rank 1 only; an L x L grid can be swept with rank L."""
    n, e = g.path(40)
    assert tn.tn_order_treesa(n, e, seed=1, ntrials=2)[1][1] <= 1.0
    n, e = g.square_lattice(8)
    assert tn.tn_order_treesa(n, e, seed=1, ntrials=4)[1][1] <= 8.0


def test_deterministic_for_a_seed_and_random_start():
    n, e = g.erdos_renyi(24, 0.2, 5)
    a = tn.tn_order_treesa(n, e, seed=9, ntrials=3, nthreads=3, niters=5)
    b = tn.tn_order_treesa(n, e, seed=9, ntrials=3, nthreads=1, niters=5)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    o, lg = tn.tn_order_treesa(n, e, seed=4, ntrials=2, niters=20, random_init=True)
    assert O.check_order(n, e, o)


@pytest.mark.parametrize("kw", [dict(betas=(1.0, 0.0, 2.0)), dict(betas=(3.0, 0.1, 2.0)), dict(ntrials=0),
                                dict(niters=-1), dict(sc_weight=-1.0)])
def test_rejects_bad_parameters(kw):
    n, e = g.petersen()
    with pytest.raises(tn.TNError) as ei:
        tn.tn_order_treesa(n, e, **kw)
    assert ei.value.code == tn.TN_EINVAL


def test_plan_with_treesa_order():
    n, e = g.random_regular3(60, 2)
    p = tn.Plan(n, e, optimizer="treesa", seed=3, treesa={"ntrials": 2})
    try:
        assert O.check_order(n, e, p.order)
        assert p.info("tropical_i32")["log2_tc"] == pytest.approx(_log2c(n, e, p.order)[0], abs=1e-9)
    finally:
        p.close()


# ------------------------------------------------------------------ slicing inside the annealing

def _plan_log2(n, e, o, sliced):
    """log2 (work of all slices, largest intermediate of one slice, reads and
    writes of all slices) of a sliced plan, from the plan builder."""
    p = tn.Plan(n, e, o, sliced=sliced)
    try:
        info = p.info("tropical_i32")
    finally:
        p.close()
    s = len(sliced)
    return info["log2_tc"] + s, info["log2_sc"], info["log2_rwc"] + s


@pytest.mark.parametrize("spec,s,fixed", [("reg3:60:2", 2, ()), ("reg3:100:1", 4, ()), ("ksg:10:0.8:3", 3, (7,)),
                                          ("petersen", 1, (0, 9)), ("square:6", 0, (14,))])
def test_sliced_orders_are_valid_and_carry_their_complexities(spec, s, fixed):
    n, e = g.by_name(spec)
    o, sl, lg = tn.tn_order_treesa_sliced(n, e, nslices=s, fixed_slices=fixed, sc_target=6.0, seed=2, ntrials=3,
                                          niters=5)
    assert O.check_order(n, e, o)
    assert len(sl) == len(fixed) + s and len(set(sl.tolist())) == len(sl)
    assert tuple(sl[: len(fixed)].tolist()) == tuple(fixed) and all(0 <= v < n for v in sl)
    assert lg == pytest.approx(_plan_log2(n, e, o, sl), abs=1e-9)


@pytest.mark.parametrize("spec,s", [("reg3:100:1", 2), ("reg3:100:1", 4), ("reg3:140:1", 4), ("ksg:12:0.8:1", 4)])
def test_annealed_slices_against_slicing_afterwards(spec, s):
    """Target s below the unsliced annealed tree's largest intermediate, s
    labels to slice: slicing inside the annealing ends with an intermediate
    no larger than slicing the annealed tree afterwards (tn_slice_labels),
    for at most twice its work; on the 3-regular graphs, where every slice
    takes a rank off, it meets the target."""
    n, e = g.by_name(spec)
    sc0 = tn.tn_order_treesa(n, e, seed=1, ntrials=4, niters=10)[1][1]
    o, sl, lg = tn.tn_order_treesa_sliced(n, e, nslices=s, sc_target=sc0 - s, seed=1, ntrials=4, niters=10)
    o0, _ = tn.tn_order_treesa(n, e, sc_target=sc0 - s, seed=1, ntrials=4, niters=10)
    post = tn.tn_slice_labels(n, e, o0, s)[1]
    assert lg[1] <= post[1] and lg[0] <= post[0] + 1.0
    if spec.startswith("reg3"):
        assert lg[1] <= sc0 - s


def test_no_slices_is_the_plain_optimiser():
    n, e = g.erdos_renyi(30, 0.15, 2)
    a = tn.tn_order_treesa(n, e, seed=5, ntrials=2, niters=5)
    o, sl, lg = tn.tn_order_treesa_sliced(n, e, seed=5, ntrials=2, niters=5)
    assert np.array_equal(a[0], o) and a[1] == lg and len(sl) == 0


def test_sliced_deterministic_for_a_seed():
    n, e = g.random_regular3(60, 3)
    a = tn.tn_order_treesa_sliced(n, e, nslices=3, sc_target=5.0, seed=9, ntrials=3, nthreads=3, niters=5)
    b = tn.tn_order_treesa_sliced(n, e, nslices=3, sc_target=5.0, seed=9, ntrials=3, nthreads=1, niters=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


@pytest.mark.parametrize("kw", [dict(nslices=-1), dict(nslices=63), dict(fixed_slices=(3, 3)),
                                dict(fixed_slices=(-1,)), dict(fixed_slices=(10,)), dict(nslices=8, fixed_slices=(1, 2, 3))])
def test_sliced_rejects_bad_arguments(kw):
    n, e = g.petersen()
    with pytest.raises(tn.TNError) as ei:
        tn.tn_order_treesa_sliced(n, e, **kw)
    assert ei.value.code == tn.TN_EINVAL


def test_plan_with_annealed_slices():
    n, e = g.random_regular3(60, 2)
    sc0 = tn.tn_order_treesa(n, e, seed=3, ntrials=2)[1][1]
    p = tn.Plan(n, e, optimizer="treesa", seed=3, treesa={"ntrials": 2, "nslices": 2, "sc_target": sc0 - 2})
    try:
        assert O.check_order(n, e, p.order) and len(p.sliced) == 2
        assert p.info("tropical_i32")["log2_sc"] <= sc0 - 2
    finally:
        p.close()
    with pytest.raises(tn.TNError):
        tn.Plan(n, e, optimizer="treesa", treesa={"nslices": 1}, sliced=[0])


def _replay_sliced(n, e, order, sliced):
    """log2 (tc of all slices, sc of one, rwc of all slices) of an SSA order
    with the labels `sliced` removed from every tensor, replayed from the
    definitions of Sec. 4.1: a contraction's output keeps the labels that a
    tensor outside it still carries; tc = sum 2^|A u B|, sc = max 2^|C|,
    rwc = sum 2^|A| + 2^|B| + 2^|C|; each 2^s-fold for the slices."""
    cut = {int(v) for v in sliced}
    m = len(e)
    live = {i: frozenset(int(x) for x in e[i]) - cut for i in range(m)}
    live.update({m + v: frozenset([v]) - cut for v in range(n)})
    nxt, tc, sc, rw = m + n, 0, 0, 0
    for a, b in np.asarray(order).reshape(-1, 2).tolist():
        A, B = live.pop(a), live.pop(b)
        outside = set().union(*live.values()) if live else set()
        C = (A | B) & outside
        tc += 2 ** len(A | B)
        sc = max(sc, len(C))
        rw += 2 ** len(A) + 2 ** len(B) + 2 ** len(C)
        live[nxt] = frozenset(C)
        nxt += 1
    s = len(cut)
    return math.log2(tc) + s, float(sc), math.log2(rw) + s


@pytest.mark.parametrize("spec,s,fixed", [("reg3:40:3", 3, ()), ("ksg:6:0.8:1", 2, (4, 9)), ("cycle:20", 1, ())])
def test_sliced_complexities_equal_a_plain_replay(spec, s, fixed):
    n, e = g.by_name(spec)
    o, sl, lg = tn.tn_order_treesa_sliced(n, e, nslices=s, fixed_slices=fixed, sc_target=3.0, seed=7, ntrials=2,
                                          niters=5)
    assert lg == pytest.approx(_replay_sliced(n, e, o, sl), abs=1e-9)
    # with nothing sliced the replay is the oracle's complexity
    o0, lg0 = tn.tn_order_treesa(n, e, seed=7, ntrials=2, niters=5)
    assert _replay_sliced(n, e, o0, []) == pytest.approx(_log2c(n, e, o0), abs=1e-9)
