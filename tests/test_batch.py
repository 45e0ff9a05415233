"""Grouped contraction of many independent networks in one persistent launch
(tn_batch_*): every network's result equals its own single contraction and
the oracle; the CUDA-graph replay gives the same results."""
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import build as B
    B.build()
    O.set_threads(os.cpu_count() or 1)


def _instances(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            n = int(rng.integers(15, 31)) * 2
            out.append(g.random_regular3(n, 1000 + i))
        elif kind == 1:
            out.append(g.kings_subgraph(int(rng.integers(4, 9)), 0.8, 2000 + i))
        elif kind == 2:
            out.append(g.erdos_renyi(int(rng.integers(8, 20)), 0.2, 3000 + i))
        else:
            out.append(g.random_regular3(int(rng.integers(15, 26)) * 2, 4000 + i))
    return out


@pytest.mark.parametrize("semiring,primes", [("tropical_i32", None), ("counting", None),
                                             ("modp", tn.PRIMES31[:3]), ("tropical_f32", None)])
def test_batch_equals_single_contractions(semiring, primes):
    graphs = _instances(24, 7)
    plans = [tn.Plan(n, e, nrepeat=2, seed=1) for n, e in graphs]
    try:
        singles = [p.contract(semiring, primes) for p in plans]
        batch = tn.Batch(plans, semiring, primes)
        try:
            for graph_mode in (False, True, True):
                res = batch.run(graph=graph_mode)
                assert res == singles
        finally:
            batch.close()
    finally:
        for p in plans:
            p.close()


def test_batch_against_oracle_and_bruteforce():
    graphs = _instances(12, 11)
    plans = [tn.Plan(n, e, nrepeat=2, seed=3) for n, e in graphs]
    try:
        bc = tn.Batch(plans, "counting")
        bm = tn.Batch(plans, "modp", tn.PRIMES31[:2])
        rc, rm = bc.run(), bm.run(graph=True)
        for (n, e), c, m in zip(graphs, rc, rm):
            o = O.greedy_order(n, e, nrepeat=1, seed=2)
            assert (c["max"], c["count"]) == O.mis_count(n, e, o)
            assert m["residues"] == O.count_modp(n, e, o, tn.PRIMES31[:2])
            if n <= 20:
                poly = O.bruteforce_poly(n, e)
                assert m["crt"] == sum(poly)
        bc.close()
        bm.close()
    finally:
        for p in plans:
            p.close()


def test_batch_of_one_and_mixed_sizes():
    """A batch may mix a large network with tiny ones (the large one's wide
    steps run next to the small networks' tasks)."""
    graphs = [g.random_regular3(100, 1), g.petersen(), g.path(3), g.empty(1), g.random_regular3(40, 2)]
    plans = [tn.Plan(n, e, nrepeat=3, seed=1) for n, e in graphs]
    try:
        for semiring, primes in (("tropical_i32", None), ("counting", None), ("modp", tn.PRIMES31[:3])):
            singles = [p.contract(semiring, primes) for p in plans]
            b = tn.Batch(plans, semiring, primes)
            assert b.run() == singles
            b.close()
        b1 = tn.Batch(plans[:1], "counting")
        assert b1.run() == [plans[0].contract("counting")]
        b1.close()
    finally:
        for p in plans:
            p.close()
