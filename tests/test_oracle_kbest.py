"""Pins for the oracle's k-best element types (Sec. 5.3, Table 1):
SizeMax(k) (ExtendedTropical{k}, the k largest configuration weights with
multiplicity) and CountingMax(k) (TruncatedPoly{k}, the k highest-order terms
of the polynomial of configuration counts by weight).

Each is checked against something other than itself: the values Sec. 5.3
prints for the Petersen graph, and brute force over all 2^n configurations
(independence polynomial, weighted-set and spin-energy histograms).  No GPU is
needed.
"""
import json
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _top_k_of_hist(hist, k, offset=0):
    """The k largest values of the multiset {w + offset: hist[w] copies}, decreasing."""
    out = []
    for w in range(len(hist) - 1, -1, -1):
        out += [w + offset] * min(int(hist[w]), k - len(out))
        if len(out) == k:
            break
    return out + [None] * (k - len(out))


def _trunc_of_hist(hist, k, offset=0):
    """(d, [c_d, ..., c_{d-k+1}]) of the polynomial sum_w hist[w] x^(w + offset)."""
    top = max(w for w, c in enumerate(hist) if c)
    return top + offset, [int(hist[top - t]) if top - t >= 0 else 0 for t in range(k)]


def test_petersen_printed_kbest():
    gold = json.load(open(os.path.join(GOLD, "petersen.json")))
    n, e = g.by_name("petersen")
    o = O.greedy_order(n, e, nrepeat=2, seed=1)
    assert O.size_max_k(n, e, o, 2) == gold["size_max_2"]               # [4, 4]
    d, c = O.counting_max_k(n, e, o, 2)                                   # 30x^3 + 5x^4
    assert {str(d - t): c[t] for t in range(2)} == {k: v for k, v in gold["counting_max_2"].items()}


def _graphs():
    return [("er", g.erdos_renyi(12, 0.3, 3)), ("er-sparse", g.erdos_renyi(14, 0.1, 8)),
            ("reg3", g.random_regular3(16, 4)), ("ksg", g.kings_subgraph(4, 0.8, 1)),
            ("path", g.path(9)), ("empty", g.empty(3))]


@pytest.mark.parametrize("name,graph", _graphs(), ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_kbest_equals_bruteforce_polynomial(name, graph, k):
    n, e = graph
    poly = O.bruteforce_poly(n, e)
    o = O.greedy_order(n, e, nrepeat=2, seed=k)
    assert O.size_max_k(n, e, o, k) == _top_k_of_hist(poly, k)
    assert O.counting_max_k(n, e, o, k) == _trunc_of_hist(poly, k)


def test_k1_reduces_to_tropical_and_counting():
    n, e = g.random_regular3(40, 2)
    o = O.greedy_order(n, e, nrepeat=2, seed=1)
    assert O.size_max_k(n, e, o, 1) == [O.mis_size(n, e, o)]
    d, c = O.counting_max_k(n, e, o, 1)
    assert (d, c[0]) == O.mis_count(n, e, o)


def test_more_k_than_sets_pads_with_minus_infinity():
    # two isolated vertices: 4 independent sets of sizes 2, 1, 1, 0
    n, e = g.empty(2)
    o = O.greedy_order(n, e, nrepeat=1, seed=0)
    assert O.size_max_k(n, e, o, 6) == [2, 1, 1, 0, None, None]
    assert O.counting_max_k(n, e, o, 4) == (2, [1, 2, 1, 0])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weighted_is_kbest_equals_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n, e = g.erdos_renyi(12, 0.3, 20 + seed)
    w = rng.integers(0, 5, size=n)
    hist = O.bruteforce_weighted_is(n, e, w)
    o = O.greedy_order(n, e, nrepeat=2, seed=seed)
    assert O.size_max_k(n, e, o, 6, "is", None, w) == _top_k_of_hist(hist, 6)
    assert O.counting_max_k(n, e, o, 4, "is", None, w) == _trunc_of_hist(hist, 4)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spin_glass_kbest_equals_bruteforce(seed):
    """Spin glass of Eq. 1: the k largest values of -H and the counts of -H
    at the top orders equal the brute-force energy histogram read from its
    low-energy end."""
    rng = np.random.default_rng(seed)
    n, e = g.random_regular3(12, 30 + seed)
    J = rng.choice([-1, 1], size=len(e))
    h = rng.integers(-1, 2, size=n)
    shift, hist = O.bruteforce_spin(n, e, J, h)   # hist[k]: H = k - shift
    neg = hist[::-1]                              # neg[k]: -H = k - shift
    o = O.greedy_order(n, e, nrepeat=2, seed=seed)
    assert O.size_max_k(n, e, o, 5, "spin", J, h) == _top_k_of_hist(neg, 5, -shift)
    assert O.counting_max_k(n, e, o, 4, "spin", J, h) == _trunc_of_hist(neg, 4, -shift)


def test_kbest_order_invariance():
    n, e = g.erdos_renyi(14, 0.22, 77)
    orders = [O.greedy_order(n, e, 1, s) for s in range(2)] + [O.random_order(n, e, s) for s in range(2)]
    ref = None
    for o in orders:
        r = (O.size_max_k(n, e, o, 4), O.counting_max_k(n, e, o, 3))
        ref = ref or r
        assert r == ref
