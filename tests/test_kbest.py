"""SizeMax(k) and CountingMax(k) (Sec. 5.3, Table 1) on the GPU: one
executor launch with the k-best element types, compared with the oracle's
element types of the same name element by element (and, on small graphs,
with brute force through the oracle's pins)."""
import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_2501_00227_gb300 import build as B
    B.build()


def test_kbest_arguments_rejected_on_the_host():
    """Argument checks that need no GPU: bad kind, k out of range, sliced plans."""
    n, e = g.by_name("petersen")
    p = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        for kind, k in ((1, 2), (4, 2), ("size_max", 0), ("size_max", tn.TN_KBEST_MAX + 1)):
            with pytest.raises(tn.TNError) as ei:
                tn.tn_kbest_workspace_bytes(p.handle, kind, k)
            assert ei.value.code == tn.TN_EINVAL
        assert tn.tn_kbest_workspace_bytes(p.handle, "counting_max", 4) > 0
    finally:
        p.close()
    ps = tn.Plan(n, e, p.order, sliced=1)
    try:
        with pytest.raises(tn.TNError):
            tn.tn_kbest_workspace_bytes(ps.handle, "size_max", 2)
    finally:
        ps.close()


def _check(n, e, ks, nrepeat=4):
    p = tn.Plan(n, e, nrepeat=nrepeat, seed=1)
    try:
        for k in ks:
            r = p.kbest("size_max", k)
            assert r["status"] == tn.TN_OK
            assert r["values"] == O.size_max_k(n, e, p.order, k), (k, r)
            r = p.kbest("counting_max", k)
            assert r["status"] == tn.TN_OK
            d, c = O.counting_max_k(n, e, p.order, k)
            assert (r["max"], r["counts"]) == (d, c), (k, r, d, c)
    finally:
        p.close()


@pytest.mark.gpu
def test_petersen_printed_kbest():
    n, e = g.by_name("petersen")
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        assert p.kbest("size_max", 2)["values"] == [4, 4]                       # SizeMax(2)
        r = p.kbest("counting_max", 2)
        assert (r["max"], r["counts"]) == (4, [5, 30])                           # 30x^3 + 5x^4
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec", ["er:12:0.3:3", "reg3:16:4", "ksg:5:0.8:1", "path:9", "empty:3", "complete:5",
                                  "cycle:11"])
def test_kbest_small_graphs_all_k(spec):
    _check(*g.by_name(spec), ks=range(1, tn.TN_KBEST_MAX + 1), nrepeat=2)


@pytest.mark.gpu
@pytest.mark.parametrize("spec", ["reg3:60:1", "reg3:100:2", "ksg:10:0.8:3", "ksg:12:0.8:1", "square:8"])
def test_kbest_medium_graphs(spec):
    _check(*g.by_name(spec), ks=(1, 2, 4))


@pytest.mark.gpu
def test_kbest_reg3_140():
    """Full-size headline graph (the GPU executes the same plan as the bench)."""
    _check(*g.random_regular3(140, 1), ks=(2,), nrepeat=10)


@pytest.mark.gpu
def test_kbest_equals_polynomial_route_and_repeats():
    """The k-best contraction equals the top of the exact independence
    polynomial (the GPU's finite-field route), and repeated calls agree."""
    n, e = g.random_regular3(80, 5)
    p = tn.Plan(n, e, nrepeat=4, seed=1)
    try:
        poly = p.independence_polynomial()
        alpha = max(i for i, c in enumerate(poly) if c)
        r1, r2 = p.kbest("counting_max", 4), p.kbest("counting_max", 4)
        assert r1 == r2
        assert r1["max"] == alpha and r1["counts"] == [poly[alpha - t] for t in range(4)]
        sizes = []
        for w in range(alpha, -1, -1):
            sizes += [w] * min(poly[w], 4 - len(sizes))
        assert p.kbest("size_max", 4)["values"] == sizes[:4]
    finally:
        p.close()
