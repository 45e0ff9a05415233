"""The packed tiles: (max,+) on int32 tropical networks (two 16-bit terms per
__viaddmax_s16x2) and the counting tile on half-precision value pairs,
against the oracle and against the 32-bit tiles.

The executor takes the packed (max,+) tile when every finite value of the
network is at most 4095 in magnitude (unit-weight networks with n <= 4095
vertices) and the packed counting tile when it is at most 1024 (n <= 1024).
These tests push tile operands close to those bounds (a random 3-regular core
whose vertices carry many pendant vertices: every pendant absorbed into its
core vertex's tensor adds one to the values the core's GEMM-shaped steps see),
check one vertex past each bound (the 32-bit tiles run), and compare the two
kinds of tiles on the same plans (TN_PACKED=0 in a child process keeps the
32-bit tiles).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import build as B
    B.build()
    O.set_threads(os.cpu_count() or 1)


def _pendant_network(core_n, seed, pendants):
    """Random 3-regular core on core_n vertices; core vertex v gets
    pendants[v] extra vertices joined to v only.  Returns (n, edges, order):
    the order absorbs every pendant (its edge, then its vertex) into its core
    vertex's tensor, then contracts the core along the core's greedy order."""
    n0, e0 = g.random_regular3(core_n, seed)
    pairs = [tuple(int(x) for x in p) for p in e0]
    owner = []
    nxt = n0
    for v in range(n0):
        for _ in range(int(pendants[v])):
            pairs.append((v, nxt))
            owner.append(v)
            nxt += 1
    n, e = g.canonical(nxt, pairs)
    m = len(e)
    T = n + m
    eid = {(int(a), int(b)): i for i, (a, b) in enumerate(e)}
    order = []
    acc = {v: m + v for v in range(n0)}  # tensor id holding core vertex v's absorbed part

    def step(x, y):
        order.append((x, y))
        return T + len(order) - 1

    for k, v in enumerate(owner):
        u = n0 + k
        t = step(eid[(v, u)], m + u)  # the pendant's edge with the pendant's vertex: a tensor on v
        acc[v] = step(acc[v], t)
    core = tn.tn_order_greedy(n0, e0, 0.0, 4, seed)
    m0, T0 = len(e0), n0 + len(e0)
    base = len(order)

    def full_id(x):
        if x < m0:
            a, b = (int(c) for c in e0[x])
            return eid[(min(a, b), max(a, b))]
        if x < T0:
            return acc[x - m0]
        return T + base + (x - T0)

    for a, b in core:
        step(full_id(int(a)), full_id(int(b)))
    return n, e, np.asarray(order, dtype=np.int32)


def _tiled_steps(plan):
    si = tn.tn_plan_step_info(plan.handle, "tropical_i32", 1)
    return int((si[:, 2] == 1).sum())


@pytest.mark.parametrize("total,seed", [(4095, 1), (4096, 2), (3000, 3)])
def test_values_near_the_packed_bound(total, seed):
    core = 100
    rng = np.random.default_rng(seed)
    extra = total - core
    cuts = np.sort(rng.integers(0, extra + 1, size=core - 1))
    pendants = np.diff(np.concatenate([[0], cuts, [extra]]))
    n, e, order = _pendant_network(core, seed, pendants)
    assert n == total
    assert O.check_order(n, e, order)
    p = tn.Plan(n, e, order)
    try:
        assert _tiled_steps(p) > 0, "the core must contract through GEMM tiles"
        want = O.mis_size(n, e, p.order)
        assert want >= extra  # all pendants together are independent: the values are large
        got = p.contract("tropical_i32")["max"]
        assert got == want
    finally:
        p.close()


@pytest.mark.parametrize("total,seed", [(1024, 4), (1025, 5), (700, 6)])
def test_counting_values_near_the_half_precision_bound(total, seed):
    """The packed counting tile (values as IEEE half pairs) runs for n <= 1024,
    where every sum of two finite values is an exact half; one vertex more
    keeps the 32-bit tile."""
    core = 100
    rng = np.random.default_rng(seed)
    extra = total - core
    cuts = np.sort(rng.integers(0, extra + 1, size=core - 1))
    pendants = np.diff(np.concatenate([[0], cuts, [extra]]))
    n, e, order = _pendant_network(core, seed, pendants)
    p = tn.Plan(n, e, order)
    try:
        assert _tiled_steps(p) > 0
        want = O.mis_count(n, e, p.order)
        assert want[0] >= extra
        r = p.contract("counting")
        assert (r["max"], r["count"]) == want
    finally:
        p.close()


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch, graphgen
from paper_2501_00227_gb300 import tn
out = {}
for spec in sys.argv[2:]:
    p = tn.Plan(*graphgen.by_name(spec), nrepeat=4, seed=1)
    c = p.contract("counting")
    out[spec] = [p.contract("tropical_i32")["max"], c["max"], c["count"]]
    p.close()
print(json.dumps(out))
"""


def test_packed_and_32bit_tiles_agree():
    specs = ["reg3:100:1", "reg3:140:2", "ksg:12:0.8:1", "ksg:14:0.8:2", "er:40:0.15:3", "square:12"]
    env = dict(os.environ)
    env["TN_PACKED"] = "0"
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, *specs], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    int32_tile = json.loads(r.stdout.strip().splitlines()[-1])
    for spec in specs:
        n, e = g.by_name(spec)
        p = tn.Plan(n, e, nrepeat=4, seed=1)
        try:
            got = p.contract("tropical_i32")["max"]
            c = p.contract("counting")
            assert got == int32_tile[spec][0] == O.mis_size(n, e, p.order), spec
            assert [c["max"], c["count"]] == int32_tile[spec][1:], spec
            assert (c["max"], c["count"]) == O.mis_count(n, e, p.order), spec
        finally:
            p.close()
