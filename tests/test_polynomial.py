"""The independence polynomial I(G, x) = sum_k c_k x^k (Eq. 13) on the GPU:
weighted mod-p evaluation (tn_contract_modp_x) and the finite-field
polynomial (tn_independence_polynomial), against the CPU oracle.

All quantities are integers: residues and coefficients must be equal.
Host-side argument checks run without a GPU.
"""
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
    O.set_threads(os.cpu_count() or 1)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _plan(spec, seed=1):
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=4, seed=seed)
    return n, e, o, tn.Plan(n, e, o)


# ------------------------------------------------------------------ host checks (no GPU)

@pytest.mark.parametrize("primes,degree", [
    ([2147483647], -1),                 # negative degree
    ([2147483647], 11),                 # degree above n = 10
    ([2147483646], 4),                  # not a prime
    ([2147483647, 2147483647], 4),      # repeated prime
    ([7], 6),                           # degree + 1 points are not distinct mod 7
    (list(tn.primes31(33)), 4),         # more than TN_POLY_MAX_PRIMES primes
])
def test_polynomial_rejects_bad_arguments(primes, degree):
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        with pytest.raises(tn.TNError) as ei:
            tn.tn_independence_polynomial(p.handle, primes, degree, 256, 1 << 20, 0)
        assert ei.value.code == tn.TN_EINVAL
    finally:
        p.close()


@pytest.mark.parametrize("primes,xs", [([], []), ([1], [3]), ([1 << 31], [3]), (list(tn.primes31(17)), [1] * 17)])
def test_weighted_evaluation_rejects_bad_slots(primes, xs):
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        with pytest.raises(tn.TNError) as ei:
            tn.tn_contract_modp_x(p.handle, primes, xs, 256, 1 << 20, 0)
        assert ei.value.code == tn.TN_EINVAL
    finally:
        p.close()


def test_primes31_are_the_largest_primes_below_2_31():
    ps = tn.primes31(12)
    assert ps[:8] == tn.PRIMES31
    assert all(a > b for a, b in zip(ps, ps[1:]))
    # every odd number between consecutive listed primes is composite
    for a, b in zip(ps[:4], ps[1:5]):
        for c in range(b + 2, a, 2):
            assert any(c % d == 0 for d in range(3, int(math.isqrt(c)) + 1, 2))


# ------------------------------------------------------------------ GPU parity

@pytest.mark.gpu
def test_petersen_polynomial_printed_gpu():
    """Sec. 5.3 / 6.2: I(Petersen, x) = 1 + 10x + 30x^2 + 30x^3 + 5x^4."""
    _cuda()
    import json
    want = json.load(open(os.path.join(GOLD, "petersen.json")))["independence_polynomial"]
    n, e, o, p = _plan("petersen")
    try:
        assert p.independence_polynomial() == want                      # degree = alpha from the GPU
        assert p.independence_polynomial(primes=tn.PRIMES31[:2], degree=n) == want + [0] * (n + 1 - len(want))
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,nslots", [("petersen", 1), ("reg3:20:1", 5), ("er:18:0.2:3", 13),
                                         ("ksg:6:0.8:2", 16), ("reg3:60:2", 16), ("reg3:100:1", 9)])
def test_weighted_evaluation_matches_oracle(spec, nslots):
    """Every slot (prime, x) against the oracle: repeated primes, x = 0, x = 1,
    x = p - 1 and large x, on general and GEMM-tile steps."""
    _cuda()
    n, e, o, p = _plan(spec)
    rng = np.random.default_rng(nslots)
    primes = [int(tn.PRIMES31[int(i)]) for i in rng.integers(0, 3, size=nslots)]
    xs = [int(v) for v in rng.integers(0, 1 << 31, size=nslots)]
    for i, x in enumerate((0, 1, -1)[:nslots]):
        xs[i] = x % primes[i]
    try:
        assert p.evaluate(primes, xs) == O.evaluate_modp(n, e, o, primes, xs)
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,nprimes", [("reg3:20:2", 1), ("er:16:0.25:1", 1), ("ksg:5:0.8:4", 2),
                                          ("reg3:60:1", 2), ("reg3:100:1", 4)])
def test_polynomial_matches_oracle(spec, nprimes):
    _cuda()
    n, e, o, p = _plan(spec)
    try:
        primes = tn.PRIMES31[:nprimes]
        want = O.independence_polynomial(n, e, o, primes)
        alpha = max(k for k, c in enumerate(want) if c)
        assert p.independence_polynomial(primes=primes, degree=alpha) == want[: alpha + 1]
        if n <= 20:
            assert want == O.bruteforce_poly(n, e)
    finally:
        p.close()


@pytest.mark.gpu
def test_polynomial_full_size_properties():
    """The 140-vertex random 3-regular graph: the recovered coefficients obey
    c_0 = 1, c_1 = n, c_2 = C(n, 2) - m, c_alpha = the number of maximum
    sets (oracle, counting element type), sum = the number of all sets
    (oracle), and I(G, x) at points that are not interpolation nodes equals
    the oracle's weighted contraction there."""
    _cuda()
    n, e, o, p = _plan("reg3:140:1")
    try:
        coeffs = p.independence_polynomial()          # degree = alpha, primes covering 2^n
        alpha, nmax = O.mis_count(n, e, o)
        assert len(coeffs) == alpha + 1 and coeffs[-1] == nmax
        assert coeffs[:3] == [1, n, math.comb(n, 2) - len(e)]
        _, total, _ = O.count_all(n, e, o, tn.PRIMES31[:5])
        assert sum(coeffs) == total
        pr = [tn.PRIMES31[0], tn.PRIMES31[1], tn.PRIMES31[0]]
        xs = [alpha + 7, 1 << 29, 987654321]
        want = O.evaluate_modp(n, e, o, pr, xs)
        assert [sum(c * pow(x, k, q) for k, c in enumerate(coeffs)) % q for q, x in zip(pr, xs)] == want
    finally:
        p.close()


# ------------------------------------------------------------------ k-best properties (Sec. 5.3)

def _all_sizes(n, e):
    """Sizes of all independent sets, by enumeration of every subset."""
    adj = [0] * n
    for u, v in e:
        adj[int(u)] |= 1 << int(v)
        adj[int(v)] |= 1 << int(u)
    out = []
    for s in range(1 << n):
        if all(not (s >> v) & 1 or not (adj[v] & s) for v in range(n)):
            out.append(bin(s).count("1"))
    return sorted(out)


def test_k_best_from_polynomial_petersen_printed():
    """Sec. 5.3 prints SizeMax(2) = [4.0, 4.0] and CountingMax(2) = 30x^3 + 5x^4."""
    import json
    from paper_2501_00227_gb300 import properties as P
    gd = json.load(open(os.path.join(GOLD, "petersen.json")))
    n, e = g.petersen()
    poly = O.bruteforce_poly(n, e)
    assert P.size_max(None, 2, poly) == gd["size_max_2"]
    assert P.counting_max(None, 2, poly) == {int(k): v for k, v in gd["counting_max_2"].items()}
    assert P.counting_max(None, 1, poly) == {gd["mis_count"][0]: gd["mis_count"][1]}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_k_best_matches_enumeration(seed):
    from paper_2501_00227_gb300 import properties as P
    n, e = g.erdos_renyi(12, 0.3, 40 + seed)
    poly = O.bruteforce_poly(n, e)
    sizes = _all_sizes(n, e)
    for k in (1, 2, 3, 7, 50, 10 ** 6):
        assert P.size_max(None, k, poly) == sizes[-k:]
        top = sorted(set(sizes))[-k:]
        assert P.counting_max(None, k, poly) == {s: sizes.count(s) for s in top}


@pytest.mark.gpu
def test_k_best_on_gpu_petersen_and_reg3():
    _cuda()
    from paper_2501_00227_gb300 import properties as P
    n, e, o, p = _plan("petersen")
    try:
        assert P.size_max(p, 2) == [4, 4]
        assert P.counting_max(p, 2) == {3: 30, 4: 5}
    finally:
        p.close()
    n, e, o, p = _plan("reg3:100:2")
    try:
        alpha, nmax = O.mis_count(n, e, o)
        assert P.counting_max(p, 1) == {alpha: nmax}
        want = O.independence_polynomial(n, e, o, tn.PRIMES31[:4], degree=alpha)
        assert P.counting_max(p, 3) == {alpha - j: want[alpha - j] for j in range(3)}
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec", ["empty:6", "path:1", "complete:9", "path:2"])
def test_polynomial_edge_cases(spec):
    """No edges ((1 + x)^n), a single vertex, a clique (1 + n x)."""
    _cuda()
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=1, seed=1) if n + len(e) > 1 else np.zeros((0, 2), dtype=np.int32)
    p = tn.Plan(n, e, o)
    try:
        want = O.bruteforce_poly(n, e)
        alpha = max(k for k, c in enumerate(want) if c)
        assert p.independence_polynomial() == want[: alpha + 1]
        assert p.independence_polynomial(primes=tn.PRIMES31[:1], degree=n) == want
    finally:
        p.close()


@pytest.mark.gpu
def test_k_best_with_vertex_weights():
    """SizeMax(k) / CountingMax(k) over total weights, from the GPU's weighted
    polynomial, against the brute-force weight histogram."""
    _cuda()
    from paper_2501_00227_gb300 import properties as P
    n, e = g.erdos_renyi(16, 0.25, 21)
    w = g.random_weights(n, 4, (0, 1, 2, 3))
    hist = O.bruteforce_weighted_is(n, e, w)
    sizes = sorted(s for s, c in enumerate(hist) for _ in range(c))
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        for k in (1, 3, 10):
            assert P.size_max(p, k, vertex_w=w) == sizes[-k:]
            top = sorted(set(sizes))[-k:]
            assert P.counting_max(p, k, vertex_w=w) == {s: hist[s] for s in top}
    finally:
        p.close()
