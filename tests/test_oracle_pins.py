"""Pins for the CPU oracle: every oracle function is checked against something
other than itself -- numbers the paper prints, closed forms, brute force over
all 2^n subsets, and special cases that reduce to a library routine.

No GPU is needed; these run under ``-m "not gpu"``.
"""
import json
import math
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def fib(k):
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def lucas(k):
    a, b = 2, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def poly_summary(poly):
    """(alpha, #max sets, #all sets) from independence-polynomial coefficients."""
    alpha = max(k for k, c in enumerate(poly) if c)
    return alpha, poly[alpha], sum(poly)


# ---------------------------------------------------------------- paper pins

def test_petersen_printed_outputs():
    gd = _gold("petersen.json")
    n, e = g.petersen()
    assert (n, len(e)) == (10, 15)
    assert all(np.bincount(e.reshape(-1), minlength=10) == 3)      # 3-regular
    o = O.greedy_order(n, e, nrepeat=10, seed=1)
    assert O.check_order(n, e, o)
    assert O.mis_size(n, e, o) == gd["mis_size"]
    assert list(O.mis_count(n, e, o)) == gd["mis_count"]
    _, x, _ = O.count_all(n, e, o)
    assert x == gd["count_all"]
    poly = O.bruteforce_poly(n, e)
    assert poly[: len(gd["independence_polynomial"])] == gd["independence_polynomial"]
    assert all(c == 0 for c in poly[len(gd["independence_polynomial"]):])


def test_petersen_greedy_complexity_matches_printed():
    gd = _gold("petersen.json")
    n, e = g.petersen()
    o = O.greedy_order(n, e, nrepeat=10, seed=1)
    tc, sc, rw = O.complexity(n, e, o)
    got = [math.log2(tc), math.log2(sc), math.log2(rw)]
    assert got == pytest.approx(gd["greedy_complexity_log2"], abs=5e-4)


def test_c4_tree_complexity_and_counts():
    gd = _gold("c4_tree.json")
    edges = [(u - 1, v - 1) for u, v in gd["edges_1based"]]
    steps = gd["tree_steps"]
    assert O.check_order(4, edges, steps)
    tc, sc, rw = O.complexity(4, edges, steps)
    assert (tc, sc, rw) == (34.0, 4.0, 69.0)
    assert [math.log2(tc), math.log2(sc), math.log2(rw)] == pytest.approx(gd["tree_log2"], abs=1e-12)
    # flat (unoptimised) contraction: one loop over 4 labels, scalar output,
    # read 4 edge tensors (4 entries) + 4 vertex tensors (2 entries) + 1 output
    assert [math.log2(2 ** 4), math.log2(1), math.log2(4 * 4 + 4 * 2 + 1)] == pytest.approx(gd["flat_log2"])
    assert O.mis_size(4, edges, steps) == gd["mis_size"]
    assert list(O.mis_count(4, edges, steps)) == gd["mis_count"]
    assert O.count_all(4, edges, steps)[1] == gd["count_all"]
    assert O.flat_contract("modp", 4, edges) == [gd["count_all"]]


@pytest.mark.slow
def test_square20_count_matches_paper():
    """The 20x20 square-lattice independent-set count printed in Sec. 5.1,
    recovered exactly from residues modulo 8 primes (prod ~ 2^248 > 2^240)."""
    gd = _gold("square20.json")
    n, e = g.square_lattice(20)
    assert (n, len(e)) == (400, 760)
    o = O.sweep_order(n, e)
    O.set_threads(os.cpu_count() or 1)
    res, x, M = O.count_all(n, e, o, O.PRIMES31)
    assert M > 2 ** 247 and x < M
    assert abs(float(x) - gd["paper_value"]) <= gd["rel_tol"] * gd["paper_value"]


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 13, 30, 62, 91])
def test_path_closed_forms(n):
    nn, e = g.path(n)
    o = O.greedy_order(nn, e, nrepeat=2, seed=n)
    assert O.mis_size(nn, e, o) == (n + 1) // 2
    size, cnt = O.mis_count(nn, e, o)
    assert size == (n + 1) // 2
    assert cnt == (1 if n % 2 else n // 2 + 1)
    _, x, M = O.count_all(nn, e, o)
    assert fib(n + 2) < M and x == fib(n + 2)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 9, 14, 31, 60, 87])
def test_cycle_closed_forms(n):
    nn, e = g.cycle(n)
    o = O.greedy_order(nn, e, nrepeat=2, seed=n)
    size, cnt = O.mis_count(nn, e, o)
    assert size == n // 2 == O.mis_size(nn, e, o)
    assert cnt == (2 if n % 2 == 0 else n)
    _, x, _ = O.count_all(nn, e, o)
    assert x == lucas(n)


def test_long_path_needs_crt():
    """#IS(P_200) = F_202 ~ 2^138: five 31-bit primes recover it, four cannot."""
    n, e = g.path(200)
    o = O.sweep_order(n, e)
    _, x5, M5 = O.count_all(n, e, o, O.PRIMES31[:5])
    assert x5 == fib(202) and M5 > fib(202)
    _, x4, M4 = O.count_all(n, e, o, O.PRIMES31[:4])
    assert M4 < fib(202) and x4 == fib(202) % M4


@pytest.mark.parametrize("n", [1, 2, 5, 12, 20])
def test_empty_graph(n):
    """No edges: every subset is independent (2^n sets, alpha = n, one maximum set).
    Exercises isolated vertices and outer products of disconnected tensors."""
    nn, e = g.empty(n)
    o = O.greedy_order(nn, e, nrepeat=1, seed=3)
    assert O.mis_size(nn, e, o) == n
    assert O.mis_count(nn, e, o) == (n, 1)
    assert O.count_all(nn, e, o)[1] == 2 ** n


@pytest.mark.parametrize("n", [2, 3, 6, 9, 12])
def test_complete_graph(n):
    nn, e = g.complete(n)
    o = O.greedy_order(nn, e, nrepeat=1, seed=4)
    assert O.mis_count(nn, e, o) == (1, n)
    assert O.count_all(nn, e, o)[1] == n + 1


# ---------------------------------------------------------------- brute force

def _small_graphs():
    out = []
    for seed in range(4):
        out.append(("er", g.erdos_renyi(10 + 2 * seed, 0.3, seed)))
    out.append(("reg3:20:1", g.random_regular3(20, 1)))
    out.append(("reg3:16:7", g.random_regular3(16, 7)))
    out.append(("ksg:5", g.kings_subgraph(5, 0.8, 2)))
    out.append(("er-sparse", g.erdos_renyi(18, 0.08, 11)))     # likely disconnected
    return out


@pytest.mark.parametrize("name,graph", _small_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_contraction_equals_bruteforce(name, graph):
    n, e = graph
    poly = O.bruteforce_poly(n, e)
    alpha, nmax, total = poly_summary(poly)
    o = O.greedy_order(n, e, nrepeat=3, seed=5)
    assert O.mis_size(n, e, o) == alpha
    assert O.mis_count(n, e, o) == (alpha, nmax)
    res, x, M = O.count_all(n, e, o, O.PRIMES31[:2])
    assert x == total
    assert res == [total % p for p in O.PRIMES31[:2]]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_flat_contraction_equals_bruteforce(seed):
    """Eq. (8): the tensors B, W and the three element types, with no order."""
    n, e = g.erdos_renyi(11, 0.35, 100 + seed)
    alpha, nmax, total = poly_summary(O.bruteforce_poly(n, e))
    assert O.flat_contract("tropical", n, e) == alpha
    assert O.flat_contract("counting", n, e) == (alpha, nmax)
    assert O.flat_contract("modp", n, e, O.PRIMES31[:3]) == [total % p for p in O.PRIMES31[:3]]


def test_order_invariance():
    """Different binary orders give identical results in all three element types."""
    n, e = g.erdos_renyi(13, 0.25, 42)
    orders = [O.greedy_order(n, e, 1, s) for s in range(3)] + [O.random_order(n, e, s) for s in range(3)]
    ref = None
    for o in orders:
        assert O.check_order(n, e, o)
        r = (O.mis_size(n, e, o), O.mis_count(n, e, o), O.count_modp(n, e, o))
        ref = ref or r
        assert r == ref


def test_invalid_orders_rejected():
    n, e = g.cycle(4)
    good = O.greedy_order(n, e, 1, 0)
    assert O.check_order(n, e, good)
    bad = good.copy(); bad[1, 0] = bad[0, 0]                 # consumes a tensor twice
    assert not O.check_order(n, e, bad)
    assert not O.check_order(n, e, good[:-1])                # incomplete
    bad2 = good.copy(); bad2[0, 1] = 99                      # id that does not exist yet
    assert not O.check_order(n, e, bad2)
    with pytest.raises(O.OracleError):
        O.mis_size(n, e, bad)
    with pytest.raises(O.OracleError):
        O.mis_size(3, [(0, 0)], [])                          # self-loop


# ---------------------------------------------------------------- pair-level pins

def _rand_trop(rng, k, neg_frac=0.2):
    v = rng.integers(0, 50, size=1 << k).astype(np.int64)
    v[rng.random(1 << k) < neg_frac] = O.OR_NEG_INF
    return v


def test_pair_tropical_is_maxplus_matmul():
    """Labels A=(m,k), B=(k,n) -> C=(m,n): the (max,+) matrix product, computed
    here with numpy broadcasting (a library routine, no index bookkeeping)."""
    rng = np.random.default_rng(0)
    A = _rand_trop(rng, 2, 0.0); B = _rand_trop(rng, 2, 0.0)     # labels m=10, k=11 ; k=11, n=12
    C = O.pair_tropical(A, [10, 11], B, [11, 12], [10, 12])
    Am = A.reshape(2, 2).T          # Am[m, k]: bit0 = m
    Bm = B.reshape(2, 2).T          # Bm[k, n]: bit0 = k
    ref = np.max(Am[:, :, None] + Bm[None, :, :], axis=1)     # [m, n]
    assert np.array_equal(C.reshape(2, 2).T, ref)


def test_pair_modp_is_matmul_mod_p():
    rng = np.random.default_rng(1)
    p = O.PRIMES31[1]
    ka, kk, kb = 3, 4, 2
    LA = list(range(ka)) + list(range(100, 100 + kk))            # A bits: m (low), then k
    LB = list(range(100, 100 + kk)) + list(range(200, 200 + kb))  # B bits: k (low), then n
    A = rng.integers(0, p, size=1 << (ka + kk), dtype=np.uint64)
    B = rng.integers(0, p, size=1 << (kk + kb), dtype=np.uint64)
    C = O.pair_modp(A, LA, B, LB, list(range(ka)) + list(range(200, 200 + kb)), p)
    Am = A.reshape(1 << kk, 1 << ka).T.astype(object)   # [m, k]
    Bm = B.reshape(1 << kb, 1 << kk).T.astype(object)   # [k, n]
    ref = (Am.dot(Bm)) % p                               # [m, n]
    assert np.array_equal(C.reshape(1 << kb, 1 << ka).T.astype(object), ref)


def test_pair_counting_bruteforce_and_overflow():
    """Counting pair vs a direct enumeration of the definition on a tiny case,
    including counts whose products exceed 2^64 (kept exactly as 128-bit)."""
    rng = np.random.default_rng(2)
    LA, LB, LC = [1, 2, 3], [2, 3, 4], [1, 4]
    An = rng.integers(0, 3, size=8).astype(np.int64); Bn = rng.integers(0, 3, size=8).astype(np.int64)
    An[5] = O.OR_NEG_INF
    Ac = rng.integers(1, 2 ** 40, size=8, dtype=np.uint64); Bc = rng.integers(1, 2 ** 40, size=8, dtype=np.uint64)
    Ac[5] = 0
    cn, cc = O.pair_counting(An, Ac, LA, Bn, Bc, LB, LC)
    for c in range(4):
        l1, l4 = c & 1, (c >> 1) & 1
        best, cnt = None, 0
        for l2 in (0, 1):
            for l3 in (0, 1):
                ia = l1 | (l2 << 1) | (l3 << 2)
                ib = l2 | (l3 << 1) | (l4 << 2)
                if An[ia] == O.OR_NEG_INF or Bn[ib] == O.OR_NEG_INF:
                    continue
                v = int(An[ia]) + int(Bn[ib]); w = int(Ac[ia]) * int(Bc[ib])
                if best is None or v > best:
                    best, cnt = v, w
                elif v == best:
                    cnt += w
        assert (None if cn[c] == O.OR_NEG_INF else int(cn[c])) == best
        assert cc[c] == cnt
    assert max(cc) > 2 ** 64


def test_pair_label_permutation_invariance():
    """Relabelling the bit order of an input (and permuting its data to match)
    leaves the result unchanged."""
    rng = np.random.default_rng(3)
    LA, LB, LC = [5, 6, 7, 8], [7, 8, 9], [5, 9, 6]
    A = _rand_trop(rng, 4); B = _rand_trop(rng, 3)
    C = O.pair_tropical(A, LA, B, LB, LC)
    perm = [2, 0, 3, 1]                      # new bit j holds old bit perm[j]
    LA2 = [LA[p] for p in perm]
    A2 = np.empty_like(A)
    for x in range(16):
        old = sum(((x >> j) & 1) << perm[j] for j in range(4))
        A2[x] = A[old]
    assert np.array_equal(O.pair_tropical(A2, LA2, B, LB, LC), C)


# ---------------------------------------------------------------- greedy property

def _replay_costs(n, edges, order):
    """For each step: (rank of the chosen output, min rank over label-sharing pairs)."""
    m = len(edges)
    labels = {i: frozenset(map(int, edges[i])) for i in range(m)}
    labels.update({m + v: frozenset([v]) for v in range(n)})
    out = []
    nxt = m + n
    for a, b in order:
        a, b = int(a), int(b)

        def oranks(i, j):
            others = [labels[t] for t in labels if t not in (i, j)]
            used = frozenset().union(*others) if others else frozenset()
            return len((labels[i] | labels[j]) & used), (labels[i] | labels[j]) & used

        live = sorted(labels)
        best = min((oranks(i, j)[0] for x, i in enumerate(live) for j in live[x + 1:]
                    if labels[i] & labels[j]), default=None)
        r, lab = oranks(a, b)
        out.append((r, best))
        del labels[a], labels[b]
        labels[nxt] = lab
        nxt += 1
    return out


def test_oracle_greedy_picks_min_cost_pair():
    """Sec. 4.2.1 with alpha = 0: each step contracts a label-sharing pair whose
    output is as small as any other label-sharing pair's."""
    for spec in ["petersen", "reg3:16:3", "ksg:5:0.8:1"]:
        n, e = g.by_name(spec)
        o = O.greedy_order(n, e, nrepeat=1, seed=7)
        for r, best in _replay_costs(n, e, o):
            assert best is not None and r == best


def test_crt_roundtrip():
    rng = np.random.default_rng(4)
    for k in range(1, 9):
        pr = O.PRIMES31[:k]
        M = math.prod(pr)
        for _ in range(20):
            x = int(rng.integers(0, 2 ** 62)) * int(rng.integers(0, 2 ** 62)) * int(rng.integers(1, 2 ** 62))
            x %= M
            assert O.crt([x % p for p in pr], pr) == (x, M)


# ---------------------------------------------------------------- independence polynomial (Eq. 13)

def test_petersen_polynomial_printed():
    """Sec. 5.3 / Sec. 6.2 print I(Petersen, x) = 1 + 10x + 30x^2 + 30x^3 + 5x^4
    (GraphPolynomial, finite-field method)."""
    gd = _gold("petersen.json")
    n, e = g.petersen()
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    poly = O.independence_polynomial(n, e, o, O.PRIMES31[:1])
    want = gd["independence_polynomial"]
    assert poly == want + [0] * (n + 1 - len(want))
    # the sum of Eq. 13 stops at alpha = 4: five points determine it
    assert O.independence_polynomial(n, e, o, O.PRIMES31[:1], degree=4) == want
    assert O.independence_polynomial(n, e, o, O.PRIMES31[:1], degree=3) != want[:4]


@pytest.mark.parametrize("n", [1, 2, 7, 20, 45])
def test_path_polynomial_closed_form(n):
    """Choosing k pairwise non-adjacent vertices of a path of n vertices:
    c_k = C(n - k + 1, k)."""
    nn, e = g.path(n)
    o = O.sweep_order(nn, e)
    poly = O.independence_polynomial(nn, e, o, O.PRIMES31[:2])
    assert poly == [math.comb(n - k + 1, k) for k in range(n + 1)]


@pytest.mark.parametrize("n", [3, 4, 9, 30])
def test_cycle_polynomial_closed_form(n):
    """On a cycle of n vertices: c_0 = 1, c_k = n / (n - k) * C(n - k, k)."""
    nn, e = g.cycle(n)
    o = O.greedy_order(nn, e, nrepeat=2, seed=n)
    poly = O.independence_polynomial(nn, e, o, O.PRIMES31[:1])
    want = [1] + [n * math.comb(n - k, k) // (n - k) for k in range(1, n)] + [0]
    assert poly == want


@pytest.mark.parametrize("n", [1, 6, 14])
def test_empty_and_complete_polynomials(n):
    """No edges: (1 + x)^n.  Complete graph: 1 + n x."""
    nn, e = g.empty(n)
    o = O.greedy_order(nn, e, nrepeat=1, seed=2)
    assert O.independence_polynomial(nn, e, o, O.PRIMES31[:2]) == [math.comb(n, k) for k in range(n + 1)]
    if n >= 2:
        nn, e = g.complete(n)
        o = O.greedy_order(nn, e, nrepeat=1, seed=2)
        assert O.independence_polynomial(nn, e, o, O.PRIMES31[:1]) == [1, n] + [0] * (n - 1)


@pytest.mark.parametrize("name,graph", _small_graphs()[:5], ids=lambda x: x if isinstance(x, str) else "")
def test_polynomial_equals_bruteforce(name, graph):
    n, e = graph
    o = O.greedy_order(n, e, nrepeat=2, seed=9)
    assert O.independence_polynomial(n, e, o, O.PRIMES31[:1]) == O.bruteforce_poly(n, e)


def test_weighted_evaluation_matches_bruteforce_sum():
    """Vertex weight x in each prime slot: the contraction equals
    sum_S x^|S| mod p over the brute-force size counts, for large x (no
    confusion with the edge entries) and for repeated primes."""
    n, e = g.erdos_renyi(14, 0.25, 3)
    poly = O.bruteforce_poly(n, e)
    o = O.greedy_order(n, e, nrepeat=2, seed=1)
    p0, p1 = O.PRIMES31[0], O.PRIMES31[3]
    primes = [p0, p0, p0, p1, p1]
    xs = [0, 2, p0 - 1, 1 << 30, 12345]
    got = O.evaluate_modp(n, e, o, primes, xs)
    assert got == [sum(c * pow(x, k, p) for k, c in enumerate(poly)) % p for p, x in zip(primes, xs)]
    assert got[0] == 1                                  # only the empty set survives x = 0


def test_interpolation_recovers_random_polynomials():
    """Lagrange interpolation mod p inverts evaluation at distinct points."""
    rng = np.random.default_rng(8)
    p = O.PRIMES31[2]
    for d in (0, 1, 5, 17):
        coeffs = [int(c) for c in rng.integers(0, p, size=d + 1)]
        xs = list(range(3, 3 + d + 1))
        ys = [sum(c * pow(x, k, p) for k, c in enumerate(coeffs)) % p for x in xs]
        assert O.interpolate_modp(xs, ys, p) == coeffs


# ---------------------------------------------------------------- recurrences (sizes beyond brute force)

def _induced(n, e, keep):
    """The subgraph induced by the vertex set `keep`, relabelled 0 .. |keep|-1."""
    idx = {v: i for i, v in enumerate(sorted(keep))}
    sub = [(idx[a], idx[b]) for a, b in np.asarray(e).reshape(-1, 2).tolist() if a in idx and b in idx]
    return len(idx), np.asarray(sub, dtype=np.int32).reshape(-1, 2)


def _poly_of(n, e, seed=1):
    if n == 0:
        return [1]
    o = O.greedy_order(n, e, nrepeat=2, seed=seed)
    return O.independence_polynomial(n, e, o, O.PRIMES31[:2])


def _polymul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_polynomial_vertex_recurrence(seed):
    """Every independent set either avoids v or holds v and nothing of its
    closed neighbourhood: I(G) = I(G - v) + x I(G - N[v]).  Checked on a
    28-vertex graph (2^28 subsets: out of brute-force reach)."""
    n, e = g.erdos_renyi(28, 0.14, 300 + seed)
    rng = np.random.default_rng(seed)
    v = int(rng.integers(0, n))
    nbr = {int(b) for a, b in e.tolist() if a == v} | {int(a) for a, b in e.tolist() if b == v}
    full = _poly_of(n, e, seed)
    minus_v = _poly_of(*_induced(n, e, set(range(n)) - {v}), seed)
    minus_nv = _poly_of(*_induced(n, e, set(range(n)) - {v} - nbr), seed)
    rhs = [0] * (n + 1)
    for k, c in enumerate(minus_v):
        rhs[k] += c
    for k, c in enumerate(minus_nv):
        rhs[k + 1] += c
    assert full == rhs
    # the unit-weight counting contraction agrees with the polynomial's top term
    o = O.greedy_order(n, e, nrepeat=2, seed=seed)
    alpha = max(k for k, c in enumerate(full) if c)
    assert O.mis_count(n, e, o) == (alpha, full[alpha])


def test_polynomial_of_disjoint_union_is_product():
    """Independent sets of a disjoint union are pairs of independent sets:
    I(G + H) = I(G) I(H)."""
    n1, e1 = g.petersen()
    n2, e2 = g.cycle(7)
    e = np.concatenate([e1, e2 + n1])
    assert _poly_of(n1 + n2, e) == _polymul(_poly_of(n1, e1), _poly_of(n2, e2))


@pytest.mark.parametrize("a,b", [(1, 1), (2, 5), (6, 6), (9, 4)])
def test_complete_bipartite_polynomial(a, b):
    """An independent set of K_{a,b} lies inside one side:
    I = (1 + x)^a + (1 + x)^b - 1."""
    e = np.asarray([(i, a + j) for i in range(a) for j in range(b)], dtype=np.int32)
    want = [math.comb(a, k) + math.comb(b, k) - (k == 0) for k in range(a + b + 1)]
    assert _poly_of(a + b, e) == want


@pytest.mark.parametrize("seed", [0, 1])
def test_weighted_is_vertex_recurrence(seed):
    """MWIS(G) = max(MWIS(G - v), w_v + MWIS(G - N[v])), and the numbers of
    optimal sets add up accordingly, on a 26-vertex graph with weights 1..5."""
    n, e = g.erdos_renyi(26, 0.15, 400 + seed)
    w = g.random_weights(n, seed, (1, 2, 3, 4, 5))
    rng = np.random.default_rng(10 + seed)
    v = int(rng.integers(0, n))
    nbr = {int(b) for a, b in e.tolist() if a == v} | {int(a) for a, b in e.tolist() if b == v}

    def best(keep):
        keep = sorted(keep)
        if not keep:
            return 0, 1
        nn, ee = _induced(n, e, set(keep))
        o = O.greedy_order(nn, ee, nrepeat=2, seed=seed)
        return O.weighted_contract("counting", "is", nn, ee, o, vertex_w=w[keep])

    full = best(range(n))
    out_v = best(set(range(n)) - {v})
    in_v = best(set(range(n)) - {v} - nbr)
    in_v = (in_v[0] + int(w[v]), in_v[1])
    top = max(out_v[0], in_v[0])
    assert full == (top, (out_v[1] if out_v[0] == top else 0) + (in_v[1] if in_v[0] == top else 0))
