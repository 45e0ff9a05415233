"""CPU oracle for the independent-set tensor-network contraction (arXiv:2501.00227).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the GPU library (``paper_2501_00227_gb300``)
and never imports it; the GPU library never imports this package.

The arithmetic lives in ``tn_oracle.c`` (plain C loops, compiled with gcc into
``oracle/_build/liboracle.so``); this module is argument marshalling plus the
Chinese-remainder recombination (Garner's method, Knuth TAOCP vol. 2 Sec. 4.3.2)
that turns residues modulo several primes into one integer (Sec. 5.3: the
count of all independent sets is an arbitrary-precision integer; the
finite-field idea of Sec. 6.2 gets it from residues).

Parity status of every function here is recorded in ``tests/test_oracle_pins.py``:
each one is pinned by brute force, closed forms or numbers the paper prints.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

OR_NEG_INF = -(2**63)

#: the eight largest primes below 2^31, in decreasing order
PRIMES31 = (2147483647, 2147483629, 2147483587, 2147483579,
            2147483563, 2147483549, 2147483543, 2147483497)


def build(force: bool = False) -> str:
    """Compile ``tn_oracle.c`` with gcc (OpenMP over the output-entry loop)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            lib.or_set_threads.argtypes = [I]
            lib.or_check_order.argtypes = [I, i32p, I, i32p, I]
            lib.or_contract_tropical.argtypes = [I, i32p, I, i32p, I, i64p]
            lib.or_contract_counting.argtypes = [I, i32p, I, i32p, I, i64p, u64p, u64p]
            lib.or_contract_modp.argtypes = [I, i32p, I, i32p, I, u32p, I, u64p]
            lib.or_contract_modp_x.argtypes = [I, i32p, I, i32p, I, u32p, u32p, I, u64p]
            lib.or_contract_weighted.argtypes = [I, I, I, i32p, I, i32p, i32p, i32p, I, u32p, u32p, I,
                                                 i64p, i64p, u64p, u64p, u64p]
            lib.or_contract_kbest.argtypes = [I, I, I, i32p, I, i32p, i32p, i32p, I, I, i64p, i64p, u64p, u64p]
            lib.or_spin_energy.argtypes = [I, i32p, I, i32p, i32p, ctypes.POINTER(ctypes.c_int8)]
            lib.or_spin_energy.restype = ctypes.c_int64
            lib.or_bruteforce_spin.argtypes = [I, i32p, I, i32p, i32p, ctypes.c_int64, u64p]
            lib.or_bruteforce_weighted_is.argtypes = [I, i32p, I, i32p, u64p]
            lib.or_pair_tropical.argtypes = [i64p, i32p, I, i64p, i32p, I, i32p, I, i64p]
            lib.or_pair_counting.argtypes = [i64p, u64p, i32p, I, i64p, u64p, i32p, I, i32p, I, i64p, u64p, u64p]
            lib.or_pair_modp.argtypes = [u64p, i32p, I, u64p, i32p, I, i32p, I, ctypes.c_uint32, u64p]
            lib.or_complexity.argtypes = [I, i32p, I, i32p, I, dp, dp, dp]
            lib.or_greedy_order.argtypes = [I, i32p, I, I, ctypes.c_uint64, i32p]
            lib.or_bruteforce_poly.argtypes = [I, i32p, I, u64p]
            lib.or_flat_contract.argtypes = [I, I, i32p, I, u32p, I, i64p, u64p, u64p, u64p]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _graph(n, edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return int(n), e, int(e.shape[0])


def _order(order):
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1, 2))
    return o, int(o.shape[0])


def set_threads(k: int) -> int:
    """Set the OpenMP thread count of the contraction loops; returns the count in use."""
    return int(_load().or_set_threads(int(k)))


def greedy_order(n, edges, nrepeat: int = 10, seed: int = 0) -> np.ndarray:
    """The oracle's own greedy order (Sec. 4.2.1, alpha = 0): an (n+m-1, 2) SSA list."""
    n, e, m = _graph(n, edges)
    out = np.zeros((max(n + m - 1, 0), 2), dtype=np.int32)
    _check(_load().or_greedy_order(n, _p(e, ctypes.c_int32), m, int(nrepeat), int(seed) & (2**64 - 1),
                                   _p(out, ctypes.c_int32)), "greedy_order")
    return out


def check_order(n, edges, order) -> bool:
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    return _load().or_check_order(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k) == 0


def complexity(n, edges, order):
    """(tc, sc, rwc) of a binary order, as element/operation counts (Sec. 4.1)."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    tc, sc, rw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_load().or_complexity(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k,
                                 ctypes.byref(tc), ctypes.byref(sc), ctypes.byref(rw)), "complexity")
    return tc.value, sc.value, rw.value


def mis_size(n, edges, order):
    """Tropical contraction (Sec. 5.2): the maximum independent set size (None for -inf)."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    r = ctypes.c_int64()
    _check(_load().or_contract_tropical(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k,
                                        ctypes.byref(r)), "contract_tropical")
    return None if r.value == OR_NEG_INF else int(r.value)


def mis_count(n, edges, order):
    """Counting-tropical contraction (Sec. 5.3, CountingMax): (size, exact count)."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    r, lo, hi = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_load().or_contract_counting(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k,
                                        ctypes.byref(r), ctypes.byref(lo), ctypes.byref(hi)),
           "contract_counting")
    size = None if r.value == OR_NEG_INF else int(r.value)
    return size, int(lo.value) | (int(hi.value) << 64)


def count_modp(n, edges, order, primes=PRIMES31[:3]):
    """Number of independent sets modulo each prime (ordinary (+,*) reduced mod p)."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    res = np.zeros(len(pr), dtype=np.uint64)
    _check(_load().or_contract_modp(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k,
                                     _p(pr, ctypes.c_uint32), len(pr), _p(res, ctypes.c_uint64)),
           "contract_modp")
    return [int(x) for x in res]


def evaluate_modp(n, edges, order, primes, xs):
    """The independence polynomial I(G, x) of Eq. 13 evaluated at xs[q]
    modulo primes[q]: the network of Eqs. 6-7 with vertex tensors W = [1, x]
    (e^{beta w} = x) contracted in the ring of integers mod p."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    xv = np.ascontiguousarray(np.asarray(xs, dtype=np.uint32))
    res = np.zeros(len(pr), dtype=np.uint64)
    _check(_load().or_contract_modp_x(n, _p(e, ctypes.c_int32), m, _p(o, ctypes.c_int32), k,
                                       _p(pr, ctypes.c_uint32), _p(xv, ctypes.c_uint32), len(pr),
                                       _p(res, ctypes.c_uint64)), "contract_modp_x")
    return [int(x) for x in res]


def interpolate_modp(xs, ys, p):
    """Coefficients (lowest first) of the polynomial of degree < len(xs)
    through the points (xs[i], ys[i]) modulo the prime p (Lagrange's form,
    expanded term by term)."""
    n = len(xs)
    coeffs = [0] * n
    for i in range(n):
        # basis polynomial prod_{j != i} (x - xs[j]) / (xs[i] - xs[j])
        basis = [1]
        denom = 1
        for j in range(n):
            if j == i:
                continue
            basis = [(a - xs[j] * b) % p for a, b in zip([0] + basis, basis + [0])]
            denom = denom * (xs[i] - xs[j]) % p
        scale = ys[i] * pow(denom, -1, p) % p
        for d in range(n):
            coeffs[d] = (coeffs[d] + scale * basis[d]) % p
    return coeffs


def independence_polynomial(n, edges, order, primes, degree=None):
    """Exact coefficients c_0 .. c_degree of the independence polynomial
    (Eq. 13; the finite-field method of Sec. 6.2): evaluations at x = 1 ..
    degree + 1 modulo each prime, Lagrange interpolation modulo each prime,
    CRT per coefficient.  Exact when prod(primes) exceeds the largest
    coefficient (at most 2^n) and degree >= alpha(G) (the sum of Eq. 13
    stops at alpha(G)); degree defaults to n."""
    d = n if degree is None else int(degree)
    xs = list(range(1, d + 2))
    per_prime = []
    for p in primes:
        ys = [evaluate_modp(n, edges, order, [p], [x])[0] for x in xs]
        per_prime.append(interpolate_modp(xs, ys, int(p)))
    return [crt([c[k] for c in per_prime], primes)[0] for k in range(d + 1)]


PROBLEMS = {"is": 0, "spin": 1}


def _weights(w, size):
    if w is None:
        return None
    a = np.ascontiguousarray(np.asarray(w, dtype=np.int32).reshape(-1))
    if a.size != size:
        raise OracleError("weights: wrong length")
    return a


def _p_opt(a, ctype):
    return None if a is None else _p(a, ctype)


def weighted_contract(kind: str, problem: str, n, edges, order, edge_w=None, vertex_w=None, primes=None, xs=None):
    """Contraction of a weighted network in one element type.
    problem 'is': vertex weights w_v (None: 1) -- tropical: the largest total
    weight of an independent set; counting: (that weight, number of sets);
    modp: sum_S x^{w(S)} per slot (primes[q], xs[q]).
    problem 'spin': the spin glass of Eq. 1 with couplings edge_w (None: 1)
    and fields vertex_w (None: 0) -- tropical: max over sigma of -H;
    counting: (-E_min, ground-state degeneracy); modp: sum_sigma
    y^{H + sum|J| + sum|h|} per slot (primes[q], xs[q])."""
    n, e, m = _graph(n, edges)
    o, k = _order(order)
    J, h = _weights(edge_w, m), _weights(vertex_w, n)
    kid = {"tropical": 1, "counting": 2, "modp": 3}[kind]
    pr = np.ascontiguousarray(np.asarray(primes if primes is not None else [2], dtype=np.uint32))
    xv = None if xs is None else np.ascontiguousarray(np.asarray(xs, dtype=np.uint32))
    t, cn, lo, hi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    res = np.zeros(len(pr), dtype=np.uint64)
    _check(_load().or_contract_weighted(kid, PROBLEMS[problem], n, _p(e, ctypes.c_int32), m,
                                        _p_opt(J, ctypes.c_int32), _p_opt(h, ctypes.c_int32),
                                        _p(o, ctypes.c_int32), k, _p(pr, ctypes.c_uint32),
                                        _p_opt(xv, ctypes.c_uint32), len(pr), ctypes.byref(t), ctypes.byref(cn),
                                        ctypes.byref(lo), ctypes.byref(hi), _p(res, ctypes.c_uint64)),
           "contract_weighted")
    if kind == "tropical":
        return None if t.value == OR_NEG_INF else int(t.value)
    if kind == "counting":
        return (None if cn.value == OR_NEG_INF else int(cn.value)), int(lo.value) | (int(hi.value) << 64)
    return [int(x) for x in res]


#: largest k of the k-best element types
MAX_K = 16


def _kbest(kind, n, edges, order, k, problem, edge_w, vertex_w):
    n, e, m = _graph(n, edges)
    o, ns = _order(order)
    J, h = _weights(edge_w, m), _weights(vertex_w, n)
    vals = np.zeros(max(k, 1), dtype=np.int64)
    lo, hi = np.zeros(max(k, 1), dtype=np.uint64), np.zeros(max(k, 1), dtype=np.uint64)
    d = ctypes.c_int64()
    _check(_load().or_contract_kbest(kind, PROBLEMS[problem], n, _p(e, ctypes.c_int32), m, _p_opt(J, ctypes.c_int32),
                                     _p_opt(h, ctypes.c_int32), _p(o, ctypes.c_int32), ns, int(k),
                                     _p(vals, ctypes.c_int64), ctypes.byref(d), _p(lo, ctypes.c_uint64),
                                     _p(hi, ctypes.c_uint64)), "contract_kbest")
    return vals, d.value, lo, hi


def size_max_k(n, edges, order, k, problem="is", edge_w=None, vertex_w=None):
    """SizeMax(k) (Sec. 5.3, Table 1: ExtendedTropical{k}): the k largest
    total weights over all configurations of the network, counted with
    multiplicity, in decreasing order (None where fewer than k exist).  For
    the unit-weight IS network these are the k largest independent-set sizes;
    for the spin glass, the k largest values of -H."""
    vals, _, _, _ = _kbest(4, n, edges, order, k, problem, edge_w, vertex_w)
    return [None if v == OR_NEG_INF else int(v) for v in vals[:k]]


def counting_max_k(n, edges, order, k, problem="is", edge_w=None, vertex_w=None):
    """CountingMax(k) (Sec. 5.3, Table 1: TruncatedPoly{k}): (d, [c_d,
    c_{d-1}, ..., c_{d-k+1}]) where d is the largest total weight and c_w the
    number of configurations of total weight w (for the IS network, the
    polynomial's k highest-order coefficients, Eq. 13)."""
    _, d, lo, hi = _kbest(5, n, edges, order, k, problem, edge_w, vertex_w)
    return (None if d == OR_NEG_INF else int(d)), [int(a) | (int(b) << 64) for a, b in zip(lo[:k], hi[:k])]


def spin_energy(n, edges, spins, edge_w=None, vertex_w=None):
    """Eq. 1 for one configuration spins in {-1, +1}^n."""
    n, e, m = _graph(n, edges)
    J, h = _weights(edge_w, m), _weights(vertex_w, n)
    sp = np.ascontiguousarray(np.asarray(spins, dtype=np.int8))
    return int(_load().or_spin_energy(n, _p(e, ctypes.c_int32), m, _p_opt(J, ctypes.c_int32),
                                      _p_opt(h, ctypes.c_int32), _p(sp, ctypes.c_int8)))


def spin_shift(n, edges, edge_w=None, vertex_w=None):
    """sum |J| + sum |h|: the largest |H| (J None: 1, h None: 0)."""
    m = len(np.asarray(edges).reshape(-1, 2))
    J = np.ones(m, dtype=np.int64) if edge_w is None else np.asarray(edge_w, dtype=np.int64)
    h = np.zeros(int(n), dtype=np.int64) if vertex_w is None else np.asarray(vertex_w, dtype=np.int64)
    return int(np.abs(J).sum() + np.abs(h).sum())


def bruteforce_spin(n, edges, edge_w=None, vertex_w=None):
    """Energy histogram over all 2^n spin configurations (n <= 30):
    hist[k] = number of sigma with H(sigma) = k - shift."""
    n, e, m = _graph(n, edges)
    J, h = _weights(edge_w, m), _weights(vertex_w, n)
    shift = spin_shift(n, e, edge_w, vertex_w)
    hist = np.zeros(2 * shift + 1, dtype=np.uint64)
    _check(_load().or_bruteforce_spin(n, _p(e, ctypes.c_int32), m, _p_opt(J, ctypes.c_int32),
                                      _p_opt(h, ctypes.c_int32), shift, _p(hist, ctypes.c_uint64)), "bruteforce_spin")
    return shift, [int(x) for x in hist]


def bruteforce_weighted_is(n, edges, vertex_w):
    """hist[k] = number of independent sets of total weight k (weights >= 0)."""
    n, e, m = _graph(n, edges)
    w = _weights(vertex_w, n)
    hist = np.zeros(int(w.sum()) + 1, dtype=np.uint64)
    _check(_load().or_bruteforce_weighted_is(n, _p(e, ctypes.c_int32), m, _p(w, ctypes.c_int32),
                                             _p(hist, ctypes.c_uint64)), "bruteforce_weighted_is")
    return [int(x) for x in hist]


def weighted_polynomial(problem: str, n, edges, order, primes, degree, edge_w=None, vertex_w=None):
    """Coefficients c_0 .. c_degree of the network's generating polynomial:
    'is': c_k = number of independent sets of weight k (weights >= 0);
    'spin': c_k = number of configurations with H = k - sum|J| - sum|h|.
    Evaluations at x = 1 .. degree + 1 modulo each prime, Lagrange
    interpolation, CRT (the finite-field method of Sec. 6.2)."""
    d = int(degree)
    xs = list(range(1, d + 2))
    per_prime = []
    for p in primes:
        ys = weighted_contract("modp", problem, n, edges, order, edge_w, vertex_w, [p] * len(xs), xs)
        per_prime.append(interpolate_modp(xs, ys, int(p)))
    return [crt([c[k] for c in per_prime], primes)[0] for k in range(d + 1)]


def log_partition_function(coeffs, shift, beta):
    """ln Z(beta) for Z = sum_sigma e^{-beta H(sigma)} (Eq. 3 with the energy
    of Eq. 1), from the exact energy histogram coeffs[k] = #{H = k - shift}:
    ln Z = ln sum_k c_k e^{-beta (k - shift)}, summed relative to the largest
    term (float64)."""
    terms = [math.log(c) - beta * (k - shift) for k, c in enumerate(coeffs) if c]
    top = max(terms)
    return top + math.log(sum(math.exp(t - top) for t in terms))


def crt(residues, primes):
    """Garner's mixed-radix recombination: the x in [0, prod p) with x = r_i mod p_i."""
    x, M = 0, 1
    for r, p in zip(residues, primes):
        r, p = int(r), int(p)
        # x_new = x + M * t with t = (r - x) * M^{-1} mod p
        t = ((r - x) * pow(M, -1, p)) % p
        x += M * t
        M *= p
    return x, M


def count_all(n, edges, order, primes=PRIMES31[:3]):
    """(residues, x, M): the independent-set count modulo M = prod(primes)."""
    res = count_modp(n, edges, order, primes)
    x, M = crt(res, primes)
    return res, x, M


def bruteforce_poly(n, edges):
    """Independence polynomial coefficients by enumerating all 2^n subsets (n <= 30)."""
    n, e, m = _graph(n, edges)
    poly = np.zeros(n + 1, dtype=np.uint64)
    _check(_load().or_bruteforce_poly(n, _p(e, ctypes.c_int32), m, _p(poly, ctypes.c_uint64)), "bruteforce")
    return [int(x) for x in poly]


def flat_contract(kind: str, n, edges, primes=(PRIMES31[0],)):
    """Eq. (8) generalised: the whole network as one sum over all 2^n label
    assignments of the product of every edge and vertex tensor entry, in the
    given element type ('tropical', 'counting' or 'modp').  n <= 26."""
    n, e, m = _graph(n, edges)
    kid = {"tropical": 1, "counting": 2, "modp": 3}[kind]
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    v = ctypes.c_int64()
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    res = np.zeros(len(pr), dtype=np.uint64)
    _check(_load().or_flat_contract(kid, n, _p(e, ctypes.c_int32), m, _p(pr, ctypes.c_uint32), len(pr),
                                    ctypes.byref(v), ctypes.byref(lo), ctypes.byref(hi),
                                    _p(res, ctypes.c_uint64)), "flat_contract")
    if kind == "tropical":
        return None if v.value == OR_NEG_INF else int(v.value)
    if kind == "counting":
        return (None if v.value == OR_NEG_INF else int(v.value)), int(lo.value) | (int(hi.value) << 64)
    return [int(x) for x in res]


# ---------------------------------------------------------------------------
# single pairwise contractions (labels: bit j of an entry index <-> label L[j])
# ---------------------------------------------------------------------------

def _labels(L):
    return np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1))


def pair_tropical(A, LA, B, LB, LC):
    """C = (+)_s A (x) B in (max,+); -inf entries are OR_NEG_INF (int64)."""
    a = np.ascontiguousarray(A, dtype=np.int64); b = np.ascontiguousarray(B, dtype=np.int64)
    la, lb, lc = _labels(LA), _labels(LB), _labels(LC)
    c = np.zeros(1 << len(lc), dtype=np.int64)
    _check(_load().or_pair_tropical(_p(a, ctypes.c_int64), _p(la, ctypes.c_int32), len(la),
                                    _p(b, ctypes.c_int64), _p(lb, ctypes.c_int32), len(lb),
                                    _p(lc, ctypes.c_int32), len(lc), _p(c, ctypes.c_int64)), "pair_tropical")
    return c


def pair_counting(An, Ac, LA, Bn, Bc, LB, LC):
    """Counting-tropical pair; returns (values int64, counts as Python ints)."""
    an = np.ascontiguousarray(An, dtype=np.int64); ac = np.ascontiguousarray(Ac, dtype=np.uint64)
    bn = np.ascontiguousarray(Bn, dtype=np.int64); bc = np.ascontiguousarray(Bc, dtype=np.uint64)
    la, lb, lc = _labels(LA), _labels(LB), _labels(LC)
    k = 1 << len(lc)
    cn = np.zeros(k, dtype=np.int64); lo = np.zeros(k, dtype=np.uint64); hi = np.zeros(k, dtype=np.uint64)
    _check(_load().or_pair_counting(_p(an, ctypes.c_int64), _p(ac, ctypes.c_uint64), _p(la, ctypes.c_int32), len(la),
                                    _p(bn, ctypes.c_int64), _p(bc, ctypes.c_uint64), _p(lb, ctypes.c_int32), len(lb),
                                    _p(lc, ctypes.c_int32), len(lc), _p(cn, ctypes.c_int64),
                                    _p(lo, ctypes.c_uint64), _p(hi, ctypes.c_uint64)), "pair_counting")
    return cn, [int(x) | (int(y) << 64) for x, y in zip(lo, hi)]


def pair_modp(A, LA, B, LB, LC, p):
    """Mod-p pair (one prime); residues as uint64."""
    a = np.ascontiguousarray(A, dtype=np.uint64); b = np.ascontiguousarray(B, dtype=np.uint64)
    la, lb, lc = _labels(LA), _labels(LB), _labels(LC)
    c = np.zeros(1 << len(lc), dtype=np.uint64)
    _check(_load().or_pair_modp(_p(a, ctypes.c_uint64), _p(la, ctypes.c_int32), len(la),
                                _p(b, ctypes.c_uint64), _p(lb, ctypes.c_int32), len(lb),
                                _p(lc, ctypes.c_int32), len(lc), ctypes.c_uint32(int(p)),
                                _p(c, ctypes.c_uint64)), "pair_modp")
    return c


def sweep_order(n, edges):
    """A line-sweep SSA order: vertices in id order; each vertex tensor is
    absorbed into a running 'frontier' tensor, then every edge whose other end
    was already absorbed.  On an L x L lattice numbered row-major the frontier
    holds at most L+1 labels (space 2^{L+1})."""
    n, e, m = _graph(n, edges)
    by_late = [[] for _ in range(n)]
    for idx, (u, v) in enumerate(e.tolist()):
        by_late[max(u, v)].append(idx)
    order, front, nxt = [], None, m + n
    for v in range(n):
        if front is None:
            front = m + v
        else:
            order.append((front, m + v)); front = nxt; nxt += 1
        for idx in by_late[v]:
            order.append((front, idx)); front = nxt; nxt += 1
    return np.asarray(order, dtype=np.int32).reshape(-1, 2)


def random_order(n, edges, seed: int):
    """A uniformly random pairing at every step (any two live tensors): valid but
    usually expensive; for order-invariance checks on small graphs only."""
    n, e, m = _graph(n, edges)
    rng = np.random.default_rng(seed)
    live = list(range(m + n))
    order, nxt = [], m + n
    while len(live) > 1:
        i, j = rng.choice(len(live), size=2, replace=False)
        a, b = live[i], live[j]
        order.append((a, b))
        live = [x for x in live if x not in (a, b)] + [nxt]
        nxt += 1
    return np.asarray(order, dtype=np.int32).reshape(-1, 2)
