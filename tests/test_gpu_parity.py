"""GPU parity: libtn's CUDA path (called through the C ABI) against the CPU
oracle, element by element for single steps and exactly for whole networks.

Every quantity here is an integer, so the bar is bit-exact equality:
  - tropical: equal maxima; an entry is "-inf" on the GPU when it is below
    TN_I32_NEG_INF / 2 (int32) or is -inf (float);
  - counting: equal maxima and, for finite entries, counts equal to
    min(exact count, 2^64 - 1) (the GPU saturates, the oracle is 128-bit);
  - mod p: equal residues; CRT integers equal.
"""
import json
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NEG = tn.TN_I32_NEG_INF
U64MAX = 2 ** 64 - 1


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import build as B
    B.build()
    O.set_threads(os.cpu_count() or 1)


def _stream():
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------ tensors

def _to_dev_i32(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda()


def _counting_buffer(vals, counts):
    """Device buffer in the TN_COUNTING_TROPICAL layout: int32 values, then
    uint64 counts at byte offset 8 * ceil(E / 2)."""
    E = len(vals)
    off = 8 * ((E + 1) // 2)
    buf = np.zeros(off + 8 * E, dtype=np.uint8)
    buf[: 4 * E] = np.asarray(vals, dtype=np.int32).view(np.uint8)
    buf[off:] = np.asarray(counts, dtype=np.uint64).view(np.uint8)
    return torch.from_numpy(buf).cuda(), off


def _gpu_pair(semiring, primes, A, LA, B, LB, LC, out_bytes):
    c = torch.zeros(out_bytes, dtype=torch.uint8, device="cuda")
    tn.tn_contract_pair(semiring, primes, A.data_ptr(), LA, B.data_ptr(), LB, LC, c.data_ptr(), _stream())
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _random_labels(rng, ra, rb, rc_frac=0.5, pool=40):
    labels = rng.choice(pool, size=ra + rb, replace=False)
    LA = list(labels[:ra])
    shared = list(rng.choice(LA, size=min(len(LA), max(0, rb // 2)), replace=False)) if LA else []
    LB = shared + list(labels[ra: ra + rb - len(shared)])
    rng.shuffle(LB)
    U = list(dict.fromkeys(LA + LB))
    LC = [l for l in U if rng.random() < rc_frac]
    rng.shuffle(LC)
    return [int(x) for x in LA], [int(x) for x in LB], [int(x) for x in LC]


PAIR_SHAPES = [(0, 0, 0), (1, 1, 1), (3, 2, 0.5), (6, 5, 0.6), (8, 9, 0.5), (10, 10, 0.4), (12, 9, 0.7),
               (14, 14, 0.5), (16, 6, 0.8), (6, 16, 0.3), (18, 18, 0.2)]


@pytest.mark.parametrize("shape", PAIR_SHAPES)
@pytest.mark.parametrize("semiring", ["tropical_i32", "tropical_f32"])
def test_pair_tropical(semiring, shape):
    ra, rb, frac = shape
    rng = np.random.default_rng(ra * 31 + rb)
    LA, LB, LC = _random_labels(rng, ra, rb, frac)
    a = rng.integers(0, 60, size=1 << len(LA)); a[rng.random(a.size) < 0.15] = -1
    b = rng.integers(0, 60, size=1 << len(LB)); b[rng.random(b.size) < 0.15] = -1
    ref = O.pair_tropical(np.where(a < 0, O.OR_NEG_INF, a), LA, np.where(b < 0, O.OR_NEG_INF, b), LB, LC)
    E = 1 << len(LC)
    if semiring == "tropical_i32":
        A = _to_dev_i32(np.where(a < 0, NEG, a)); B = _to_dev_i32(np.where(b < 0, NEG, b))
        got = _gpu_pair(tn.TN_TROPICAL_I32, None, A, LA, B, LB, LC, 4 * E).view(np.int32).astype(np.int64)
        got = np.where(got < NEG // 2, O.OR_NEG_INF, got)
    else:
        fa = np.where(a < 0, -np.inf, a).astype(np.float32); fb = np.where(b < 0, -np.inf, b).astype(np.float32)
        A = torch.from_numpy(fa).cuda(); B = torch.from_numpy(fb).cuda()
        gf = _gpu_pair(tn.TN_TROPICAL_F32, None, A, LA, B, LB, LC, 4 * E).view(np.float32)
        got = np.where(np.isneginf(gf), O.OR_NEG_INF, gf.astype(np.int64))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", PAIR_SHAPES)
@pytest.mark.parametrize("big", [False, True])
def test_pair_counting(shape, big):
    ra, rb, frac = shape
    rng = np.random.default_rng(1000 + ra * 31 + rb + big)
    LA, LB, LC = _random_labels(rng, ra, rb, frac)
    hi = 2 ** 40 if big else 2 ** 12
    a = rng.integers(0, 6, size=1 << len(LA)); ac = rng.integers(1, hi, size=a.size, dtype=np.uint64)
    b = rng.integers(0, 6, size=1 << len(LB)); bc = rng.integers(1, hi, size=b.size, dtype=np.uint64)
    a[rng.random(a.size) < 0.1] = -1; b[rng.random(b.size) < 0.1] = -1
    ac[a < 0] = 0; bc[b < 0] = 0
    rn, rc = O.pair_counting(np.where(a < 0, O.OR_NEG_INF, a), ac, LA, np.where(b < 0, O.OR_NEG_INF, b), bc, LB, LC)
    A, _ = _counting_buffer(np.where(a < 0, NEG, a), ac)
    B, _ = _counting_buffer(np.where(b < 0, NEG, b), bc)
    E = 1 << len(LC)
    off = 8 * ((E + 1) // 2)
    out = _gpu_pair(tn.TN_COUNTING_TROPICAL, None, A, LA, B, LB, LC, off + 8 * E)
    gv = out[: 4 * E].view(np.int32).astype(np.int64)
    gc = out[off: off + 8 * E].view(np.uint64)
    for i in range(E):
        if rn[i] == O.OR_NEG_INF:
            assert gv[i] < NEG // 2
        else:
            assert gv[i] == rn[i]
            assert int(gc[i]) == min(rc[i], U64MAX)


@pytest.mark.parametrize("shape", PAIR_SHAPES)
def test_pair_modp(shape):
    ra, rb, frac = shape
    rng = np.random.default_rng(2000 + ra * 31 + rb)
    LA, LB, LC = _random_labels(rng, ra, rb, frac)
    primes = [tn.PRIMES31[0], tn.PRIMES31[3], 1000003]
    E = 1 << len(LC)
    A = np.stack([rng.integers(0, p, size=1 << len(LA), dtype=np.uint64) for p in primes])
    B = np.stack([rng.integers(0, p, size=1 << len(LB), dtype=np.uint64) for p in primes])
    Ad = torch.from_numpy(A.astype(np.uint32).reshape(-1).view(np.int32)).cuda()
    Bd = torch.from_numpy(B.astype(np.uint32).reshape(-1).view(np.int32)).cuda()
    out = _gpu_pair(tn.TN_COUNT_MODP, primes, Ad, LA, Bd, LB, LC, 4 * E * len(primes)).view(np.uint32)
    for q, p in enumerate(primes):
        ref = O.pair_modp(A[q], LA, B[q], LB, LC, p)
        assert np.array_equal(out[q * E:(q + 1) * E].astype(np.uint64), ref)


# ------------------------------------------------------------------ networks

def _gpu_all(n, e, order, primes=tn.PRIMES31[:3]):
    p = tn.Plan(n, e, order)
    try:
        return {
            "f32": p.contract("tropical_f32")["max"],
            "i32": p.contract("tropical_i32")["max"],
            "cnt": (lambda r: (r["max"], r["count"], r["status"]))(p.contract("counting")),
            "mod": (lambda r: (r["residues"], r["crt"]))(p.contract("modp", primes)),
        }
    finally:
        p.close()


SMALL = ["petersen", "reg3:20:1", "reg3:20:2", "er:16:0.25:1", "er:18:0.1:2", "ksg:5:0.8:4", "path:2",
         "cycle:3", "complete:7", "empty:1", "empty:6", "er:12:0.0:0"]


@pytest.mark.parametrize("spec", SMALL)
def test_network_small_vs_bruteforce(spec):
    n, e = g.by_name(spec)
    poly = O.bruteforce_poly(n, e)
    alpha = max(k for k, c in enumerate(poly) if c)
    total = sum(poly)
    orders = [O.greedy_order(n, e, nrepeat=2, seed=3)]
    if n + len(e) > 1:
        orders.append(tn.tn_order_greedy(n, e, 0.0, 3, 7))
        orders.append(O.random_order(n, e, 5))
    for order in orders:
        r = _gpu_all(n, e, order)
        assert r["f32"] == alpha and r["i32"] == alpha
        assert r["cnt"] == (alpha, poly[alpha], tn.TN_OK)
        assert r["mod"] == ([total % p for p in tn.PRIMES31[:3]], total)


def test_config1_reg20_fp32_and_counting_vs_bruteforce():
    """Random 3-regular graph n = 20: tropical FP32 and (max, count) against
    enumeration of all 2^20 vertex subsets."""
    n, e = g.random_regular3(20, 1)
    poly = O.bruteforce_poly(n, e)
    alpha = max(k for k, c in enumerate(poly) if c)
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        r = p.contract("tropical_f32")
        assert r["max"] == alpha and r["max_f32"] == float(alpha)
        r = p.contract("counting")
        assert (r["max"], r["count"]) == (alpha, poly[alpha])
    finally:
        p.close()


@pytest.mark.parametrize("execu", ["1", "0"])
@pytest.mark.parametrize("spec", ["reg3:100:1", "reg3:100:2", "reg3:100:3", "reg3:140:1", "reg3:140:2", "reg3:140:3"])
def test_config2_regular_vs_oracle(spec, execu, monkeypatch):
    """n = 100 and 140 random 3-regular graphs: tropical int32, counting
    tropical and the count mod three 31-bit primes (+ CRT).  The GPU runs the
    library's greedy order, the oracle its own order: exact semirings give the
    same scalar for any order.  Run through the persistent executor and through
    per-step launches."""
    monkeypatch.setenv("TN_EXEC", execu)
    n, e = g.by_name(spec)
    primes = tn.PRIMES31[:3]
    oo = O.greedy_order(n, e, nrepeat=4, seed=1)
    ref_size = O.mis_size(n, e, oo)
    ref_cnt = O.mis_count(n, e, oo)
    ref_res, ref_x, _ = O.count_all(n, e, oo, primes)
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        assert p.contract("tropical_i32")["max"] == ref_size
        r = p.contract("counting")
        assert (r["max"], r["count"]) == ref_cnt
        r = p.contract("modp", primes)
        assert r["residues"] == ref_res and r["crt"] == ref_x
    finally:
        p.close()


@pytest.mark.parametrize("fill", [0x00, 0xFF, 0xA5])
def test_workspace_contents_do_not_matter(fill):
    """The executor clears its own counters and header at the start of each
    launch (no memset before it): a workspace full of any bytes, or left by a
    different plan, gives the same exact results, launch after launch."""
    n, e = g.random_regular3(100, 2)
    p = tn.Plan(n, e, nrepeat=4, seed=1)
    q = tn.Plan(*g.kings_subgraph(8, 0.8, 1), nrepeat=2, seed=1)
    pr = tn.PRIMES31[:3]
    want_size = O.mis_size(n, e, p.order)
    want_count = O.mis_count(n, e, p.order)
    want_res = O.count_modp(n, e, p.order, pr)
    try:
        need = max(p.workspace_bytes(s, 3) for s in ("tropical_i32", "counting", "modp"))
        need = max(need, q.workspace_bytes("modp", 3))
        ws = torch.full((need,), fill, dtype=torch.uint8, device="cuda")
        for _ in range(2):
            r = tn.tn_contract(p.handle, "tropical_i32", None, ws.data_ptr(), need, _stream())
            assert r["max"] == want_size
            r = tn.tn_contract(p.handle, "counting", None, ws.data_ptr(), need, _stream())
            assert (r["max"], r["count"]) == want_count
            r = tn.tn_contract(p.handle, "modp", pr, ws.data_ptr(), need, _stream())
            assert r["residues"] == want_res
            tn.tn_contract(q.handle, "modp", pr, ws.data_ptr(), need, _stream())
            ws.fill_(fill)
    finally:
        p.close()
        q.close()


def test_square20_count_matches_paper():
    gd = json.load(open(os.path.join(GOLD, "square20.json")))
    n, e = g.square_lattice(20)
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        r = p.contract("modp", tn.PRIMES31)
    finally:
        p.close()
    assert abs(float(r["crt"]) - gd["paper_value"]) <= gd["rel_tol"] * gd["paper_value"]
    # the same integer from the oracle's residues (sweep order, independent code path)
    res, x, _ = O.count_all(n, e, O.sweep_order(n, e), tn.PRIMES31)
    assert r["residues"] == res and r["crt"] == x


def test_counting_overflow_saturates():
    """66 disjoint edges have 2^66 maximum independent sets (one endpoint of
    every edge): the uint64 count saturates and TN_EOVERFLOW is reported;
    63 disjoint edges give 2^63, which fits."""
    pairs = [(2 * i, 2 * i + 1) for i in range(66)]
    n, e = g.canonical(132, pairs)
    p = tn.Plan(n, e, nrepeat=1, seed=0)
    try:
        r = p.contract("counting")
    finally:
        p.close()
    assert r["max"] == 66 and r["status"] == tn.TN_EOVERFLOW and r["count"] == U64MAX
    pairs = [(2 * i, 2 * i + 1) for i in range(63)]
    n, e = g.canonical(126, pairs)
    p = tn.Plan(n, e, nrepeat=1, seed=0)
    try:
        r = p.contract("counting")
    finally:
        p.close()
    assert (r["max"], r["count"], r["status"]) == (63, 2 ** 63, tn.TN_OK)


def test_workspace_too_small_rejected():
    n, e = g.petersen()
    p = tn.Plan(n, e)
    try:
        need = p.workspace_bytes("tropical_i32")
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        with pytest.raises(tn.TNError) as ei:
            tn.tn_contract(p.handle, "tropical_i32", None, ws.data_ptr(), need - 1, _stream())
        assert ei.value.code == tn.TN_ENOMEM
    finally:
        p.close()


# ------------------------------------------------------------------ GEMM-shaped steps, both kernels

def _gemm_labels(rng, nb, nm, nn, nk):
    pool = [int(x) for x in rng.permutation(200)[: nb + nm + nn + nk]]
    bt, M, N, K = pool[:nb], pool[nb:nb + nm], pool[nb + nm:nb + nm + nn], pool[nb + nm + nn:]
    LA = bt + M + K; LB = bt + K + N; LC = bt + M + N
    rng.shuffle(LA); rng.shuffle(LB); rng.shuffle(LC)
    return LA, LB, LC


GEMM_SHAPES = [(0, 7, 8, 11), (2, 8, 9, 6), (1, 9, 3, 7), (0, 3, 3, 14), (4, 4, 4, 4), (0, 8, 8, 2),
               (0, 1, 9, 9), (3, 6, 7, 5), (0, 10, 10, 3), (5, 2, 2, 2)]


@pytest.mark.parametrize("mode", ["auto", "tiled", "naive"])
@pytest.mark.parametrize("shape", GEMM_SHAPES)
def test_gemm_steps_all_semirings(shape, mode, monkeypatch):
    monkeypatch.setenv("TN_KERNEL", mode)
    rng = np.random.default_rng(hash(shape) % 2 ** 32)
    LA, LB, LC = _gemm_labels(rng, *shape)
    ea, eb, E = 1 << len(LA), 1 << len(LB), 1 << len(LC)
    # tropical int32
    a = rng.integers(0, 40, size=ea); a[rng.random(ea) < 0.1] = -1
    b = rng.integers(0, 40, size=eb); b[rng.random(eb) < 0.1] = -1
    ref = O.pair_tropical(np.where(a < 0, O.OR_NEG_INF, a), LA, np.where(b < 0, O.OR_NEG_INF, b), LB, LC)
    got = _gpu_pair(tn.TN_TROPICAL_I32, None, _to_dev_i32(np.where(a < 0, NEG, a)), LA,
                    _to_dev_i32(np.where(b < 0, NEG, b)), LB, LC, 4 * E).view(np.int32).astype(np.int64)
    assert np.array_equal(np.where(got < NEG // 2, O.OR_NEG_INF, got), ref)
    # counting (small counts: no overflow)
    ac = rng.integers(1, 2 ** 10, size=ea, dtype=np.uint64); ac[a < 0] = 0
    bc = rng.integers(1, 2 ** 10, size=eb, dtype=np.uint64); bc[b < 0] = 0
    av = rng.integers(0, 4, size=ea); av[a < 0] = -1
    bv = rng.integers(0, 4, size=eb); bv[b < 0] = -1
    rn, rcnt = O.pair_counting(np.where(av < 0, O.OR_NEG_INF, av), ac, LA, np.where(bv < 0, O.OR_NEG_INF, bv), bc, LB, LC)
    A, _ = _counting_buffer(np.where(av < 0, NEG, av), ac)
    B, _ = _counting_buffer(np.where(bv < 0, NEG, bv), bc)
    off = 8 * ((E + 1) // 2)
    out = _gpu_pair(tn.TN_COUNTING_TROPICAL, None, A, LA, B, LB, LC, off + 8 * E)
    gv = out[: 4 * E].view(np.int32).astype(np.int64)
    gc = out[off: off + 8 * E].view(np.uint64)
    fin = rn != O.OR_NEG_INF
    assert np.array_equal(gv[fin], rn[fin]) and (gv[~fin] < NEG // 2).all()
    assert [int(x) for x in gc[fin]] == [min(c, U64MAX) for c, f in zip(rcnt, fin) if f]
    # mod p, two primes
    primes = [tn.PRIMES31[1], tn.PRIMES31[5]]
    Am = np.stack([rng.integers(0, p, size=ea, dtype=np.uint64) for p in primes])
    Bm = np.stack([rng.integers(0, p, size=eb, dtype=np.uint64) for p in primes])
    out = _gpu_pair(tn.TN_COUNT_MODP, primes, torch.from_numpy(Am.astype(np.uint32).reshape(-1).view(np.int32)).cuda(),
                    LA, torch.from_numpy(Bm.astype(np.uint32).reshape(-1).view(np.int32)).cuda(), LB, LC,
                    4 * E * len(primes)).view(np.uint32)
    for q, p in enumerate(primes):
        assert np.array_equal(out[q * E:(q + 1) * E].astype(np.uint64), O.pair_modp(Am[q], LA, Bm[q], LB, LC, p))


@pytest.mark.parametrize("height", ["1", "4", "64"])
@pytest.mark.parametrize("execu", ["1", "0"])
@pytest.mark.parametrize("mode", ["tiled", "naive", "auto"])
def test_networks_both_kernels(mode, execu, height, monkeypatch):
    """Whole contractions with every step forced onto one kernel, through the
    persistent executor (one launch; tiny steps grouped up to `height` per
    CTA task) and through per-step launches."""
    monkeypatch.setenv("TN_KERNEL", mode)
    monkeypatch.setenv("TN_EXEC", execu)
    monkeypatch.setenv("TN_GROUP_HEIGHT", height)
    for spec in ["reg3:20:1", "ksg:5:0.8:4", "er:16:0.25:1", "empty:3", "er:20:0.12:9"]:
        n, e = g.by_name(spec)
        poly = O.bruteforce_poly(n, e)
        alpha = max(k for k, c in enumerate(poly) if c)
        r = _gpu_all(n, e, tn.tn_order_greedy(n, e, 0.0, 3, 7))
        assert r["i32"] == alpha and r["f32"] == alpha
        assert r["cnt"] == (alpha, poly[alpha], tn.TN_OK)
        assert r["mod"][1] == sum(poly)


@pytest.mark.slow
def test_config4_kings_subgraph_20_vs_oracle():
    """20 x 20 King's subgraph at filling 0.8 (seed 1, ~324 vertices): tropical
    int32, counting tropical and the count modulo four 31-bit primes against
    the oracle on its own greedy order; CRT of 4 residues is the count modulo
    their product (the count itself exceeds that product; six primes hold it)."""
    n, e = g.kings_subgraph(20, 0.8, 1)
    primes = tn.PRIMES31[:4]
    oo = O.greedy_order(n, e, nrepeat=3, seed=1)
    ref_size = O.mis_size(n, e, oo)
    ref_cnt = O.mis_count(n, e, oo)
    ref_res = O.count_modp(n, e, oo, primes)
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        assert p.contract("tropical_i32")["max"] == ref_size
        r = p.contract("counting")
        assert (r["max"], r["count"]) == ref_cnt
        r = p.contract("modp", primes)
        assert r["residues"] == ref_res
        assert r["crt"] == O.crt(ref_res, primes)[0]
    finally:
        p.close()


def test_kings_subgraph_count_exact_with_six_primes():
    """The all-independent-set count of a 12 x 12 King's subgraph, exact from
    6 primes, equals the oracle's (and its float agrees with a 7-prime CRT)."""
    n, e = g.kings_subgraph(12, 0.8, 2)
    oo = O.greedy_order(n, e, nrepeat=2, seed=1)
    res6 = O.count_modp(n, e, oo, tn.PRIMES31[:6])
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        r6 = p.contract("modp", tn.PRIMES31[:6])
        r7 = p.contract("modp", tn.PRIMES31[:7])
    finally:
        p.close()
    assert r6["residues"] == res6
    assert r6["crt"] == r7["crt"]          # 6 primes already exceed the count
